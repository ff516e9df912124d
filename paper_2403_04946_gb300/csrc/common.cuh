// Shared device helpers: complex float64 arithmetic on double2, block
// reductions, and a bounded grid-wide barrier for cooperative launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

typedef double2 cplx;

#define HD __host__ __device__ __forceinline__
#define DV __device__ __forceinline__

HD cplx mk(double re, double im) { return make_double2(re, im); }
HD cplx cadd(cplx a, cplx b) { return mk(a.x + b.x, a.y + b.y); }
HD cplx csub(cplx a, cplx b) { return mk(a.x - b.x, a.y - b.y); }
HD cplx cscale(cplx a, double s) { return mk(a.x * s, a.y * s); }
HD cplx cconj(cplx a) { return mk(a.x, -a.y); }
HD cplx cmul(cplx a, cplx b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
HD cplx cmulc(cplx a, cplx b) { return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
HD double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
// acc + a * b
DV cplx cfma(cplx a, cplx b, cplx acc) {
  return mk(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc + conj(a) * b
DV cplx cfmac(cplx a, cplx b, cplx acc) {
  return mk(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
HD cplx cinv(cplx a) {
  double s = 1.0 / (a.x * a.x + a.y * a.y);
  return mk(a.x * s, -a.y * s);
}

// Single-precision complex (mixed-precision trailing updates and products).
typedef float2 cplxf;
HD cplxf mkf(float re, float im) { return make_float2(re, im); }
HD cplxf tof(cplx a) { return make_float2((float)a.x, (float)a.y); }
HD cplx tod(cplxf a) { return make_double2((double)a.x, (double)a.y); }
// acc + a * b
DV cplxf cfmaf(cplxf a, cplxf b, cplxf acc) {
  return mkf(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
// acc + conj(a) * b
DV cplxf cfmacf(cplxf a, cplxf b, cplxf acc) {
  return mkf(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}

// Double-float arithmetic: a value is hi + lo with hi, lo in FP32 (about 48
// significant bits).  Used by the mixed-precision trailing updates: the FP32
// pipe is 64 times the FP64 pipe on this GPU, so ~13 FP32 operations per
// real multiply-add still beat one FP64 FMA by a wide margin.
struct df2 {   // complex double-float: (re.hi, im.hi, re.lo, im.lo)
  float rh, ih, rl, il;
};
HD df2 df_zero() { return df2{0.f, 0.f, 0.f, 0.f}; }
HD df2 df_from(cplx a) {
  const float rh = (float)a.x, ih = (float)a.y;
  return df2{rh, ih, (float)(a.x - (double)rh), (float)(a.y - (double)ih)};
}
HD cplx df_to(df2 a) { return make_double2((double)a.rh + (double)a.rl, (double)a.ih + (double)a.il); }
// (hi, lo) += a * b for double-float reals a = (ah, al), b = (bh, bl):
// exact product of the high parts (TwoProduct with an FMA), exact sum
// (TwoSum), the low-order cross terms added to lo.
DV void df_mac(float& hi, float& lo, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  const float pe = fmaf(ah, bh, -p);
  const float cross = fmaf(ah, bl, al * bh);
  const float s = hi + p;
  const float bb = s - hi;
  const float se = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += se + pe + cross;
}
// acc += conj(a) * b
DV void df_cmac_conj(df2& acc, const df2& a, const df2& b) {
  df_mac(acc.rh, acc.rl, a.rh, a.rl, b.rh, b.rl);
  df_mac(acc.rh, acc.rl, a.ih, a.il, b.ih, b.il);
  df_mac(acc.ih, acc.il, a.rh, a.rl, b.ih, b.il);
  df_mac(acc.ih, acc.il, -a.ih, -a.il, b.rh, b.rl);
}
// acc += a * b
DV void df_cmac(df2& acc, const df2& a, const df2& b) {
  df_mac(acc.rh, acc.rl, a.rh, a.rl, b.rh, b.rl);
  df_mac(acc.rh, acc.rl, -a.ih, -a.il, b.ih, b.il);
  df_mac(acc.ih, acc.il, a.rh, a.rl, b.ih, b.il);
  df_mac(acc.ih, acc.il, a.ih, a.il, b.rh, b.rl);
}

// a + b for complex double-float values (TwoSum on each part, then
// renormalised).
DV void df_add_part(float& h, float& l, float bh, float bl) {
  const float s = h + bh;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (bh - bb) + l + bl;
  h = s + e;
  l = e - (h - s);
}
DV df2 df_cadd(df2 a, const df2& b) {
  df_add_part(a.rh, a.rl, b.rh, b.rl);
  df_add_part(a.ih, a.il, b.ih, b.il);
  return a;
}

// Sum over a warp (all 32 lanes active).
DV double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
DV cplx warp_sum(cplx v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}
DV float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum; `red` needs blockDim.x/32 slots.  Every thread
// gets the result.
template <typename T>
DV T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T s = red[0];
  for (int i = 1; i < nw; ++i) s = s + red[i];
  __syncthreads();
  return s;
}
template <>
DV cplx block_sum<cplx>(cplx v, cplx* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  cplx s = red[0];
  for (int i = 1; i < nw; ++i) s = cadd(s, red[i]);
  __syncthreads();
  return s;
}

DV uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier state (device memory).  `count` is zeroed by the host before
// every cooperative launch; `err` records an expired wait.
struct GridBar {
  unsigned int count;
  unsigned int limit_us;  // wait limit in microseconds (0: kBarrierTimeoutNs)
  int err;                // nonzero after a wait expired
  int pad;
};

// Barrier across all CTAs of a cooperative launch (co-residency guaranteed
// by cudaLaunchCooperativeKernel).  The arrival counter only grows: on its
// k-th barrier every CTA adds one and waits until the counter reaches
// k * gridDim, so no CTA has to reset anything between barriers (one atomic
// and one polled load per CTA per barrier).  Every wait is bounded: after
// kBarrierTimeoutNs of wall time (or the context's limit_us) the CTA records
// the expiry in err and leaves; callers check grid_failed() and return
// early.
constexpr uint64_t kBarrierTimeoutNs = 4000000000ull;  // 4 s

struct GridSync {
  GridBar* bar;
  unsigned int target;  // used by thread 0 of each CTA
};

// Arrival is a release reduction (the CTA's writes, ordered before it by
// the CTA barrier, become visible with it; the arriving thread does not
// wait for a returned value), polling an acquire load: one L2 round trip
// after the last arrival instead of a fence, a returning atomic and a
// trailing fence.
DV void bar_arrive_release(unsigned int* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}
DV unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

DV void grid_sync(GridSync& gs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* verr = &gs.bar->err;
    gs.target += gridDim.x * gridDim.y * gridDim.z;
    if (*verr == 0) {
      bar_arrive_release(&gs.bar->count);
      const unsigned int lim = *((volatile unsigned int*)&gs.bar->limit_us);
      const uint64_t limit_ns = lim ? (uint64_t)lim * 1000ull : kBarrierTimeoutNs;
      uint64_t t0 = 0;
      unsigned int spins = 0;
      while ((int)(ld_acquire_gpu(&gs.bar->count) - gs.target) < 0) {
        if (((++spins) & 31u) == 0u) {
          if (*verr != 0) break;
          const uint64_t now = global_ns();
          if (t0 == 0) {
            t0 = now;
          } else if (now - t0 > limit_ns) {
            atomicExch(&gs.bar->err, 1);
            break;
          }
        }
        __nanosleep(32);
      }
    }
  }
  __syncthreads();
}

DV bool grid_failed(const GridBar* bar) {
  return *((volatile const int*)&bar->err) != 0;
}
