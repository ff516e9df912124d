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

// Conversions between FP64 and double-float by integer arithmetic on the
// IEEE bit patterns (on this GPU an FP64 conversion, scaling or addition
// occupies the narrow FP64 pipe; these use the integer and FP32 pipes).
// (double)f * 2^E (negated if neg) from the bit pattern of f: sign, exponent
// rebiased from 127 to 1023 plus E, significand shifted into place.  Zero
// and FP32 subnormals give 0 (a subnormal low part sits below 2^-149 of its
// high part); an exponent outside the double range saturates to 0 or inf.
DV double f2d_scaled(float f, int E, int neg) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e8 = (u >> 23) & 0xFFu;
  if (e8 == 0) return 0.0;
  const long long sgn = (long long)((u >> 31) ^ (unsigned)neg) << 63;
  const int e11 = (int)e8 - 127 + 1023 + E;
  if (e11 <= 0) return 0.0;
  if (e11 >= 2047) return __longlong_as_double(sgn | (0x7FFll << 52));
  return __longlong_as_double(sgn | ((long long)e11 << 52) | ((long long)(u & 0x7FFFFFu) << 29));
}

// 2^d as a float for -126 <= d <= 127 (exact), 0 below: multiplying by it
// scales exactly while the result stays normal.
DV float pow2f(int d) { return d >= -126 ? __int_as_float((127 + d) << 23) : 0.f; }

// x 2^-E as a double-float pair (hi, lo): hi is the 53-bit significand
// rounded to 24 bits, lo the remainder (|lo| <= ulp(hi) / 2, itself rounded
// to 24 bits).  Values whose hi part would fall below the FP32 normal range
// (|x 2^-E| < 2^-126), zeros and FP64 subnormals give (0, 0).
DV void df_split_scaled(double x, int E, float& hi, float& lo) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const int e = ex - 1023 - E;  // |x| 2^-E = M 2^(e - 52), M in [2^52, 2^53)
  if (ex == 0 || e < -126) {
    hi = 0.f;
    lo = 0.f;
    return;
  }
  const long long M = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
  long long Mh = (M + (1ll << 28)) >> 29;  // 24 bits, or 2^24 after a carry
  const int r = (int)(M - (Mh << 29));     // |r| <= 2^28
  int eh = e;
  if (Mh == (1ll << 24)) {
    Mh >>= 1;
    eh += 1;
  }
  const unsigned int sgn = (unsigned int)((unsigned long long)b >> 63) << 31;
  if (eh > 127) {  // beyond the FP32 range
    hi = __uint_as_float(sgn | 0x7F800000u);
    lo = 0.f;
    return;
  }
  hi = __uint_as_float(sgn | ((unsigned int)(eh + 127) << 23) | ((unsigned int)Mh & 0x7FFFFFu));
  // r 2^(e - 52) in two exact steps (e - 52 can be below -126)
  const int s1 = (e - 52) / 2;
  const float l = (float)r * pow2f(s1) * pow2f(e - 52 - s1);
  lo = sgn ? -l : l;
}
DV df2 df_from_scaled(cplx a, int E) {
  df2 r;
  df_split_scaled(a.x, E, r.rh, r.rl);
  df_split_scaled(a.y, E, r.ih, r.il);
  return r;
}
// (hi + lo) 2^E in FP64: the two parts converted exactly from their bits,
// one FP64 addition.
DV cplx df_to_scaled(const df2& a, int E) {
  return make_double2(f2d_scaled(a.rh, E, 0) + f2d_scaled(a.rl, E, 0), f2d_scaled(a.ih, E, 0) + f2d_scaled(a.il, E, 0));
}
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
