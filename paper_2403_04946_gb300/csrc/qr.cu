// Householder QR (geqrf) and application of its Q (ormqr) for tall complex
// float64 matrices, as cooperative persistent kernels.
//
// The rounding sweep (App. A, Alg. 1 mirrored and Alg. 4) factors one
// flattening per core, (n r) x K with K = 6 r after the operator apply.
// FP64 throughput on this part is a few FLOP per clock per SM, so every panel
// is spread over all SMs: CTA g owns a contiguous block of rows, keeps its
// rows of the current panel in shared memory, and the CTAs meet at bounded
// grid barriers for the column reductions (two per column) and the blocked
// trailing update (three per panel of width nb).  Reductions over CTAs are
// done in a fixed order, so results are bitwise reproducible.
#include <algorithm>

#include "kernels.h"

namespace hk {

constexpr int kQrThreads = 256;
// Mixed-precision kernels run 16 warps per SM: their double-float chains
// are latency-bound with 8 (each FP32 operation waits ~4.5 cycles on the
// previous one), and they need fewer registers than the FP64 variants.
constexpr int kQrThreadsMixed = 512;
constexpr int qr_threads(bool mixed) { return mixed ? kQrThreadsMixed : kQrThreads; }
constexpr int kNbMax = 32;

struct QrSmem {
  // sizes in cplx
  static size_t bytes(int R, int nb) {
    return sizeof(cplx) * ((size_t)nb * R + (size_t)nb * nb + 2 * kNbMax + 32) + 256;
  }
};

// v_s(i) for the panel held in P (after fix-up P holds pure V: zeros above
// the unit diagonal).
__device__ __forceinline__ cplx ld_cg(const cplx* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

// Loads of values other CTAs wrote before a grid barrier go to L2 (ld.cg):
// this SM's L1 may hold the line from the previous use of the buffer.
DV df2 ld_cg_df(const cplx* p) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  return df2{v.x, v.y, v.z, v.w};
}

// Warp reduce-scatter of CH per-lane values: afterwards a[0] of lane l
// holds the sum over all 32 lanes of value number rs_index<CH>(l), with the
// lanes that differ only in their low log2(32/CH) bits holding the same sum
// (rs_writer picks one of them).  31 exchanges for 32 values instead of 5
// per value: on this GPU the FP64 additions of a per-value warp sum cost
// more than the products they reduce.
template <int CH>
DV int rs_index(int lane) {
  int s = 0, o = 16;
#pragma unroll
  for (int h = CH / 2; h >= 1; h >>= 1, o >>= 1)
    if (lane & o) s += h;
  return s;
}
template <int CH>
DV bool rs_writer(int lane) {
  return (lane & (32 / CH - 1)) == 0;
}
template <int CH>
DV void reduce_scatter(cplx (&a)[CH], int lane) {
  int o = 16;
#pragma unroll
  for (int h = CH / 2; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const cplx send = up ? a[j] : a[j + h];
      const cplx keep = up ? a[j + h] : a[j];
      a[j] = mk(keep.x + __shfl_xor_sync(0xffffffffu, send.x, o), keep.y + __shfl_xor_sync(0xffffffffu, send.y, o));
    }
  }
  for (; o >= 1; o >>= 1) {
    a[0].x += __shfl_xor_sync(0xffffffffu, a[0].x, o);
    a[0].y += __shfl_xor_sync(0xffffffffu, a[0].y, o);
  }
}
DV df2 df_shfl_xor(const df2& v, int o) {
  return df2{__shfl_xor_sync(0xffffffffu, v.rh, o), __shfl_xor_sync(0xffffffffu, v.ih, o),
             __shfl_xor_sync(0xffffffffu, v.rl, o), __shfl_xor_sync(0xffffffffu, v.il, o)};
}
template <int CH>
DV void reduce_scatter(df2 (&a)[CH], int lane) {
  int o = 16;
#pragma unroll
  for (int h = CH / 2; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const df2 send = up ? a[j] : a[j + h];
      const df2 keep = up ? a[j + h] : a[j];
      a[j] = df_cadd(keep, df_shfl_xor(send, o));
    }
  }
  for (; o >= 1; o >>= 1) a[0] = df_cadd(a[0], df_shfl_xor(a[0], o));
}

// Partial products V^H X over this CTA's rows [lo, hi) (global row index),
// V in shared memory (P, leading dimension R, rows offset r0), X column l
// given by a pointer.  One warp per column; results to out[s + nbk * l].
template <int NB>
__device__ void partial_vhx(const cplx* P, int R, int r0, int lo, int hi, int nbk,
                            const cplx* X, int ldx, int ncol, cplx* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = w; l < ncol; l += nw) {
    cplx acc[NB];
#pragma unroll
    for (int s = 0; s < NB; ++s) acc[s] = mk(0, 0);
    const cplx* x = X + (size_t)ldx * l;
    // one row of look-ahead: the next row's load is in flight while this
    // row's NB complex multiply-adds run
    cplx xn = (lo + lane < hi) ? x[lo + lane] : mk(0, 0);
    for (int i = lo + lane; i < hi; i += 32) {
      const cplx xi = xn;
      if (i + 32 < hi) xn = x[i + 32];
      const cplx* pv = P + (i - r0);
#pragma unroll
      for (int s = 0; s < NB; ++s)
        if (s < nbk) acc[s] = cfmac(pv[(size_t)s * R], xi, acc[s]);
    }
    reduce_scatter<NB>(acc, lane);
    const int s = rs_index<NB>(lane);
    if (rs_writer<NB>(lane) && s < nbk) out[s + (size_t)nbk * l] = acc[0];
  }
}

// X[:, l] -= V * W2[:, l] over this CTA's rows [lo, hi); W2 column l at
// w2 + nbk * l.
template <int NB>
__device__ void update_x(const cplx* P, int R, int r0, int lo, int hi, int nbk, cplx* X,
                         int ldx, int ncol, const cplx* w2) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = w; l < ncol; l += nw) {
    cplx wc[NB];
#pragma unroll
    for (int s = 0; s < NB; ++s) {
      const cplx w = (s < nbk) ? ld_cg(w2 + s + (size_t)nbk * l) : mk(0, 0);
      wc[s] = mk(-w.x, -w.y);
    }
    cplx* x = X + (size_t)ldx * l;
    cplx xn = (lo + lane < hi) ? x[lo + lane] : mk(0, 0);
    for (int i = lo + lane; i < hi; i += 32) {
      cplx acc = xn;
      if (i + 32 < hi) xn = x[i + 32];
      const cplx* pv = P + (i - r0);
#pragma unroll
      for (int s = 0; s < NB; ++s)
        if (s < nbk) acc = cfma(pv[(size_t)s * R], wc[s], acc);  // wc holds -W2: 4 FMAs
      x[i] = acc;
    }
  }
}

// Mixed-precision versions: the panel V in shared memory and the matrix X
// both as double-float values (hi, lo in FP32, the same 16 bytes per
// complex as FP64); products and sums in double-float arithmetic on the
// FP32 pipe, partials handed on in FP64.  X stays in double-float form for
// the whole kernel, so the FP64 pipe (1/64 of the FP32 rate on this GPU)
// sees no per-element conversions.
template <int NB>
__device__ void partial_vhx_f(const df2* P, int R, int r0, int lo, int hi, int nbk,
                              const df2* X, int ldx, int ncol, cplx* out) {
  // 16 reflectors per pass over the rows keep the double-float accumulators
  // in registers
  constexpr int CH = NB < 16 ? NB : 16;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = w; l < ncol; l += nw) {
    const df2* x = X + (size_t)ldx * l;
    for (int s0 = 0; s0 < nbk; s0 += CH) {
      df2 acc[CH];
#pragma unroll
      for (int s = 0; s < CH; ++s) acc[s] = df_zero();
      df2 xn = (lo + lane < hi) ? x[lo + lane] : df_zero();
      for (int i = lo + lane; i < hi; i += 32) {
        const df2 xi = xn;
        if (i + 32 < hi) xn = x[i + 32];
        const df2* pv = P + (i - r0) + (size_t)s0 * R;
#pragma unroll
        for (int s = 0; s < CH; ++s)
          if (s0 + s < nbk) df_cmac_conj(acc[s], pv[(size_t)s * R], xi);
      }
      reduce_scatter<CH>(acc, lane);
      const int s = s0 + rs_index<CH>(lane);
      if (rs_writer<CH>(lane) && s < nbk) out[s + (size_t)nbk * l] = df_to_scaled(acc[0], 0);
    }
  }
}

template <int NB>
__device__ void update_x_f(const df2* P, int R, int r0, int lo, int hi, int nbk, df2* X,
                           int ldx, int ncol, const cplx* w2) {
  // the column's coefficients -W2[:, l] live in shared memory (every lane
  // reads the same one: broadcast), the running update in registers
  __shared__ df2 wsh[kQrThreadsMixed / 32][kNbMax];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l0 = 0; l0 < ncol; l0 += nw) {
    const int l = l0 + w;
    if (l < ncol && lane < nbk) {
      const cplx wv = ld_cg(w2 + lane + (size_t)nbk * l);
      wsh[w][lane] = df_from_scaled(mk(-wv.x, -wv.y), 0);
    }
    __syncwarp();
    if (l < ncol) {
      // four rows per lane at a time: four independent accumulation chains
      // (a double-float multiply-add is a chain of ~16 dependent FP32
      // operations, and only 8 warps share the SM)
      df2* x = X + (size_t)ldx * l;
      for (int i0 = lo + lane; i0 < hi; i0 += 128) {
        df2 xi[4], dlt[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = i0 + 32 * q;
          xi[q] = (i < hi) ? x[i] : df_zero();
          dlt[q] = df_zero();
        }
        const df2* pv = P + (i0 - r0);
#pragma unroll 4
        for (int s = 0; s < NB; ++s) {
          if (s < nbk) {
            const df2 ws = wsh[w][s];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (i0 + 32 * q < hi) df_cmac(dlt[q], pv[(size_t)s * R + 32 * q], ws);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (i0 + 32 * q < hi) x[i0 + 32 * q] = df_cadd(xi[q], dlt[q]);
      }
    }
    __syncwarp();
  }
}

// Rows [r0, r1) of columns [c0, c1) of the column-major A (lda) between
// FP64 and double-float form, in place (one CTA's rows), with a power-of-two
// scale: df = A * 2^-E on the way in, A = df * 2^E on the way out.  The
// scale keeps every entry below 1 in magnitude, so the FP32 exponent range
// of the double-float parts (and of their products) is never exceeded
// (entries below 2^-126 of the largest one become zero).  Integer
// conversions: no FP64 instructions.
__device__ void rows_to_df(cplx* A, int lda, int r0, int r1, int c0, int c1, int E) {
  const int nr = r1 - r0;
  if (nr <= 0) return;
  for (long long e = threadIdx.x; e < (long long)nr * (c1 - c0); e += blockDim.x) {
    const int c = c0 + (int)(e / nr), i = r0 + (int)(e % nr);
    cplx* p = A + i + (size_t)lda * c;
    const cplx v = *p;
    *reinterpret_cast<df2*>(p) = df_from_scaled(v, E);
  }
}
__device__ void rows_to_fp64(cplx* A, int lda, int r0, int r1, int c0, int c1, int E) {
  const int nr = r1 - r0;
  if (nr <= 0) return;
  for (long long e = threadIdx.x; e < (long long)nr * (c1 - c0); e += blockDim.x) {
    const int c = c0 + (int)(e / nr), i = r0 + (int)(e % nr);
    cplx* p = A + i + (size_t)lda * c;
    *p = df_to_scaled(*reinterpret_cast<const df2*>(p), E);
  }
}

// Power-of-two exponent E with max |entry| * 2^-E < 1 over rows [r0, r1) of
// columns [0, k) of every CTA: one grid barrier; the per-CTA maxima go to
// slot[0..G).  Returns E (0 for an all-zero matrix).
__device__ int grid_scale_exponent(const cplx* A, int lda, int r0, int r1, int k, double* slot,
                                   double* red, GridSync& gs, const GridBar* bar) {
  const int nr = r1 - r0;
  double mx = 0.0;
  if (nr > 0)
    for (long long e = threadIdx.x; e < (long long)nr * k; e += blockDim.x) {
      const cplx v = A[r0 + (int)(e % nr) + (size_t)lda * (int)(e / nr)];
      mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
  for (int o = 16; o >= 1; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, red[w]);
    slot[blockIdx.x] = b;
  }
  grid_sync(gs);
  if (grid_failed(bar)) return 0;
  // every warp takes the maximum over the CTAs' values, lanes in parallel
  double g = 0.0;
  for (int c = threadIdx.x & 31; c < (int)gridDim.x; c += 32) g = fmax(g, __ldcg(slot + c));
  for (int o = 16; o >= 1; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
  return (g > 0.0) ? ilogb(g) + 1 : 0;
}

// a * 2^e for a double-float value (exact unless the result leaves the
// FP32 range).
DV df2 df_scalb(const df2& a, int e) {
  return df2{scalbnf(a.rh, e), scalbnf(a.ih, e), scalbnf(a.rl, e), scalbnf(a.il, e)};
}

// Partials that other CTAs published are read kLoadBatch at a time: the
// loads of a batch are independent and in flight together (one L2 round
// trip per batch instead of one per CTA, on a path every column waits for);
// the additions keep their order.
constexpr int kLoadBatch = 8;

// Sum over the G per-CTA partials of entry e (stride pstride) by one warp.
__device__ __forceinline__ cplx reduce_partials(const cplx* pc, size_t pstride, int G, size_t e) {
  const int lane = threadIdx.x & 31;
  cplx acc = mk(0, 0);
  for (int g0 = lane; g0 < G; g0 += 32 * kLoadBatch) {
    cplx v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int g = g0 + 32 * u;
      v[u] = (g < G) ? ld_cg(pc + (size_t)g * pstride + e) : mk(0, 0);
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u)
      if (g0 + 32 * u < G) acc = cadd(acc, v[u]);
  }
  return warp_sum(acc);
}

template <int NB, bool MIXED>
__global__ void __launch_bounds__(qr_threads(MIXED), 1)
geqrf_kernel(cplx* A, int lda, int m, int k, cplx* tau, cplx* Tg, int nb, int R,
             CoopWs ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx* P = reinterpret_cast<cplx*>(smem_raw);
  cplx* Ts = P + (size_t)nb * R;
  cplx* wl = Ts + (size_t)nb * nb;  // [2*kNbMax]
  __shared__ double dred[32];
  __shared__ cplx bc[4];
  __shared__ df2 bcd[4];  // mixed: conj(tau), conj(scale), scale, beta as double-float values
  __shared__ float2 dredf[32];
  __shared__ int dtiny[32];

  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int r0 = g * R, r1 = min(m, r0 + R);
  const int p = min(m, k);
  const size_t pstride = ws.pc_elems / G;
  GridSync gs{ws.bar, 0u};
  // Mixed precision: this CTA's rows of A in double-float form, scaled by
  // 2^-E, until each column is factored (panel columns are written back in
  // FP64, the R part rescaled by 2^E; reflectors are scale-free).
  int E = 0;
  __shared__ int esc_sh;
  if (MIXED) {
    E = grid_scale_exponent(A, lda, r0, r1, k, ws.pr + 2 * G, dred, gs, ws.bar);
    if (grid_failed(ws.bar)) return;
    rows_to_df(A, lda, r0, r1, 0, k, E);
    __syncthreads();
  }

  // Per-CTA tail of the partial buffer, beyond what S1 uses: the in-panel
  // partial dot products (two parities x nb) and, for the CTA that owns the
  // pivot row, that row (two parities x nb).
  const size_t tail0 = pstride - (size_t)4 * nb;
  __shared__ cplx praw[kNbMax];

  for (int j0 = 0, panel = 0; j0 < p; j0 += nb, ++panel) {
    const int nbk = min(nb, p - j0);
    const int lo = max(r0, j0);  // rows of this CTA that the panel touches
    // load panel rows [r0, r1) of columns j0..j0+nbk-1 into shared memory
    // (FP64, or double-float in mixed precision)
    for (int t = 0; t < nbk; ++t)
      for (int i = r0 + tid; i < r1; i += blockDim.x) {
        const size_t e = i + (size_t)lda * (j0 + t);
        P[(size_t)t * R + (i - r0)] = A[e];  // same 16 bytes in either form
      }
    __syncthreads();

    // Panel factorisation with one grid barrier per column.  For column jj
    // with x its entries below the diagonal, v = [1; x * scale] and
    //   v^H a_l = a_l[jj] + conj(scale) * sum_{i>jj} conj(x_i) a_l[i],
    // so before the barrier each CTA publishes sum |x_i|^2 and the raw sums
    // over its own rows (and the owner of row jj publishes that row); after
    // it every CTA forms the reflector and updates its own rows.
    for (int t = 0; t < nbk; ++t) {
      const int jj = j0 + t;
      const int par = t & 1;
      const int nrem = nbk - t - 1;
      const int ilo = max(lo, jj + 1);  // own rows strictly below jj
      const int gown = jj / R;         // CTA owning row jj
      cplx* myp = ws.pc + (size_t)g * pstride + tail0 + (size_t)par * nb;
      cplx* rowp = ws.pc + (size_t)gown * pstride + tail0 + 2 * (size_t)nb + (size_t)par * nb;
      double* prp = ws.pr + par * G;
      // (a) partial sums over own rows > jj
      if constexpr (MIXED) {
        const df2* Pd = reinterpret_cast<const df2*>(P);
        const df2* xt = Pd + (size_t)t * R;
        // The squared norm in double-float arithmetic (rows are scaled
        // below 1), published in FP64; only thread 0 needs the CTA's sum:
        // warp sums in the warps that hold rows, then warp 0 over them (the
        // FP64 pipe runs at 1/64 of the FP32 rate).  A square or its low
        // part would leave the FP32 range for entries below 2^-39; a column
        // made only of such entries still needs its norm to full relative
        // precision (the reflector is unitary only with it), so a CTA that
        // holds one sums its squares in FP64 instead.
        float qh = 0.f, ql = 0.f;
        bool tiny = false;
        for (int i = ilo + tid; i < r1; i += blockDim.x) {
          const df2 x = xt[i - r0];
          const float mx = fmaxf(fabsf(x.rh), fabsf(x.ih));
          tiny |= (mx > 0.f && mx < 0x1p-39f);
          df_mac(qh, ql, x.rh, x.rl, x.rh, x.rl);
          df_mac(qh, ql, x.ih, x.il, x.ih, x.il);
        }
        if (ilo + 32 * wid < r1)
          for (int o = 16; o >= 1; o >>= 1)
            df_add_part(qh, ql, __shfl_xor_sync(0xffffffffu, qh, o), __shfl_xor_sync(0xffffffffu, ql, o));
        tiny = __any_sync(0xffffffffu, tiny);
        if (lane == 0) {
          dredf[wid] = make_float2(qh, ql);
          dtiny[wid] = tiny ? 1 : 0;
        }
        __syncthreads();
        if (wid == 0) {
          if (__any_sync(0xffffffffu, lane < nw && dtiny[lane])) {
            double v = 0.0;
            for (int i = ilo + lane; i < r1; i += 32) v += cabs2(df_to_scaled(xt[i - r0], 0));
            v = warp_sum(v);
            if (lane == 0) prp[g] = v;
          } else {
            float2 v = (lane < nw) ? dredf[lane] : make_float2(0.f, 0.f);
            for (int o = 16; o >= 1; o >>= 1)
              df_add_part(v.x, v.y, __shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
            if (lane == 0) prp[g] = f2d_scaled(v.x, 0, 0) + f2d_scaled(v.y, 0, 0);
          }
        }
        // up to four columns per warp, interleaved (independent chains)
        for (int cb = wid; cb < nrem; cb += 4 * nw) {
          df2 acc[4] = {df_zero(), df_zero(), df_zero(), df_zero()};
          for (int i = ilo + lane; i < r1; i += 32) {
            const df2 x = xt[i - r0];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (cb + q * nw < nrem) df_cmac_conj(acc[q], x, Pd[(size_t)(t + 1 + cb + q * nw) * R + (i - r0)]);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (cb + q * nw < nrem) {
              for (int o = 16; o >= 1; o >>= 1) acc[q] = df_cadd(acc[q], df_shfl_xor(acc[q], o));
              if (lane == 0) reinterpret_cast<df2*>(myp)[cb + q * nw] = acc[q];
            }
          }
        }
        if (g == gown)
          for (int c = tid; c < nbk - t; c += blockDim.x)
            reinterpret_cast<df2*>(rowp)[c] = Pd[(size_t)(t + c) * R + (jj - r0)];
      } else {
        const cplx* xt = P + (size_t)t * R;
        double sq = 0.0;
        for (int i = ilo + tid; i < r1; i += blockDim.x) sq += cabs2(xt[i - r0]);
        sq = block_sum(sq, dred);
        if (tid == 0) prp[g] = sq;
        for (int cb = wid; cb < nrem; cb += 4 * nw) {
          cplx acc[4] = {mk(0, 0), mk(0, 0), mk(0, 0), mk(0, 0)};
          for (int i = ilo + lane; i < r1; i += 32) {
            const cplx x = xt[i - r0];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (cb + q * nw < nrem) acc[q] = cfmac(x, P[(size_t)(t + 1 + cb + q * nw) * R + (i - r0)], acc[q]);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (cb + q * nw < nrem) {
              acc[q] = warp_sum(acc[q]);
              if (lane == 0) myp[cb + q * nw] = acc[q];
            }
          }
        }
        if (g == gown)
          for (int c = tid; c < nbk - t; c += blockDim.x) rowp[c] = P[(size_t)(t + c) * R + (jj - r0)];
      }
      grid_sync(gs);
      if (grid_failed(ws.bar)) return;
      // (b) the reflector (zlarfg conventions: beta real, v_jj = 1), in FP64
      if (wid == 0) {
        // the pivot row's entry alpha is loaded with the first batch of
        // partial norms (both are one L2 round trip away)
        cplx al;
        if constexpr (MIXED) al = df_to_scaled(ld_cg_df(rowp), 0);
        else al = ld_cg(rowp);
        double s2 = 0.0;
        for (int g0 = lane; g0 < G; g0 += 32 * kLoadBatch) {
          double v[kLoadBatch];
#pragma unroll
          for (int u = 0; u < kLoadBatch; ++u) v[u] = (g0 + 32 * u < G) ? ld_cg(prp + g0 + 32 * u) : 0.0;
#pragma unroll
          for (int u = 0; u < kLoadBatch; ++u)
            if (g0 + 32 * u < G) s2 += v[u];
        }
        s2 = warp_sum(s2);
        if (lane == 0) {
          cplx tu, sc;
          double beta;
          if (s2 == 0.0 && al.y == 0.0) {
            tu = mk(0, 0);
            beta = al.x;
            sc = mk(0, 0);
          } else {
            // one division for tau, one for the scale
            const double an = sqrt(al.x * al.x + al.y * al.y + s2);
            beta = (al.x >= 0.0) ? -an : an;
            const double ib = 1.0 / beta;
            tu = mk((beta - al.x) * ib, -al.y * ib);
            sc = cinv(mk(al.x - beta, al.y));
          }
          if (MIXED) {
            // the scale can leave the FP32 range (tiny columns): keep it as
            // mantissa x 2^esc
            const double smax = fmax(fabs(sc.x), fabs(sc.y));
            const int es = (smax > 0.0) ? ilogb(smax) : 0;
            sc = mk(scalbn(sc.x, -es), scalbn(sc.y, -es));
            esc_sh = es;
            bcd[0] = df_from_scaled(cconj(tu), 0);
            bcd[1] = df_from_scaled(cconj(sc), 0);
            bcd[2] = df_from_scaled(sc, 0);
            bcd[3] = df_from_scaled(mk(beta, 0.0), 0);
          }
          bc[0] = tu;
          bc[1] = sc;
          bc[2] = mk(beta, 0.0);
        }
      }
      // raw sums over the CTAs of the dot products (tpc threads per
      // column); in mixed precision warp 0 is left out, so that these sums
      // run while it forms the reflector
      const int skip = MIXED ? 32 : 0;
      if (nrem > 0 && tid >= skip) {
        const int nthr = blockDim.x - skip, t2 = tid - skip;
        int tpc = 32;
        while (tpc > 1 && tpc * nrem > nthr) tpc >>= 1;
        const int per = nthr / tpc, sub = t2 % tpc;
        for (int base = 0; base < nrem; base += per) {
          const int c = base + t2 / tpc;
          const bool valid = c < nrem && t2 / tpc < per;
          const cplx* src = ws.pc + tail0 + (size_t)par * nb + c;
          if constexpr (MIXED) {
            df2 acc = df_zero();
            if (valid)
              for (int g0 = sub; g0 < G; g0 += tpc * kLoadBatch) {
                df2 v[kLoadBatch];
#pragma unroll
                for (int u = 0; u < kLoadBatch; ++u) {
                  const int gg = g0 + tpc * u;
                  v[u] = (gg < G) ? ld_cg_df(src + (size_t)gg * pstride) : df_zero();
                }
#pragma unroll
                for (int u = 0; u < kLoadBatch; ++u)
                  if (g0 + tpc * u < G) acc = df_cadd(acc, v[u]);
              }
            for (int o = 1; o < tpc; o <<= 1) acc = df_cadd(acc, df_shfl_xor(acc, o));
            if (valid && sub == 0) reinterpret_cast<df2*>(praw)[c] = acc;
          } else {
            cplx acc = mk(0, 0);
            if (valid)
              for (int g0 = sub; g0 < G; g0 += tpc * kLoadBatch) {
                cplx v[kLoadBatch];
#pragma unroll
                for (int u = 0; u < kLoadBatch; ++u) {
                  const int gg = g0 + tpc * u;
                  v[u] = (gg < G) ? ld_cg(src + (size_t)gg * pstride) : mk(0, 0);
                }
#pragma unroll
                for (int u = 0; u < kLoadBatch; ++u)
                  if (g0 + tpc * u < G) acc = cadd(acc, v[u]);
              }
            for (int o = 1; o < tpc; o <<= 1) {
              acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
              acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (valid && sub == 0) praw[c] = acc;
          }
        }
      }
      __syncthreads();
      const cplx tu = bc[0], sc = bc[1];
      // f_c = conj(tau) (a_c[jj] + conj(scale) raw_c) into wl; scale column t
      if constexpr (MIXED) {
        df2* Pd = reinterpret_cast<df2*>(P);
        const df2 ctu = bcd[0], csc = bcd[1], scd = bcd[2];
        const int es = esc_sh;
        for (int c = tid; c < nrem; c += blockDim.x) {
          df2 cr = df_zero();
          df_cmac(cr, csc, reinterpret_cast<const df2*>(praw)[c]);
          const df2 w = df_cadd(ld_cg_df(rowp + 1 + c), df_scalb(cr, es));
          df2 f = df_zero();
          df_cmac(f, ctu, w);
          f = df_cadd(f, df_zero());
          reinterpret_cast<df2*>(wl)[c] = df2{-f.rh, -f.ih, -f.rl, -f.il};  // -f
        }
        df2* xt = Pd + (size_t)t * R;
        for (int i = ilo + tid; i < r1; i += blockDim.x) {
          df2 v = df_zero();
          df_cmac(v, xt[i - r0], scd);
          xt[i - r0] = df_scalb(df_cadd(v, df_zero()), es);
        }
        if (tid == 0 && jj >= r0 && jj < r1) xt[jj - r0] = bcd[3];
      } else {
        for (int c = tid; c < nrem; c += blockDim.x) {
          const cplx w = cadd(ld_cg(rowp + 1 + c), cmul(cconj(sc), praw[c]));
          const cplx f = cmul(cconj(tu), w);
          wl[c] = mk(-f.x, -f.y);  // -f
        }
        cplx* xt = P + (size_t)t * R;
        for (int i = ilo + tid; i < r1; i += blockDim.x) xt[i - r0] = cmul(xt[i - r0], sc);
        if (tid == 0 && jj >= r0 && jj < r1) xt[jj - r0] = bc[2];
      }
      if (tid == 0 && g == 0) tau[jj] = tu;
      __syncthreads();
      // apply H^H = I - conj(tau) v v^H to panel columns t+1..nbk-1 of own
      // rows >= jj (v_jj = 1)
      if (nrem > 0) {
        const int ifrom = max(lo, jj);
        const int nrow = r1 - ifrom;
        if constexpr (MIXED) {
          df2* Pd = reinterpret_cast<df2*>(P);
          const df2* xt = Pd + (size_t)t * R;
          const df2* nf = reinterpret_cast<const df2*>(wl);
          for (int e = tid; e < nrow * nrem; e += blockDim.x) {
            const int c = e / nrow, i = ifrom + e % nrow;
            const df2 v = (i == jj) ? df2{1.f, 0.f, 0.f, 0.f} : xt[i - r0];
            df2& a = Pd[(size_t)(t + 1 + c) * R + (i - r0)];
            df2 dlt = df_zero();
            df_cmac(dlt, v, nf[c]);
            a = df_cadd(a, dlt);
          }
        } else {
          const cplx* xt = P + (size_t)t * R;
          for (int e = tid; e < nrow * nrem; e += blockDim.x) {
            const int c = e / nrow, i = ifrom + e % nrow;
            const cplx v = (i == jj) ? mk(1, 0) : xt[i - r0];
            cplx& a = P[(size_t)(t + 1 + c) * R + (i - r0)];
            a = cfma(v, wl[c], a);
          }
        }
      }
      __syncthreads();
    }
    // write the factored panel back in FP64 (R on/above the diagonal, V below)
    for (int t = 0; t < nbk; ++t)
      for (int i = r0 + tid; i < r1; i += blockDim.x) {
        const size_t e = (size_t)t * R + (i - r0);
        if (MIXED) {
          const int sh = (i <= j0 + t) ? E : 0;  // R part scaled back, reflector tails scale-free
          A[i + (size_t)lda * (j0 + t)] = df_to_scaled(reinterpret_cast<const df2*>(P)[e], sh);
        } else {
          A[i + (size_t)lda * (j0 + t)] = P[e];
        }
      }
    __syncthreads();
    // fix up P to hold pure reflectors: zero above, one on the diagonal
    for (int t = 0; t < nbk; ++t)
      for (int i = r0 + tid; i < r1; i += blockDim.x) {
        const size_t e = (size_t)t * R + (i - r0);
        if (i < j0 + t) {
          if (MIXED) reinterpret_cast<df2*>(P)[e] = df_zero();
          else P[e] = mk(0, 0);
        } else if (i == j0 + t) {
          if (MIXED) reinterpret_cast<df2*>(P)[e] = df2{1.f, 0.f, 0.f, 0.f};
          else P[e] = mk(1, 0);
        }
      }
    __syncthreads();

    // S1: partials of V^H [V | A_trail]
    const int c0 = j0 + nbk;
    const int nt = k - c0;
    const int ncol = nbk + nt;
    if (MIXED) {
      cplx* out = ws.pc + (size_t)g * pstride;
      // the Gram block (its columns are the reflectors themselves) and the
      // trailing products from the double-float panel, on the FP32 pipe
      const df2* Pd = reinterpret_cast<const df2*>(P);
      partial_vhx_f<NB>(Pd, R, r0, lo, r1, nbk, Pd - r0, R, nbk, out);
      if (nt > 0)
        partial_vhx_f<NB>(Pd, R, r0, lo, r1, nbk, reinterpret_cast<const df2*>(A) + (size_t)lda * c0, lda, nt,
                          out + (size_t)nbk * nbk);
    } else {
      cplx* out = ws.pc + (size_t)g * pstride;
      // Gram block: columns are the reflectors themselves (from shared memory)
      for (int l = wid; l < nbk; l += nw) {
        cplx acc[NB];
#pragma unroll
        for (int s = 0; s < NB; ++s) acc[s] = mk(0, 0);
        for (int i = lo + lane; i < r1; i += 32) {
          const cplx xi = P[(size_t)l * R + (i - r0)];
#pragma unroll
          for (int s = 0; s < NB; ++s)
            if (s < nbk) acc[s] = cfmac(P[(size_t)s * R + (i - r0)], xi, acc[s]);
        }
        reduce_scatter<NB>(acc, lane);
        const int s = rs_index<NB>(lane);
        if (rs_writer<NB>(lane) && s < nbk) out[s + (size_t)nbk * l] = acc[0];
      }
      __syncthreads();
      if (nt > 0) partial_vhx<NB>(P, R, r0, lo, r1, nbk, A + (size_t)lda * c0, lda, nt, out + (size_t)nbk * nbk);
    }
    grid_sync(gs);
    if (grid_failed(ws.bar)) return;
    // S2: reduce columns l % G == g into wfin
    for (int l = g; l < ncol; l += G) {
      for (int s = wid; s < nbk; s += nw) {
        cplx v = reduce_partials(ws.pc, pstride, G, s + (size_t)nbk * l);
        if (lane == 0) ws.wfin[s + (size_t)nbk * l] = v;
      }
    }
    grid_sync(gs);
    if (grid_failed(ws.bar)) return;
    // S3: W2 = T^H W for the trailing columns this CTA reduced, without
    // forming T: applying H_0^H, H_1^H, ... in turn gives, with
    // Gram[s,u] = v_s^H v_u,
    //   w2_s = conj(tau_s) (W[s] - sum_{u<s} Gram[s,u] w2_u),
    // a chain of nbk steps per column (lanes = s; one warp per column).  The
    // panel's Gram (strict upper triangle) and tau (diagonal) are kept in
    // Tg for ormqr, which runs the mirrored recurrence.
    for (int e = tid; e < nbk * nbk; e += blockDim.x) {
      const int u = e % nbk, c = e / nbk;
      Ts[e] = (u < c) ? ld_cg(ws.wfin + e) : (u == c ? ld_cg(tau + j0 + c) : mk(0, 0));
    }
    __syncthreads();
    if (g == 0)
      for (int e = tid; e < nbk * nbk; e += blockDim.x) Tg[(size_t)panel * nb * nb + e] = Ts[e];
    {
      const cplx ctl = (lane < nbk) ? cconj(Ts[lane + nbk * lane]) : mk(0, 0);  // conj(tau_lane)
      for (int l = nbk + g + wid * G; l < ncol; l += nw * G) {
        cplx acc = (lane < nbk) ? ld_cg(ws.wfin + lane + (size_t)nbk * l) : mk(0, 0);
        cplx mine = mk(0, 0);
        for (int u = 0; u < nbk; ++u) {
          const cplx wu = cmul(ctl, acc);  // valid on lane u
          const cplx w2u = make_double2(__shfl_sync(0xffffffffu, wu.x, u), __shfl_sync(0xffffffffu, wu.y, u));
          if (lane == u) mine = w2u;
          // Gram[lane, u] = conj(v_u^H v_lane) for u < lane
          if (lane > u && lane < nbk) acc = csub(acc, cmulc(Ts[u + nbk * lane], w2u));
        }
        if (lane < nbk) ws.wfin[lane + (size_t)nbk * l] = mine;
      }
    }
    grid_sync(gs);
    if (grid_failed(ws.bar)) return;
    // S4: trailing update over this CTA's rows
    if (nt > 0) {
      if (MIXED)
        update_x_f<NB>(reinterpret_cast<const df2*>(P), R, r0, lo, r1, nbk, reinterpret_cast<df2*>(A) + (size_t)lda * c0,
                       lda, nt, ws.wfin + (size_t)nbk * nbk);
      else
        update_x<NB>(P, R, r0, lo, r1, nbk, A + (size_t)lda * c0, lda, nt, ws.wfin + (size_t)nbk * nbk);
    }
    __syncthreads();
  }
  // columns never factored (k > m) go back to FP64
  if (MIXED && k > p) rows_to_fp64(A, lda, r0, r1, p, k, E);
}

template <int NB, bool MIXED>
__global__ void __launch_bounds__(qr_threads(MIXED), 1)
ormqr_kernel(const cplx* A, int lda, int m, int p, const cplx* Tg, int nb, cplx* C, int ldc,
             int q, int R, CoopWs ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx* P = reinterpret_cast<cplx*>(smem_raw);
  cplx* Ts = P + (size_t)nb * R;
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int r0 = g * R, r1 = min(m, r0 + R);
  const size_t pstride = ws.pc_elems / G;
  const int npanel = (p + nb - 1) / nb;
  GridSync gs{ws.bar, 0u};
  // Mixed precision: this CTA's rows of C in double-float form (scaled by
  // 2^-E) throughout
  __shared__ double dred[32];
  int E = 0;
  if (MIXED) {
    E = grid_scale_exponent(C, ldc, r0, r1, q, ws.pr, dred, gs, ws.bar);
    if (grid_failed(ws.bar)) return;
    rows_to_df(C, ldc, r0, r1, 0, q, E);
    __syncthreads();
  }
  for (int panel = npanel - 1; panel >= 0; --panel) {
    const int j0 = panel * nb;
    const int nbk = min(nb, p - j0);
    const int lo = max(r0, j0);
    for (int t = 0; t < nbk; ++t)
      for (int i = r0 + tid; i < r1; i += blockDim.x) {
        cplx v;
        if (i < j0 + t) v = mk(0, 0);
        else if (i == j0 + t) v = mk(1, 0);
        else v = A[i + (size_t)lda * (j0 + t)];
        if (MIXED) reinterpret_cast<df2*>(P)[(size_t)t * R + (i - r0)] = df_from_scaled(v, 0);
        else P[(size_t)t * R + (i - r0)] = v;
      }
    // the panel's Gram (strict upper triangle) and tau (diagonal), packed
    // with leading dimension nbk
    for (int e = tid; e < nbk * nbk; e += blockDim.x) Ts[e] = Tg[(size_t)panel * nb * nb + e];
    __syncthreads();
    if (MIXED)
      partial_vhx_f<NB>(reinterpret_cast<const df2*>(P), R, r0, lo, r1, nbk, reinterpret_cast<const df2*>(C), ldc, q,
                        ws.pc + (size_t)g * pstride);
    else
      partial_vhx<NB>(P, R, r0, lo, r1, nbk, C, ldc, q, ws.pc + (size_t)g * pstride);
    grid_sync(gs);
    if (grid_failed(ws.bar)) return;
    // reduce, then W2 = T W (apply Q, not Q^H) from the stored Gram and tau:
    // applying H_{nbk-1}, ..., H_0 in turn gives
    //   w2_s = tau_s (W[s] - sum_{u>s} Gram[s,u] w2_u),  Gram[s,u] = v_s^H v_u
    for (int l = g; l < q; l += G) {
      for (int s = wid; s < nbk; s += nw) {
        cplx v = reduce_partials(ws.pc, pstride, G, s + (size_t)nbk * l);
        if (lane == 0) ws.wfin[s + (size_t)nbk * l] = v;
      }
    }
    __syncthreads();
    {
      const cplx tl = (lane < nbk) ? Ts[lane + nbk * lane] : mk(0, 0);  // tau_lane
      for (int l = g + wid * G; l < q; l += nw * G) {
        cplx acc = (lane < nbk) ? ws.wfin[lane + (size_t)nbk * l] : mk(0, 0);
        cplx mine = mk(0, 0);
        for (int u = nbk - 1; u >= 0; --u) {
          const cplx wu = cmul(tl, acc);  // valid on lane u
          const cplx w2u = make_double2(__shfl_sync(0xffffffffu, wu.x, u), __shfl_sync(0xffffffffu, wu.y, u));
          if (lane == u) mine = w2u;
          // Gram[lane, u] = v_lane^H v_u, stored for lane < u
          if (lane < u) acc = csub(acc, cmul(Ts[lane + nbk * u], w2u));
        }
        if (lane < nbk) ws.wfin[lane + (size_t)nbk * l] = mine;
      }
    }
    grid_sync(gs);
    if (grid_failed(ws.bar)) return;
    if (MIXED)
      update_x_f<NB>(reinterpret_cast<const df2*>(P), R, r0, lo, r1, nbk, reinterpret_cast<df2*>(C), ldc, q, ws.wfin);
    else
      update_x<NB>(P, R, r0, lo, r1, nbk, C, ldc, q, ws.wfin);
    __syncthreads();
    // No barrier needed here: the next panel writes wfin only after its
    // first grid_sync, which every CTA reaches after finishing this update.
  }
  if (MIXED) rows_to_fp64(C, ldc, r0, r1, 0, q, E);
}

static void pick_layout(int m, const CoopWs& ws, int* G, int* R, int* nb, size_t* smem) {
  const DevInfo& di = dev_info();
  // row blocks of >= 64 rows, but small matrices (the wide first and last
  // cores) still spread over up to 16 CTAs of >= 8 rows
  int g = std::max(1, std::min(coop_sms(ws), std::max((m + 63) / 64, std::min(16, (m + 7) / 8))));
  int r = (m + g - 1) / g;
  int b = kNbMax;
  const size_t lim = (size_t)di.max_smem_optin - 16384;  // static shared memory too
  while (b > 4 && QrSmem::bytes(r, b) > lim) b >>= 1;
  *G = g;
  *R = r;
  *nb = b;
  *smem = QrSmem::bytes(r, b);
}

cudaError_t geqrf(cplx* A, int lda, int m, int k, cplx* tau, cplx* T, int* nb_out,
                  const CoopWs& ws, cudaStream_t s, int mixed) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  int G, R, nb;
  size_t smem;
  pick_layout(m, ws, &G, &R, &nb, &smem);
  // per CTA: S1 partials nb (nb + k), then the panel's exchange tail 4 nb
  if ((size_t)G * ((size_t)nb * (nb + k) + 4 * (size_t)nb) > ws.pc_elems || (size_t)nb * (nb + k) > ws.wfin_elems)
    return cudaErrorInvalidValue;
  *nb_out = nb;
  void* fn;
  if (mixed) {
    if (nb == 32) fn = (void*)geqrf_kernel<32, true>;
    else if (nb == 16) fn = (void*)geqrf_kernel<16, true>;
    else fn = (void*)geqrf_kernel<8, true>;
  } else {
    if (nb == 32) fn = (void*)geqrf_kernel<32, false>;
    else if (nb == 16) fn = (void*)geqrf_kernel<16, false>;
    else fn = (void*)geqrf_kernel<8, false>;
  }
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  CoopWs w = ws;
  e = cudaMemsetAsync(&ws.bar->count, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&A, &lda, &m, &k, &tau, &T, &nb, &R, &w};
  return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(qr_threads(mixed != 0)), args, smem, s);
}

cudaError_t ormqr(const cplx* A, int lda, int m, int p, const cplx* tau, const cplx* T,
                  int nb, cplx* C, int ldc, int q, const CoopWs& ws, cudaStream_t s, int mixed) {
  (void)tau;
  if (m <= 0 || p <= 0 || q <= 0) return cudaSuccess;
  int G, R, nb2;
  size_t smem;
  pick_layout(m, ws, &G, &R, &nb2, &smem);
  if (nb2 != nb) {
    // the layout depends only on m, so geqrf and ormqr agree
    return cudaErrorInvalidValue;
  }
  if ((size_t)G * nb * (size_t)q > ws.pc_elems || (size_t)nb * q > ws.wfin_elems)
    return cudaErrorInvalidValue;
  void* fn;
  if (mixed) {
    if (nb == 32) fn = (void*)ormqr_kernel<32, true>;
    else if (nb == 16) fn = (void*)ormqr_kernel<16, true>;
    else fn = (void*)ormqr_kernel<8, true>;
  } else {
    if (nb == 32) fn = (void*)ormqr_kernel<32, false>;
    else if (nb == 16) fn = (void*)ormqr_kernel<16, false>;
    else fn = (void*)ormqr_kernel<8, false>;
  }
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  CoopWs w = ws;
  e = cudaMemsetAsync(&ws.bar->count, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&A, &lda, &m, &p, (void*)&T, &nb, &C, &ldc, &q, &R, &w};
  return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(qr_threads(mixed != 0)), args, smem, s);
}

}  // namespace hk
