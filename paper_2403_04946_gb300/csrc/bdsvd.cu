// SVD of the small square factor R through bidiagonalisation.
//
// The truncation at a bond needs every singular value of the triangular
// factor R (the discarded tail) and the left singular vectors of the kept
// ones (App. A, the QR-then-SVD structure of Alg. 4).  Instead of Jacobi
// rotations (O(n^3) flops per sweep, a dozen sweeps), R is reduced once:
//
//  1. Householder bidiagonalisation R = Q B P^H (Golub & Kahan 1965), B real
//     upper bidiagonal, with the reflector conventions of LAPACK's zgebrd.
//     One cooperative launch; CTA g keeps the rows r = g (mod G) of R in
//     shared memory and the CTAs meet once per column (see gebrd_kernel).
//  2. Singular values of B: eigenvalues of the Golub-Kahan tridiagonal T_GK
//     (order 2n, zero diagonal, off-diagonals d_1, e_1, d_2, ..., d_n, whose
//     eigenvalues are +-sigma) by Sturm-count multisection, one warp per
//     value.  Counts are taken in double-float arithmetic (hi + lo FP32
//     pair, ~2^-47 relative): a Sturm count is exact for a matrix whose
//     entries are perturbed by a few units of the working precision, and
//     the singular values of a bidiagonal move by a relative amount of the
//     same order under such perturbations (Demmel & Kahan 1990), so every
//     value, large or small, is found to a relative accuracy of ~1e-13.
//  3. Left singular vectors of B for the kept values: inverse iteration on
//     T_GK - sigma I (the eigenvector for +sigma is (v_1, u_1, ..., v_n,
//     u_n)/sqrt 2), FP64, tridiagonal LU with partial pivoting, modified
//     Gram-Schmidt inside clusters of close values (as in LAPACK's dstein).
//     Kept values at the rounding-noise level of R get an orthonormal
//     completion instead (their vectors are not determined by R).
//  4. U = Q [u_1 .. u_rho] by applying the left reflectors.
#include <algorithm>
#include <cfloat>

#include "kernels.h"

namespace hk {

constexpr int kBdThreads = 256;

// Values other CTAs published are read kBdBatch at a time per lane: the
// loads of a batch are independent and in flight together, one L2 round
// trip per batch on a path every column waits for; sums keep their order.
constexpr int kBdBatch = 8;
DV double sum_published(const double* p, int G) {  // lane-strided partial sum
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int g0 = lane; g0 < G; g0 += 32 * kBdBatch) {
    double v[kBdBatch];
#pragma unroll
    for (int u = 0; u < kBdBatch; ++u) v[u] = (g0 + 32 * u < G) ? __ldcg(p + g0 + 32 * u) : 0.0;
#pragma unroll
    for (int u = 0; u < kBdBatch; ++u)
      if (g0 + 32 * u < G) s += v[u];
  }
  return s;
}
DV cplx sum_published(const cplx* p, size_t stride, int G) {
  const int lane = threadIdx.x & 31;
  cplx s = mk(0, 0);
  for (int g0 = lane; g0 < G; g0 += 32 * kBdBatch) {
    cplx v[kBdBatch];
#pragma unroll
    for (int u = 0; u < kBdBatch; ++u) v[u] = (g0 + 32 * u < G) ? __ldcg(p + (size_t)(g0 + 32 * u) * stride) : mk(0, 0);
#pragma unroll
    for (int u = 0; u < kBdBatch; ++u)
      if (g0 + 32 * u < G) s = cadd(s, v[u]);
  }
  return s;
}
// Sum over the block delivered to warp 0 only (the other warps' FP64 work
// in a block-wide reduction costs more, on this GPU's narrow FP64 pipe,
// than the column's arithmetic).  Warps whose `has` is false contribute
// zero without reducing.  Ends with __syncthreads (so it also publishes
// the block's shared-memory writes made before it).
DV double sum_to_warp0(double v, bool has, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (has) v = warp_sum(v);
  if (lane == 0) red[w] = has ? v : 0.0;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (lane < nw) ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  __syncthreads();
  return s;
}

DV void house_scalars(cplx alpha, double xnorm2, cplx* tau, cplx* scale, double* beta) {
  // H^H [alpha; x] = [beta; 0] with H = I - tau v v^H, v = [1; x * scale]
  if (xnorm2 == 0.0 && alpha.y == 0.0) {
    *tau = mk(0, 0);
    *scale = mk(0, 0);
    *beta = alpha.x;
    return;
  }
  // two FP64 divisions (each ~640 cycles of latency on this GPU), issued
  // independently of each other
  const double an = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2);
  const double b = (alpha.x >= 0.0) ? -an : an;
  const double ib = 1.0 / b;
  const double dr = alpha.x - b, di = alpha.y;
  const double id2 = 1.0 / (dr * dr + di * di);
  *tau = mk((b - alpha.x) * ib, -alpha.y * ib);
  *scale = mk(dr * id2, -di * id2);
  *beta = b;
}

// ---- 1. bidiagonalisation -------------------------------------------------------
// Column i, with H = I - tau v v^H the left reflector (v_i = 1,
// v_r = A[r,i] * scale for r > i) and w_c = sum_r conj(v_r) A[r,c]:
//   w_c = A[i,c] + conj(scale) * sum_{r>i} conj(A[r,i]) A[r,c].
// Each CTA writes its partial sums over its own rows (and the owner of row
// i publishes that row); after a grid barrier, CTA g reduces the columns
// c = i+1+g (mod G) and publishes conj(tau) w_c and the updated row i,
// A[i,c] - conj(tau) w_c; after a second barrier every CTA forms the right
// reflector G = I - taup u u^H of that row itself and applies both
// reflectors to its own rows.  (Reducing every column in every CTA would
// save the second barrier but costs G times the FP64 additions, which on
// this GPU's narrow FP64 pipe outweigh the barrier.)  The exchange buffers
// alternate between two halves by column parity: a CTA writing column
// i+2's data has passed both barriers of column i+1, so every reader of
// column i's half is done.
__global__ void __launch_bounds__(kBdThreads, 1)
gebrd_kernel(cplx* A, int lda, int n, int nloc, double* dg, double* eg, cplx* tauq, cplx* taup,
             CoopWs ws, cplx* rows_global) {
  extern __shared__ __align__(16) unsigned char bd_smem[];
  // own rows (nloc x n, row-major) in shared memory, or, for a factor too
  // large for it, in this CTA's slice of a global workspace (L2-resident)
  cplx* rows = rows_global ? rows_global + (size_t)blockIdx.x * nloc * n : reinterpret_cast<cplx*>(bd_smem);
  cplx* fv = rows_global ? reinterpret_cast<cplx*>(bd_smem) : rows + (size_t)nloc * n;  // conj(tau) w_c
  cplx* nrow = fv + n;                           // updated row i
  cplx* uv = nrow + n;                           // right reflector u
  cplx* vloc = uv + n;                           // v_r of own rows (nloc)
  __shared__ double dred[32];
  __shared__ cplx bc[4];
  __shared__ cplx bcr[4];
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const size_t pstride = (size_t)n + 1;
  GridSync gs{ws.bar, 0u};
  auto grow = [&](int lr) { return g + lr * G; };
  auto R = [&](int lr, int c) -> cplx& { return rows[(size_t)lr * n + c]; };
  const int nact = min(nloc, (n - g + G - 1) / G);  // local rows that exist

  for (int lr = 0; lr < nloc; ++lr) {
    const int r = grow(lr);
    for (int c = tid; c < n; c += blockDim.x) R(lr, c) = (r < n) ? A[r + (size_t)lda * c] : mk(0, 0);
  }
  __syncthreads();

  for (int i = 0; i < n; ++i) {
    const int buf = i & 1;
    cplx* pc = ws.pc + (size_t)buf * G * pstride;
    double* pr = ws.pr + buf * G;
    cplx* rowb = ws.wfin + (size_t)buf * 3 * n;  // row i as published by its owner
    cplx* fvg = rowb + n;                        // conj(tau) w_c
    cplx* nrg = fvg + n;                         // updated row i
    const int C = n - i - 1;
    // first own local row strictly below i (rows of this CTA: g + lr G)
    const int lr0 = (i + 1 > g) ? (i + 1 - g + G - 1) / G : 0;
    const bool owner = (i % G == g);
    // (a) partial sums over own rows r > i
    double sq = 0.0;
    for (int lr = lr0 + tid; lr < nact; lr += blockDim.x) sq += cabs2(R(lr, i));
    sq = sum_to_warp0(sq, lr0 + 32 * wid < nact, dred);
    for (int c = i + 1 + tid; c < n; c += blockDim.x) {
      cplx acc = mk(0, 0);
      for (int lr = lr0; lr < nact; ++lr) acc = cfmac(R(lr, i), R(lr, c), acc);
      pc[(size_t)g * pstride + c] = acc;
    }
    if (tid == 0) pr[g] = sq;
    if (owner)
      for (int c = i + tid; c < n; c += blockDim.x) rowb[c] = R(i / G, c);
    grid_sync(gs);
    if (grid_failed(ws.bar)) return;
    // (b1) left reflector of column i (every CTA), reduction of its columns
    if (wid == 0) {
      const double s2 = warp_sum(sum_published(pr, G));
      if (lane == 0) {
        cplx tq, sc;
        double beta;
        house_scalars(__ldcg(rowb + i), s2, &tq, &sc, &beta);
        bc[0] = tq;
        bc[1] = sc;
        bc[2] = mk(beta, 0.0);
      }
    }
    __syncthreads();
    const cplx tq = bc[0], scq = bc[1];
    const cplx ctq = cconj(tq), cscq = cconj(scq);
    for (int cc = g + wid * G; cc < C; cc += nw * G) {
      const int c = i + 1 + cc;
      const cplx acc = warp_sum(sum_published(pc + c, pstride, G));
      if (lane == 0) {
        const cplx a_ic = __ldcg(rowb + c);
        const cplx f = cmul(ctq, cadd(a_ic, cmul(cscq, acc)));
        fvg[c] = f;
        nrg[c] = csub(a_ic, f);
      }
    }
    grid_sync(gs);
    if (grid_failed(ws.bar)) return;
    // (b2) left update of own rows r > i: A[r,c] -= v_r conj(tau) w_c;
    // column i keeps v_r
    for (int lr = lr0 + tid; lr < nact; lr += blockDim.x) vloc[lr] = cmul(R(lr, i), scq);
    double sqp = 0.0;
    for (int c = i + 1 + tid; c < n; c += blockDim.x) {
      fv[c] = __ldcg(fvg + c);
      const cplx nr = __ldcg(nrg + c);
      nrow[c] = nr;
      if (c >= i + 2) sqp += cabs2(nr);
    }
    sqp = sum_to_warp0(sqp, i + 1 + 32 * wid < n, dred);  // its barriers also publish fv / nrow / vloc
    if (owner && tid == 0) {
      R(i / G, i) = bc[2];
      dg[i] = bc[2].x;
      tauq[i] = tq;
    }
    // warp 0 forms the right reflector of the updated row i (every CTA
    // does; it zeroes the row beyond i+1) while warps 1.. apply the left
    // reflector to the own rows: A[r,c] -= v_r conj(tau) w_c, column i
    // keeps v_r
    if (wid == 0) {
      if (lane == 0 && i + 1 < n) {
        cplx tp, sp;
        double beta;
        house_scalars(cconj(nrow[i + 1]), sqp, &tp, &sp, &beta);
        bcr[0] = tp;
        bcr[1] = sp;
        bcr[2] = mk(beta, 0.0);
      }
    } else {
      const int t1 = tid - 32, nt1 = blockDim.x - 32;
      for (int c = i + 1 + t1; c < n; c += nt1) {
        const cplx f = fv[c];
        const cplx nf = mk(-f.x, -f.y);
        for (int lr = lr0; lr < nact; ++lr) R(lr, c) = cfma(vloc[lr], nf, R(lr, c));
      }
      for (int lr = lr0 + t1; lr < nact; lr += nt1) R(lr, i) = vloc[lr];
    }
    if (i + 1 >= n) break;
    __syncthreads();
    const cplx tp = bcr[0], scp = bcr[1];
    for (int c = i + 1 + tid; c < n; c += blockDim.x) {
      const cplx u = (c == i + 1) ? mk(1, 0) : cmul(cconj(nrow[c]), scp);
      uv[c] = u;
      if (owner) R(i / G, c) = (c == i + 1) ? bcr[2] : cconj(u);
    }
    if (owner && tid == 0) {
      eg[i] = bcr[2].x;
      taup[i] = tp;
    }
    __syncthreads();
    // right update of own rows r > i: A[r,:] -= taup (A[r,:] . u) u^H
    for (int lr = lr0 + wid; lr < nact; lr += nw) {
      // four interleaved partial dot products (a dependent FP64 FMA chain
      // costs 64-128 cycles per step on this GPU)
      cplx d0 = mk(0, 0), d1 = mk(0, 0), d2 = mk(0, 0), d3 = mk(0, 0);
      int c = i + 1 + lane;
      for (; c + 96 < n; c += 128) {
        d0 = cfma(R(lr, c), uv[c], d0);
        d1 = cfma(R(lr, c + 32), uv[c + 32], d1);
        d2 = cfma(R(lr, c + 64), uv[c + 64], d2);
        d3 = cfma(R(lr, c + 96), uv[c + 96], d3);
      }
      for (; c < n; c += 32) d0 = cfma(R(lr, c), uv[c], d0);
      cplx dot = warp_sum(cadd(cadd(d0, d1), cadd(d2, d3)));
      const cplx f = cmul(tp, dot);
      const cplx nf = mk(-f.x, -f.y);
      for (int c = i + 1 + lane; c < n; c += 32) R(lr, c) = cfma(nf, cconj(uv[c]), R(lr, c));
    }
    __syncthreads();
  }
  __syncthreads();
  for (int lr = 0; lr < nact; ++lr) {
    const int r = grow(lr);
    for (int c = tid; c < n; c += blockDim.x) A[r + (size_t)lda * c] = R(lr, c);
  }
}

// Grid of the bidiagonalisation: rows resident in shared memory when they
// fit (*global_rows = false), else all SMs with the rows in a global
// workspace of gebrd_rows_elems(n) elements (when allowed).
int gebrd_grid(int n, int sms, int* nloc_out, size_t* smem_out, bool allow_global, bool* global_rows) {
  const DevInfo& di = dev_info();
  int G = std::max(1, std::min(sms, (n + 2) / 3));
  *global_rows = false;
  for (;;) {
    const int nloc = (n + G - 1) / G;
    const size_t smem = ((size_t)nloc * n + 3 * (size_t)n + nloc) * sizeof(cplx);
    if (smem + 8192 <= (size_t)di.max_smem_optin) {
      *nloc_out = nloc;
      *smem_out = smem;
      return G;
    }
    if (G >= sms) break;
    G = std::min(sms, G + 8);
  }
  const int nloc = (n + G - 1) / G;
  const size_t smem = (3 * (size_t)n + nloc) * sizeof(cplx);
  if (!allow_global || smem + 8192 > (size_t)di.max_smem_optin) return 0;
  *global_rows = true;
  *nloc_out = nloc;
  *smem_out = smem;
  return G;
}

size_t gebrd_rows_elems(int n, int sms) {
  const int G = std::max(1, std::min(sms, (n + 2) / 3));
  return (size_t)(n + G) * (size_t)n;
}

size_t bd_vectors_smem(int n);

bool gebrd_fits(int n, const CoopWs& ws, bool have_rows_ws) {
  int nloc;
  size_t smem;
  bool glob;
  return n >= 1 && gebrd_grid(n, coop_sms(ws), &nloc, &smem, have_rows_ws, &glob) > 0 &&
         bd_vectors_smem(n) <= (size_t)dev_info().max_smem_optin;
}

cudaError_t gebrd(cplx* A, int lda, int n, double* d, double* e, cplx* tauq, cplx* taup,
                  const CoopWs& ws, cudaStream_t s, cplx* rows_ws) {
  if (n <= 0) return cudaSuccess;
  int nloc;
  size_t smem;
  bool glob = false;
  const int G = gebrd_grid(n, coop_sms(ws), &nloc, &smem, rows_ws != nullptr, &glob);
  if (G <= 0) return cudaErrorInvalidValue;
  cplx* rows_global = glob ? rows_ws : nullptr;
  if ((size_t)2 * G * (n + 1) > ws.pc_elems || (size_t)6 * n > ws.wfin_elems || 2 * G > 1024)
    return cudaErrorInvalidValue;
  cudaError_t err = allow_smem((const void*)gebrd_kernel, smem);
  if (err != cudaSuccess) return err;
  err = cudaMemsetAsync(&ws.bar->count, 0, sizeof(unsigned int), s);
  if (err != cudaSuccess) return err;
  CoopWs w = ws;
  void* args[] = {&A, &lda, &n, &nloc, &d, &e, &tauq, &taup, &w, &rows_global};
  return cudaLaunchCooperativeKernel((void*)gebrd_kernel, dim3(G), dim3(kBdThreads), args, smem, s);
}

// ---- 2. singular values ------------------------------------------------------------
// Double-float reals: value = h + l, |l| <= ulp(h)/2.
struct dfr {
  float h, l;
};
DV dfr df_quick(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return dfr{s, b - (s - a)};
}
DV dfr df_add(dfr a, dfr b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float e = (a.h - (s - bb)) + (b.h - bb) + a.l + b.l;
  return df_quick(s, e);
}
DV dfr df_div(dfr a, dfr b) {
  // long division: q1 = a/b to FP32, exact remainder a - q1 b, q2 = rem/b
  const float r = __frcp_rn(b.h);
  const float q1 = a.h * r;
  const float p = q1 * b.h;
  const float pe = fmaf(q1, b.h, -p);
  const float rem = (((a.h - p) - pe) + a.l) - q1 * b.l;
  return df_quick(q1, rem * r);
}
DV dfr df_of(double x) {
  const float h = (float)x;
  return dfr{h, (float)(x - (double)h)};
}

// Prepare the scaled squared off-diagonals of T_GK: a_k = d[k/2] (k even),
// e[k/2] (k odd), k < 2n-1; a2[k] = (a_k / amax)^2 as double-float;
// info[0] = amax, info[1] = Gershgorin bound of T_GK / amax.
__global__ void bd_prep_kernel(const double* __restrict__ d, const double* __restrict__ e, int n,
                               float2* __restrict__ a2, double* __restrict__ info) {
  __shared__ double red[32];
  const int N = 2 * n;
  auto off = [&](int k) { return (k & 1) ? e[k >> 1] : d[k >> 1]; };
  const int nw = blockDim.x >> 5;
  double m = 0.0;
  for (int k = threadIdx.x; k < N - 1; k += blockDim.x) m = fmax(m, fabs(off(k)));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double amax = 0.0;
  for (int w = 0; w < nw; ++w) amax = fmax(amax, red[w]);
  __syncthreads();
  const double inv = amax > 0.0 ? 1.0 / amax : 0.0;
  double bnd = 0.0;
  for (int k = threadIdx.x; k < N - 1; k += blockDim.x) {
    const double a = fabs(off(k)) * inv;
    const double a_sq = a * a;
    float2 v = make_float2(0.f, 0.f);
    if (a_sq >= 1e-36) {
      v.x = (float)a_sq;
      v.y = (float)(a_sq - (double)v.x);
    }
    a2[k] = v;
    // row k+1 of T_GK holds a_k and a_{k+1}
    const double nb = (k + 1 < N - 1) ? fabs(off(k + 1)) * inv : 0.0;
    bnd = fmax(bnd, a + nb);
  }
  for (int o = 16; o > 0; o >>= 1) bnd = fmax(bnd, __shfl_xor_sync(0xffffffffu, bnd, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bnd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < nw; ++w) b = fmax(b, red[w]);
    info[0] = amax;
    info[1] = b * (1.0 + 1e-6) + 1e-30;
  }
}

// Number of eigenvalues of the scaled T_GK below x: negative pivots of the
// LDL^T factorisation of T_GK - x I (pivots clamped away from zero).
__device__ __forceinline__ int sturm_count_df(const float2* __restrict__ a2, int N, double x) {
  const float pivmin = 1e-30f;
  const dfr xd = df_of(x);
  dfr q{-xd.h, -xd.l};
  if (fabsf(q.h) < pivmin) q = dfr{-pivmin, 0.f};
  int cnt = (q.h < 0.f);
  for (int k = 1; k < N; ++k) {
    const float2 a = __ldg(a2 + k - 1);
    const dfr t = df_div(dfr{a.x, a.y}, q);
    const dfr s = df_add(xd, t);
    q = dfr{-s.h, -s.l};
    if (fabsf(q.h) < pivmin) q = dfr{-pivmin, 0.f};
    cnt += (q.h < 0.f);
  }
  return cnt;
}

// One warp per value: sig[k] = k-th largest singular value of B.  The
// bracket [lo, hi) keeps #{sigma < lo} < target <= #{sigma < hi} with
// target = n - k; each round the lanes count at 32 interior points.
__global__ void bd_sigma_kernel(const float2* __restrict__ a2, const double* __restrict__ info, int n,
                                double* __restrict__ sig) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= n) return;
  const double amax = info[0];
  if (amax == 0.0) {
    if (lane == 0) sig[k] = 0.0;
    return;
  }
  const int N = 2 * n, target = n - k;
  double lo = 0.0, hi = info[1];
  for (int it = 0; it < 24; ++it) {
    if (hi - lo <= 0x1p-42 * hi || hi - lo <= 1e-32) break;
    const double x = lo + (hi - lo) * (double)(lane + 1) * (1.0 / 33.0);
    const int below = sturm_count_df(a2, N, x) - n;
    const unsigned ok = __ballot_sync(0xffffffffu, below >= target);
    const int first = ok ? (__ffs(ok) - 1) : 32;
    const double xl = __shfl_sync(0xffffffffu, x, first == 0 ? 0 : first - 1);
    const double xh = __shfl_sync(0xffffffffu, x, first == 32 ? 31 : first);
    if (first > 0) lo = xl;
    if (first < 32) hi = xh;
  }
  if (lane == 0) sig[k] = 0.5 * (lo + hi) * amax;
}

cudaError_t bd_sigma(const double* d, const double* e, int n, float2* a2, double* info, double* sig,
                     cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  bd_prep_kernel<<<1, 256, 0, s>>>(d, e, n, a2, info);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int warps = 4;
  bd_sigma_kernel<<<(n + warps - 1) / warps, 32 * warps, 0, s>>>(a2, info, n, sig);
  return cudaGetLastError();
}
// Rank rule on the sorted values (the same rule as rank_select), one CTA:
// suffix sums of sigma^2 by a block scan, the rank as the smallest index
// that passes the test.
constexpr int kRankThreads = 256;
__global__ void __launch_bounds__(kRankThreads)
bd_rank_kernel(const double* __restrict__ sig, int n, const double* __restrict__ eps_hat, int cap,
               int forced, int* __restrict__ out_int, double* __restrict__ out_dbl,
               double* __restrict__ tail2) {
  __shared__ double wtot[kRankThreads / 32];
  __shared__ int rmin[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = (n + kRankThreads - 1) / kRankThreads;
  const int a = min(n, tid * per), b = min(n, a + per);
  double own = 0.0;
  for (int r = a; r < b; ++r) own += sig[r] * sig[r];
  // suffix sum over threads: inclusive from the right within the warp
  double suf = own;
  for (int o = 1; o < 32; o <<= 1) {
    const double v = __shfl_down_sync(0xffffffffu, suf, o);
    if (lane + o < 32) suf += v;
  }
  if (lane == 0) wtot[wid] = suf;
  if (tid == 0) {
    rmin[0] = n;
    rmin[1] = n;
  }
  __syncthreads();
  double after = 0.0;  // sum over later warps
  for (int w = wid + 1; w < kRankThreads / 32; ++w) after += wtot[w];
  // tail2[r] = sum_{q >= r} sig_q^2 for this thread's chunk
  double run = suf - own + after;  // everything after this chunk
  for (int r = b - 1; r >= a; --r) {
    run += sig[r] * sig[r];
    tail2[r] = run;
  }
  if (tid == 0) tail2[n] = 0.0;
  __syncthreads();
  const double eh = *eps_hat;
  const double fro = sqrt(tail2[0]);
  const double thr = 2.0 * n * DBL_EPSILON * fro;
  for (int r = 1 + tid; r <= n; r += kRankThreads)
    if (sqrt(tail2[r]) <= eh) atomicMin(&rmin[0], r);
  for (int k = tid; k < n; k += kRankThreads)
    if (!(sig[k] > thr)) atomicMin(&rmin[1], k);
  __syncthreads();
  if (tid == 0) {
    const int rho_tol = rmin[0];
    int rho = forced > 0 ? forced : (rho_tol < cap ? rho_tol : cap);
    rho = rho < 1 ? 1 : (rho > n ? n : rho);
    // kept values at the noise level of a factorisation of B (their vectors
    // are not determined by B and are completed instead)
    const int kt = min(rmin[1], rho);
    out_int[0] = rho;
    out_int[1] = rho_tol;
    out_int[2] = kt;
    out_dbl[0] = sqrt(tail2[rho]);
    out_dbl[1] = sig[rho - 1];
    out_dbl[2] = tail2[0];
  }
}

cudaError_t bd_rank(const double* sig, int n, const double* eps_hat, int cap, int forced, int* out_int,
                    double* out_dbl, double* tail2, cudaStream_t s) {
  bd_rank_kernel<<<1, kRankThreads, 0, s>>>(sig, n, eps_hat, cap, forced, out_int, out_dbl, tail2);
  return cudaGetLastError();
}

// ---- 3. singular vectors of B -------------------------------------------------------------
DV double hash_unit(unsigned a, unsigned b) {
  unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (double)(h & 0xFFFFFFu) * (1.0 / 16777216.0) - 0.5;
}

// Solver arrays of T_GK - lam I (length N each) in shared memory, and the
// scaled off-diagonals (staged once per launch).
enum { L_DINV = 0, L_C1 = 1, L_C2 = 2, L_DL = 3, L_PV = 4, L_B = 5, L_OFF = 6 };
constexpr int kSolveArrays = 7;
size_t bd_vectors_smem(int n) { return sizeof(double) * kSolveArrays * 2 * (size_t)n; }

// LU with partial pivoting of T_GK - lam I (off-diagonals at L_OFF, scaled
// by 1 / amax); one thread.  Row i of U is stored as (1 / pivot, super /
// pivot, second super / pivot), so that the back substitution has one
// dependent multiply-add per row, and the multiplier uses the reciprocal of
// the pivot: one reciprocal and one multiply-add on the serial chain.
DV void gk_factor(int N, double lam, double* w) {
  double* Dinv = w + L_DINV * N;
  double* C1 = w + L_C1 * N;
  double* C2 = w + L_C2 * N;
  double* DL = w + L_DL * N;
  double* PV = w + L_PV * N;
  const double* off = w + L_OFF * N;
  const double tiny = 4.0 * DBL_EPSILON;
  auto guard = [&](double p) { return fabs(p) < tiny ? (p < 0.0 ? -tiny : tiny) : p; };
  double di = -lam, dui = (N > 1) ? off[0] : 0.0;
  double sub = dui;
  for (int i = 0; i < N - 1; ++i) {
    const double un = (i + 1 < N - 1) ? off[i + 1] : 0.0;
    if (fabs(di) >= fabs(sub)) {
      const double rp = 1.0 / guard(di);
      const double f = sub * rp;
      Dinv[i] = rp;
      C1[i] = dui * rp;
      C2[i] = 0.0;
      DL[i] = f;
      PV[i] = 0.0;
      di = fma(-f, dui, -lam);
      dui = un;
    } else {
      // rows i and i+1 swapped: new row i = (sub, -lam, un)
      const double rs = 1.0 / sub;
      const double f = di * rs;
      Dinv[i] = rs;
      C1[i] = -lam * rs;
      C2[i] = un * rs;
      DL[i] = f;
      PV[i] = 1.0;
      di = fma(f, lam, dui);
      dui = -f * un;
    }
    sub = un;  // the sub-diagonal of row i+2 equals the super-diagonal off(i+1)
  }
  Dinv[N - 1] = 1.0 / guard(di);
}

// Solve with the factors, in place on B; one thread.
DV void gk_solve(int N, double* w) {
  const double* Dinv = w + L_DINV * N;
  const double* C1 = w + L_C1 * N;
  const double* C2 = w + L_C2 * N;
  const double* DL = w + L_DL * N;
  const double* PV = w + L_PV * N;
  double* B = w + L_B * N;
  double cur = B[0];
  for (int i = 0; i < N - 1; ++i) {
    const double bn = B[i + 1], f = DL[i];
    if (PV[i] != 0.0) {
      B[i] = bn;
      cur = fma(-f, bn, cur);
    } else {
      B[i] = cur;
      cur = fma(-f, cur, bn);
    }
  }
  double x2 = 0.0, x1 = cur * Dinv[N - 1];
  B[N - 1] = x1;
  for (int i = N - 2; i >= 0; --i) {
    // x2 is known one row earlier than x1: only the last multiply-add waits on x1
    const double t = fma(-C2[i], x2, B[i] * Dinv[i]);
    const double x = fma(-C1[i], x1, t);
    B[i] = x;
    x2 = x1;
    x1 = x;
  }
}

// One warp per cluster of kept values (consecutive values closer than
// 1e-3 sigma_max): inverse iteration for each member, re-orthogonalised
// against the members before it.  Lane 0 runs the tridiagonal recurrences
// out of shared memory; the warp does the products and norms.  X (n x
// nvec, ldx) receives the normalised left vectors u_k.  Every k < nvec is
// above the noise level (the caller passes the count of such values).
__global__ void bd_vectors_kernel(const double* __restrict__ d, const double* __restrict__ e, int n,
                                  const double* __restrict__ info, const double* __restrict__ sig,
                                  int nvec, double* __restrict__ X, int ldx, double* __restrict__ Zs) {
  extern __shared__ __align__(16) double vsm[];  // kSolveArrays * N
  const int k0 = blockIdx.x, lane = threadIdx.x;
  const int N = 2 * n;
  if (k0 >= nvec) return;
  const double amax = info[0];
  if (amax == 0.0) return;
  const double gap_tol = 1e-3 * sig[0];
  if (k0 > 0 && sig[k0 - 1] - sig[k0] < gap_tol) return;  // not the first of its cluster
  int k1 = k0 + 1;
  while (k1 < nvec && sig[k1 - 1] - sig[k1] < gap_tol) ++k1;
  const double inv = 1.0 / amax;
  double* B = vsm + L_B * N;
  double* off = vsm + L_OFF * N;
  for (int i = lane; i < N - 1; i += 32) off[i] = ((i & 1) ? e[i >> 1] : d[i >> 1]) * inv;
  __syncwarp();
  for (int k = k0; k < k1; ++k) {
    if (lane == 0) gk_factor(N, sig[k] * inv, vsm);
    for (int i = lane; i < N; i += 32) B[i] = 1.0 + 0.25 * hash_unit((unsigned)i, (unsigned)k);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
      if (lane == 0) gk_solve(N, vsm);
      __syncwarp();
      for (int j = k0; j < k; ++j) {
        const double* zj = Zs + (size_t)j * N;
        double dot = 0.0;
        for (int i = lane; i < N; i += 32) dot += zj[i] * B[i];
        dot = warp_sum(dot);
        for (int i = lane; i < N; i += 32) B[i] -= dot * zj[i];
        __syncwarp();
      }
      double nrm = 0.0;
      for (int i = lane; i < N; i += 32) nrm += B[i] * B[i];
      nrm = warp_sum(nrm);
      const double s = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
      for (int i = lane; i < N; i += 32) B[i] *= s;
      __syncwarp();
    }
    double* zk = Zs + (size_t)k * N;
    double un = 0.0;
    for (int i = lane; i < N; i += 32) {
      const double z = B[i];
      zk[i] = z;
      if (i & 1) un += z * z;
    }
    un = warp_sum(un);
    const double s = un > 0.0 ? 1.0 / sqrt(un) : 0.0;
    for (int i = lane; i < n; i += 32) X[i + (size_t)ldx * k] = B[2 * i + 1] * s;
    __syncwarp();
  }
}

// Orthonormal completion for kept values at the noise level (indices
// kt..nvec-1): pseudo-random vectors, classical Gram-Schmidt twice against
// every earlier column of X.  One CTA.
__global__ void bd_complete_kernel(int n, int kt, int nvec, double* __restrict__ X, int ldx) {
  extern __shared__ __align__(16) unsigned char cs_smem[];
  double* x = reinterpret_cast<double*>(cs_smem);  // n
  double* dots = x + n;                             // nvec
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = kt; k < nvec; ++k) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = hash_unit((unsigned)i + 7919u, (unsigned)k * 31u + 3u);
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = wid; j < k; j += nw) {
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s += X[i + (size_t)ldx * j] * x[i];
        s = warp_sum(s);
        if (lane == 0) dots[j] = s;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = x[i];
        for (int j = 0; j < k; ++j) v -= dots[j] * X[i + (size_t)ldx * j];
        x[i] = v;
      }
      __syncthreads();
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i] * x[i];
    s = block_sum(s, red);
    const double sc = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) X[i + (size_t)ldx * k] = x[i] * sc;
    __syncthreads();
  }
}


cudaError_t bd_vectors(const double* d, const double* e, int n, const double* info, const double* sig,
                       int kt, int nvec, double* X, int ldx, double* Zs, cudaStream_t s) {
  if (nvec <= 0) return cudaSuccess;
  if (kt > 0) {
    const size_t smem = bd_vectors_smem(n);
    cudaError_t err = allow_smem((const void*)bd_vectors_kernel, smem);
    if (err != cudaSuccess) return err;
    bd_vectors_kernel<<<kt, 32, smem, s>>>(d, e, n, info, sig, kt, X, ldx, Zs);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (kt < nvec) {
    const size_t smem = sizeof(double) * ((size_t)n + nvec);
    bd_complete_kernel<<<1, 256, smem, s>>>(n, kt, nvec, X, ldx);
  }
  return cudaGetLastError();
}

// ---- 4. back-transformation -------------------------------------------------------------------
// u_k <- Q u_k with Q = H_0 H_1 ... H_{n-1} (reflector j: unit entry at j,
// tail A[j+1:n, j], tau[j]).  One vector per CTA, so that the FP64 work
// (about 10 n^2 / 2 operations per vector) spreads over many SMs; warp 0
// applies reflector j while warp 1 stages reflector j-1 in shared memory.
// The result goes to U (n x nvec, ldu) and to Xp (mrows x nvec, ldp, zero
// below row n).
__global__ void __launch_bounds__(64)
bd_back_kernel(const cplx* __restrict__ A, int lda, const cplx* __restrict__ tauq, int n,
               const double* __restrict__ Xr, int ldx, int nvec, cplx* __restrict__ U, int ldu,
               cplx* __restrict__ Xp, int ldp, int mrows) {
  extern __shared__ __align__(16) unsigned char bk_smem[];
  cplx* vb = reinterpret_cast<cplx*>(bk_smem);  // [2][n] staged reflectors
  cplx* x = vb + 2 * (size_t)n;                 // [n]
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x;
  if (k >= nvec) return;
  auto stage = [&](int j) {  // reflector j into vb[j & 1][j..n)
    cplx* v = vb + (size_t)(j & 1) * n;
    for (int i = j + lane; i < n; i += 32) v[i] = (i == j) ? mk(1, 0) : __ldg(A + i + (size_t)lda * j);
  };
  if (wid == 0) {
    for (int i = lane; i < n; i += 32) x[i] = mk(Xr[i + (size_t)ldx * k], 0.0);
  } else {
    stage(n - 1);
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    if (wid == 1) {
      if (j > 0) stage(j - 1);
    } else {
      const cplx t = __ldg(tauq + j);
      if (t.x != 0.0 || t.y != 0.0) {
        const cplx* v = vb + (size_t)(j & 1) * n;
        cplx acc = mk(0, 0);
        for (int i = j + lane; i < n; i += 32) acc = cfmac(v[i], x[i], acc);
        acc = warp_sum(acc);
        const cplx f = cmul(t, acc);
        const cplx nf = mk(-f.x, -f.y);
        for (int i = j + lane; i < n; i += 32) x[i] = cfma(v[i], nf, x[i]);
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < mrows; i += blockDim.x) {
    const cplx v = (i < n) ? x[i] : mk(0, 0);
    if (i < n) U[i + (size_t)ldu * k] = v;
    Xp[i + (size_t)ldp * k] = v;
  }
}

cudaError_t bd_back(const cplx* A, int lda, const cplx* tauq, int n, const double* X, int ldx, int nvec,
                    cplx* U, int ldu, cplx* Xp, int ldp, int mrows, cudaStream_t s) {
  if (nvec <= 0) return cudaSuccess;
  const size_t smem = sizeof(cplx) * (size_t)n * 3;
  cudaError_t err = allow_smem((const void*)bd_back_kernel, smem);
  if (err != cudaSuccess) return err;
  bd_back_kernel<<<nvec, 64, smem, s>>>(A, lda, tauq, n, X, ldx, nvec, U, ldu, Xp, ldp, mrows);
  return cudaGetLastError();
}

}  // namespace hk
