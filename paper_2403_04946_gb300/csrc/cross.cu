// TT-cross interpolation of the Gaussian initial state (Sec. 5's Gaussian
// random initial condition; TT cross approximation after Oseledets &
// Tyrtyshnikov 2010) for grids too large to form in full.
//
// Phi0(a) = exp(i a.m - a^T C a / 2) is evaluated exactly on index sets:
// a left set I_k (multi-indices over modes 0..k-1), every grid point of
// mode k, and a right set J_{k+1} (modes k+1..d-1).  Complete-pivoting
// elimination on that fiber matrix picks a well-conditioned square
// submatrix G (rows -> the next left set, columns -> the right indices
// kept); the core is the chosen columns of the fiber matrix times G^-1, so
// the TT reproduces Phi0 exactly on the cross points.  Slot 0 of every mode
// is the zero boundary slot and is never a pivot.
#include <algorithm>
#include <cfloat>

#include "kernels.h"

namespace hk {

constexpr int kCrossMaxD = 64;

// A[(alpha + rl i) + rl n beta] = Phi0(Il[alpha], i, Jr[beta]) with the free
// index on mode kl: Il is rl x kl (row-major tuples over modes 0..kl-1), Jr
// is rr x (d-kl-1) (modes kl+1..d-1).  One thread per (alpha, beta) forms
// the quadratic form of the fixed modes once and runs over i.
__global__ void gauss_fibers_kernel(const double* __restrict__ agrid, int n, int d,
                                    const double* __restrict__ m, const double* __restrict__ C,
                                    const int* __restrict__ Il, int rl, int kl,
                                    const int* __restrict__ Jr, int rr, cplx* __restrict__ A) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)rl * rr) return;
  const int alpha = (int)(tid % rl), beta = (int)(tid / rl);
  const int kr = d - kl - 1;
  double a[kCrossMaxD];
  int zero = 0;
  for (int t = 0; t < d; ++t) {
    int idx = -1;
    if (t < kl) idx = Il[(size_t)alpha * kl + t];
    else if (t > kl) idx = Jr[(size_t)beta * kr + (t - kl - 1)];
    if (idx == 0) zero = 1;
    a[t] = (idx > 0) ? agrid[idx] : 0.0;
  }
  cplx* out = A + (size_t)rl * n * beta + alpha;
  if (zero) {
    for (int i = 0; i < n; ++i) out[(size_t)rl * i] = mk(0, 0);
    return;
  }
  // q = sum_{s,t != kl} a_s C_st a_t, lin = sum_{t != kl} C_{kl,t} a_t,
  // ph = sum_{t != kl} m_t a_t (a_kl = 0 in the array)
  double q = 0.0, lin = 0.0, ph = 0.0;
  for (int s = 0; s < d; ++s) {
    double row = 0.0;
    for (int t = 0; t < d; ++t) row += C[s + (size_t)d * t] * a[t];
    q += a[s] * row;
    lin += C[kl + (size_t)d * s] * a[s];
    ph += m[s] * a[s];
  }
  const double ckk = C[kl + (size_t)d * kl], mkl = m[kl];
  out[0] = mk(0, 0);  // zero boundary slot
  for (int i = 1; i < n; ++i) {
    const double x = agrid[i];
    const double re = -0.5 * (q + 2.0 * x * lin + ckk * x * x);
    double sn, cn;
    sincos(ph + mkl * x, &sn, &cn);
    const double e = exp(re);
    out[(size_t)rl * i] = mk(e * cn, e * sn);
  }
}

cudaError_t gauss_fibers(const double* agrid, int n, int d, const double* m, const double* C, const int* Il,
                         int rl, int kl, const int* Jr, int rr, cplx* A, cudaStream_t s) {
  if (d > kCrossMaxD || kl < 0 || kl >= d || rl < 1 || rr < 1) return cudaErrorInvalidValue;
  const long long total = (long long)rl * rr;
  const int threads = 128;
  gauss_fibers_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>(agrid, n, d, m, C, Il, rl,
                                                                                       kl, Jr, rr, A);
  return cudaGetLastError();
}

// Complete-pivoting elimination of the M x c matrix A (lda = M), FP64, as
// a cooperative kernel: CTA g owns rows [g R, g R + R) of the working copy
// W (M x c).  Step j: every CTA offers the entry of largest modulus among
// its rows and the columns not yet used; after one grid barrier every CTA
// picks the same winner (p, q) (ties: lowest flat index), reads row p, and
// removes the pivot from its own rows: W[i,l] -= (W[i,q] / W[p,q]) W[p,l].
// Used rows and columns are skipped, never rewritten, so the pivot row read
// in step j is final.  Stops when the largest remaining entry is below
// rel_tol times the first pivot.  rows[cnt], cols[cnt], *count = cnt.
constexpr int kPivThreads = 256;
__global__ void __launch_bounds__(kPivThreads, 1)
cross_pivots_kernel(const cplx* __restrict__ A, int M, int c, int R, double rel_tol, cplx* __restrict__ W,
                    int* __restrict__ rows, int* __restrict__ cols, int* __restrict__ count, CoopWs ws) {
  __shared__ double bv[kPivThreads / 32];
  __shared__ long long bi[kPivThreads / 32];
  __shared__ cplx prow[256];
  __shared__ unsigned char colused[256];
  __shared__ unsigned char rowused[1024];
  __shared__ long long pick;
  __shared__ double pickv;
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int r0 = g * R, r1 = min(M, r0 + R), nr = max(0, r1 - r0);
  GridSync gs{ws.bar, 0u};
  for (long long e = tid; e < (long long)nr * c; e += blockDim.x) {
    const int i = r0 + (int)(e % nr), l = (int)(e / nr);
    W[i + (size_t)M * l] = A[i + (size_t)M * l];
  }
  for (int l = tid; l < c; l += blockDim.x) colused[l] = 0;
  for (int i = tid; i < nr; i += blockDim.x) rowused[i] = 0;
  __syncthreads();
  double first = 0.0;
  int cnt = 0;
  const int steps = min(M, c);
  for (int j = 0; j < steps; ++j) {
    // local candidate
    double best = -1.0;
    long long be = 0;
    for (long long e = tid; e < (long long)nr * c; e += blockDim.x) {
      const int il = (int)(e % nr), l = (int)(e / nr);
      if (rowused[il] || colused[l]) continue;
      const long long fe = (long long)(r0 + il) + (long long)M * l;
      const double v = cabs2(W[fe]);
      if (v > best || (v == best && fe < be)) {
        best = v;
        be = fe;
      }
    }
    for (int o = 16; o >= 1; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const long long oe = __shfl_xor_sync(0xffffffffu, be, o);
      if (ov > best || (ov == best && oe < be)) {
        best = ov;
        be = oe;
      }
    }
    if (lane == 0) {
      bv[wid] = best;
      bi[wid] = be;
    }
    __syncthreads();
    cplx* cand = ws.pc + (size_t)(j & 1) * G;
    if (tid == 0) {
      double b = bv[0];
      long long ee = bi[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (bv[w] > b || (bv[w] == b && bi[w] < ee)) {
          b = bv[w];
          ee = bi[w];
        }
      cand[g] = mk(b, (double)ee);  // flat index < 2^53: exact in a double
    }
    grid_sync(gs);
    if (grid_failed(ws.bar)) return;
    if (tid == 0) {
      double b = -1.0;
      long long ee = 0;
      for (int gg = 0; gg < G; ++gg) {
        const cplx v = __ldcg(cand + gg);
        const long long ve = (long long)v.y;
        if (v.x > b || (v.x == b && ve < ee)) {
          b = v.x;
          ee = ve;
        }
      }
      pick = ee;
      pickv = b;
    }
    __syncthreads();
    const double b = pickv;
    if (j == 0) first = b;
    if (!(b > 0.0) || b < rel_tol * rel_tol * first) break;
    const int p = (int)(pick % M), q = (int)(pick / M);
    if (g == 0 && tid == 0) {
      rows[j] = p;
      cols[j] = q;
    }
    for (int l = tid; l < c; l += blockDim.x) prow[l] = __ldcg(W + p + (size_t)M * l);
    if (tid == 0) colused[q] = 1;
    if (tid == 0 && p >= r0 && p < r1) rowused[p - r0] = 1;
    __syncthreads();
    const cplx pinv = cinv(prow[q]);
    for (int il = tid; il < nr; il += blockDim.x) {
      if (rowused[il]) continue;
      const int i = r0 + il;
      const cplx f = cmul(W[i + (size_t)M * q], pinv);
      const cplx nf = mk(-f.x, -f.y);
      for (int l = 0; l < c; ++l)
        if (!colused[l]) W[i + (size_t)M * l] = cfma(nf, prow[l], W[i + (size_t)M * l]);
    }
    __syncthreads();
    cnt = j + 1;
  }
  if (g == 0 && tid == 0) *count = cnt;
}

cudaError_t cross_pivots(const cplx* A, int M, int c, double rel_tol, cplx* W, int* rows, int* cols, int* count,
                         const CoopWs& ws, cudaStream_t s) {
  if (c > 256 || M < 1 || c < 1) return cudaErrorInvalidValue;
  const DevInfo& di = dev_info();
  const int sms = coop_sms(ws);
  int G = std::max(1, std::min(sms, (M + 63) / 64));
  int R = (M + G - 1) / G;
  if (R > 1024) {
    R = 1024;
    G = (M + R - 1) / R;
    if (G > sms) return cudaErrorInvalidValue;
  }
  if ((size_t)2 * G > ws.pc_elems) return cudaErrorInvalidValue;
  cudaError_t err = cudaMemsetAsync(&ws.bar->count, 0, sizeof(unsigned int), s);
  if (err != cudaSuccess) return err;
  CoopWs w = ws;
  void* args[] = {(void*)&A, &M, &c, &R, &rel_tol, &W, &rows, &cols, &count, &w};
  return cudaLaunchCooperativeKernel((void*)cross_pivots_kernel, dim3(G), dim3(kPivThreads), args, 0, s);
}

// core (M x cnt) = A[:, cols] * G^-1 with G = A[rows, cols] (cnt x cnt),
// FP64.  One CTA inverts G by Gauss-Jordan with partial pivoting (in
// scratch Gi, cnt x cnt), then all CTAs form the product.
__global__ void cross_ginv_kernel(const cplx* __restrict__ A, int M, const int* __restrict__ rows,
                                  const int* __restrict__ cols, int cnt, cplx* __restrict__ Gw,
                                  cplx* __restrict__ Gi) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  __shared__ int piv;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int r = cnt;
  // Gw = G, Gi = I
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    Gw[e] = A[rows[i] + (size_t)M * cols[j]];
    Gi[e] = (i == j) ? mk(1, 0) : mk(0, 0);
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    // partial pivot in column j among rows >= j
    double best = -1.0;
    int bidx = j;
    for (int i = j + tid; i < r; i += blockDim.x) {
      const double v = cabs2(Gw[i + r * j]);
      if (v > best) {
        best = v;
        bidx = i;
      }
    }
    for (int o = 16; o >= 1; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ov > best || (ov == best && oi < bidx)) {
        best = ov;
        bidx = oi;
      }
    }
    if (lane == 0) {
      bv[wid] = best;
      bi[wid] = bidx;
    }
    __syncthreads();
    if (tid == 0) {
      double b = bv[0];
      int ii = bi[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (bv[w] > b || (bv[w] == b && bi[w] < ii)) {
          b = bv[w];
          ii = bi[w];
        }
      piv = ii;
    }
    __syncthreads();
    const int p = piv;
    if (p != j)
      for (int l = tid; l < r; l += blockDim.x) {
        cplx t = Gw[j + r * l];
        Gw[j + r * l] = Gw[p + r * l];
        Gw[p + r * l] = t;
        t = Gi[j + r * l];
        Gi[j + r * l] = Gi[p + r * l];
        Gi[p + r * l] = t;
      }
    __syncthreads();
    const cplx dinv = cinv(Gw[j + r * j]);
    for (int l = tid; l < r; l += blockDim.x) {
      Gw[j + r * l] = cmul(Gw[j + r * l], dinv);
      Gi[j + r * l] = cmul(Gi[j + r * l], dinv);
    }
    __syncthreads();
    // eliminate column j from the other rows; column j of Gw itself is not
    // rewritten here (other threads read it as the multipliers)
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e % r, l = e / r;
      if (i == j) continue;
      const cplx f = Gw[i + r * j];
      if (l != j) Gw[e] = csub(Gw[e], cmul(f, Gw[j + r * l]));
      Gi[e] = csub(Gi[e], cmul(f, Gi[j + r * l]));
    }
    __syncthreads();
    for (int i = tid; i < r; i += blockDim.x)
      if (i != j) Gw[i + r * j] = mk(0, 0);
    __syncthreads();
  }
}

__global__ void cross_core_kernel(const cplx* __restrict__ A, int M, const int* __restrict__ cols, int cnt,
                                  const cplx* __restrict__ Gi, cplx* __restrict__ core) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * cnt) return;
  const int i = (int)(e % M), j = (int)(e / M);
  cplx acc = mk(0, 0);
  for (int t = 0; t < cnt; ++t) acc = cfma(A[i + (size_t)M * cols[t]], Gi[t + (size_t)cnt * j], acc);
  core[e] = acc;
}

__global__ void cross_gather_kernel(const cplx* __restrict__ A, int M, const int* __restrict__ cols, int cnt,
                                    cplx* __restrict__ out, cplx* __restrict__ eye, int* __restrict__ seq) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * cnt) return;
  const int i = (int)(e % M), j = (int)(e / M);
  out[e] = A[i + (size_t)M * cols[j]];
  eye[e] = (i == j) ? mk(1, 0) : mk(0, 0);
  if (e < cnt) seq[e] = (int)e;
}

cudaError_t cross_gather(const cplx* A, int M, const int* cols, int cnt, cplx* out, cplx* eye, int* seq,
                         cudaStream_t s) {
  const long long total = (long long)M * cnt;
  cross_gather_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(A, M, cols, cnt, out, eye, seq);
  return cudaGetLastError();
}

cudaError_t cross_core(const cplx* A, int M, const int* rows, const int* cols, int cnt, cplx* Gw, cplx* Gi,
                       cplx* core, cudaStream_t s) {
  if (cnt < 1) return cudaErrorInvalidValue;
  cross_ginv_kernel<<<1, 1024, 0, s>>>(A, M, rows, cols, cnt, Gw, Gi);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const long long total = (long long)M * cnt;
  cross_core_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(A, M, cols, cnt, Gi, core);
  return cudaGetLastError();
}

}  // namespace hk
