// TT-level kernels: the operator apply (memory-bound stencil over the cores),
// block sums, point evaluation, Gaussian set-up, moments, and the dense
// FP64 helpers (transposes, norms, small GEMMs) the rounding sweep uses.
#include <algorithm>

#include <mutex>
#include <unordered_map>

#include "kernels.h"

namespace hk {

cudaError_t allow_smem(const void* fn, size_t need) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find(fn);
  if (it == done.end()) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    const size_t cap = (size_t)dev_info().max_smem_optin - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
    if (e != cudaSuccess) return e;
    it = done.emplace(fn, cap).first;
  }
  return need <= it->second ? cudaSuccess : cudaErrorInvalidValue;
}

int coop_sms(const CoopWs& ws) {
  const int sm = dev_info().sm_count;
  return ws.max_ctas > 0 ? std::min(ws.max_ctas, sm) : sm;
}

const DevInfo& dev_info() {
  static DevInfo di = [] {
    DevInfo d{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return d;
  }();
  return di;
}

static inline int nblk(size_t n, int t) { return (int)((n + t - 1) / t); }

// ---- operator apply ------------------------------------------------------------
// Y[(alpha, i), m, (beta, j)] = sum_m' W[alpha, beta][m, m'] X[i, m', j] with
// every W block one of the per-mode operators (op_apply): tridiagonal in
// (m, m'), or the CDF equation's cumulative K.  One thread per
// output element, consecutive threads along the fastest (left-rank) index, so
// loads of X and stores of Y are both coalesced 16-byte accesses.  The grid's
// y index walks the right-rank index q = (beta, j) and x the (alpha, i, m)
// plane, so that every index comes from 32-bit arithmetic (the plane is
// below 2^31 elements, checked by the launcher).
__global__ void apply_core_kernel(const cplx* __restrict__ X, int a, int n, int c,
                                  cplx* __restrict__ Y, int Al, int Ar,
                                  const unsigned char* __restrict__ blocks,
                                  const cplx* __restrict__ coef) {
  const int rows = Al * a;
  const int plane = rows * n;
  for (int q = blockIdx.y; q < Ar * c; q += gridDim.y) {
    const int be = q / c, j = q - be * c;
    const cplx* Xj = X + (size_t)a * n * j;
    cplx* Yq = Y + (size_t)plane * q;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < plane; idx += gridDim.x * blockDim.x) {
      const int m = idx / rows, p = idx - m * rows;
      const int al = p / a, i = p - al * a;
      const int op = blocks[al * Ar + be];
      cplx v = mk(0, 0);
      if (op != OP_NONE) v = op_apply(coef, op, n, Xj + i, (size_t)a, m);  // X[i, :, j], stride a
      Yq[idx] = v;
    }
  }
}

cudaError_t apply_core(const cplx* in, int a, int n, int c, cplx* out, int Al, int Ar,
                       const unsigned char* blocks_dev, const OpTable& ops, cudaStream_t s) {
  const size_t plane = (size_t)Al * a * n;
  const size_t nq = (size_t)Ar * c;
  if (plane == 0 || nq == 0) return cudaSuccess;
  if (plane >= (1u << 31) || nq >= (1u << 31)) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)std::min<size_t>(nblk(plane, 256), 1024), (unsigned)std::min<size_t>(nq, 65535));
  apply_core_kernel<<<grid, 256, 0, s>>>(in, a, n, c, out, Al, Ar, blocks_dev, ops.coef);
  return cudaGetLastError();
}

// ---- TT sum ----------------------------------------------------------------------
__global__ void sum_core_kernel(const SumTerm* __restrict__ terms, int nterms, int kind, int n,
                                cplx* __restrict__ out, int ora, int orc) {
  const size_t total = (size_t)ora * n * orc;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % ora);
    const size_t rest = e / ora;
    const int m = (int)(rest % n);
    const int q = (int)(rest / n);
    cplx v = mk(0, 0);
    int offa = 0, offc = 0;
    for (int t = 0; t < nterms; ++t) {
      const SumTerm T = terms[t];
      bool inside;
      int ii, jj;
      if (kind == 0) {  // first core: side by side along the right rank
        inside = (q >= offc && q < offc + T.rc);
        ii = p;
        jj = q - offc;
      } else if (kind == 2) {  // last core: stacked along the left rank
        inside = (p >= offa && p < offa + T.ra);
        ii = p - offa;
        jj = q;
      } else {  // interior: block diagonal
        inside = (p >= offa && p < offa + T.ra && q >= offc && q < offc + T.rc);
        ii = p - offa;
        jj = q - offc;
      }
      if (inside) {
        v = T.p[ii + (size_t)T.ra * m + (size_t)T.ra * n * jj];
        if (kind == 0) v = cmul(T.coef, v);
        break;
      }
      offa += T.ra;
      offc += T.rc;
    }
    out[e] = v;
  }
}

cudaError_t sum_core(const SumTerm* terms_dev, int nterms, int kind, int n, cplx* out, int ora,
                     int orc, cudaStream_t s) {
  const size_t total = (size_t)ora * n * orc;
  const int grid = std::min<size_t>(nblk(total, 256), (size_t)dev_info().sm_count * 16);
  sum_core_kernel<<<grid, 256, 0, s>>>(terms_dev, nterms, kind, n, out, ora, orc);
  return cudaGetLastError();
}

// ---- point evaluation --------------------------------------------------------------
// Phi[i_1..i_d] = C_1[0,i_1,:] C_2[:,i_2,:] ... C_d[:,i_d,0]; one CTA per point.
__global__ void eval_points_kernel(const cplx* const* __restrict__ cores,
                                   const int* __restrict__ ranks, int d, int n,
                                   const int* __restrict__ idx, cplx* __restrict__ vals) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int maxr = blockDim.y;  // unused, kept for clarity
  (void)maxr;
  cplx* v = reinterpret_cast<cplx*>(sm);
  const int pt = blockIdx.x;
  int rmax = 1;
  for (int k = 0; k <= d; ++k) rmax = max(rmax, ranks[k]);
  cplx* w = v + rmax;
  if (threadIdx.x == 0) v[0] = mk(1, 0);
  __syncthreads();
  for (int k = 0; k < d; ++k) {
    const int a = ranks[k], c = ranks[k + 1];
    const int ik = idx[(size_t)pt * d + k];
    const cplx* C = cores[k] + (size_t)a * ik;  // C[:, ik, :] with column stride a*n
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
      const cplx* col = C + (size_t)a * n * j;
      cplx acc = mk(0, 0);
      for (int i = 0; i < a; ++i) acc = cfma(v[i], col[i], acc);
      w[j] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < c; j += blockDim.x) v[j] = w[j];
    __syncthreads();
  }
  if (threadIdx.x == 0) vals[pt] = v[0];
}

cudaError_t eval_points(const cplx* const* cores_dev, const int* ranks_dev, int d, int n, int maxr,
                        int npts, const int* idx_dev, cplx* vals, cudaStream_t s) {
  if (npts <= 0) return cudaSuccess;
  const size_t smem = sizeof(cplx) * 2 * (size_t)std::max(maxr, 1);
  eval_points_kernel<<<npts, 128, smem, s>>>(cores_dev, ranks_dev, d, n, idx_dev, vals);
  return cudaGetLastError();
}

// ---- Gaussian initial state ------------------------------------------------------------
__global__ void gauss_rank1_kernel(const double* agrid, int n, double m, double c, cplx* core) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double a = agrid[i];
    const double mag = (i == 0) ? 0.0 : exp(-0.5 * c * a * a);
    double sn, cs;
    sincos(a * m, &sn, &cs);
    core[i] = mk(mag * cs, mag * sn);
  }
}

cudaError_t gauss_rank1_core(const double* agrid, int n, double m, double c, cplx* core,
                             cudaStream_t s) {
  gauss_rank1_kernel<<<nblk(n, 128), 128, 0, s>>>(agrid, n, m, c, core);
  return cudaGetLastError();
}

// Middle core of the exact full-grid TT: C[x, i, y] = Phi0(modes) with
// x = i_0 + n i_1 + ... (modes 0..c-1) and y = i_{c+1} + n i_{c+2} + ...
__global__ void gauss_full_kernel(const double* agrid, int n, int d, int c, const double* m0,
                                  const double* C0, cplx* core, size_t A, size_t B) {
  const size_t total = A * n * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int ind[64];
    size_t x = e % A;
    const size_t rest = e / A;
    ind[c] = (int)(rest % n);
    size_t y = rest / n;
    for (int k = 0; k < c; ++k) {
      ind[k] = (int)(x % n);
      x /= n;
    }
    for (int k = c + 1; k < d; ++k) {
      ind[k] = (int)(y % n);
      y /= n;
    }
    bool zero = false;
    double ph = 0.0, q = 0.0;
    for (int j = 0; j < d; ++j) {
      zero |= (ind[j] == 0);
      const double aj = agrid[ind[j]];
      ph += aj * m0[j];
      double row = 0.0;
      for (int k = 0; k < d; ++k) row += C0[j + (size_t)d * k] * agrid[ind[k]];
      q += aj * row;
    }
    cplx v = mk(0, 0);
    if (!zero) {
      const double mag = exp(-0.5 * q);
      double sn, cs;
      sincos(ph, &sn, &cs);
      v = mk(mag * cs, mag * sn);
    }
    core[e] = v;
  }
}

cudaError_t gauss_full_core(const double* agrid, int n, int d, int c, const double* m0,
                            const double* C0, cplx* core, cudaStream_t s) {
  size_t A = 1, B = 1;
  for (int k = 0; k < c; ++k) A *= n;
  for (int k = c + 1; k < d; ++k) B *= n;
  const size_t total = A * n * B;
  const int grid = std::min<size_t>(nblk(total, 256), (size_t)dev_info().sm_count * 16);
  gauss_full_kernel<<<grid, 256, 0, s>>>(agrid, n, d, c, m0, C0, core, A, B);
  return cudaGetLastError();
}

// Left identity core a x n x (a n): C[x, i, y] = [y == x + a i];
// right identity core (n b) x n x b: C[x, i, y] = [x == i + n y].
__global__ void identity_core_kernel(int n, int a, int b, int left, cplx* core) {
  const size_t total = (size_t)a * n * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t x = e % a;
    const size_t rest = e / a;
    const size_t i = rest % n;
    const size_t y = rest / n;
    const bool one = left ? (y == x + (size_t)a * i) : (x == i + (size_t)n * y);
    core[e] = mk(one ? 1.0 : 0.0, 0.0);
  }
}

cudaError_t identity_core(int n, int a, int b, int left, cplx* core, cudaStream_t s) {
  const size_t total = (size_t)a * n * b;
  const int grid = std::min<size_t>(nblk(total, 256), (size_t)dev_info().sm_count * 16);
  identity_core_kernel<<<grid, 256, 0, s>>>(n, a, b, left, core);
  return cudaGetLastError();
}

// Cell moments by tensor Gauss-Legendre (nodes/weights on [0,1] in gl[0..q),
// gl[q..2q)).  One thread per (j, k) pair; thread k of row d computes m0_k.
__global__ void cell_moments_kernel(int d, int nmodes, const double* alpha, const double* beta,
                                    double sigma, double ell, const double* gl, int q,
                                    double* m0, double* C0) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const double h = 2.0 * 3.14159265358979323846 / d;
  if (e < d * d) {
    const int j = e % d, k = e / d;
    double acc = 0.0;
    for (int u = 0; u < q; ++u) {
      const double x = (j + gl[u]) * h;
      double inner = 0.0;
      for (int v = 0; v < q; ++v) {
        const double y = (k + gl[v]) * h;
        const double sh = sin(0.5 * (x - y));
        inner += gl[q + v] * exp(-2.0 * sh * sh / (ell * ell));
      }
      acc += gl[q + u] * inner;
    }
    C0[e] = sigma * sigma * acc;
  } else if (e < d * d + d) {
    const int k = e - d * d;
    double acc = 0.0;
    for (int u = 0; u < q; ++u) {
      const double x = (k + gl[u]) * h;
      double mu = 0.0;
      for (int mm = 1; mm <= nmodes; ++mm) {
        double sn, cs;
        sincos(mm * x, &sn, &cs);
        mu += alpha[mm - 1] * cs + beta[mm - 1] * sn;
      }
      acc += gl[q + u] * mu;
    }
    m0[k] = acc;
  }
}

cudaError_t cell_moments(int d, int nmodes, const double* alpha, const double* beta,
                         double sigma, double ell, const double* gl, int q, double* m0,
                         double* C0, cudaStream_t s) {
  cell_moments_kernel<<<nblk((size_t)d * d + d, 128), 128, 0, s>>>(d, nmodes, alpha, beta, sigma,
                                                                  ell, gl, q, m0, C0);
  return cudaGetLastError();
}

__global__ void init_sh_pad_kernel(const cplx* S, int lds, int q, int p, cplx* X, int ldx,
                                   int mrows) {
  const size_t total = (size_t)mrows * q;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % mrows), l = (int)(e / mrows);
    X[r + (size_t)ldx * l] = (r < p) ? cconj(S[l + (size_t)lds * r]) : mk(0, 0);
  }
}

cudaError_t init_sh_pad(const cplx* S, int lds, int q, int p, cplx* X, int ldx, int mrows,
                        cudaStream_t s) {
  const size_t total = (size_t)mrows * q;
  if (total == 0) return cudaSuccess;
  const int grid = std::min<size_t>(nblk(total, 256), (size_t)dev_info().sm_count * 8);
  init_sh_pad_kernel<<<grid, 256, 0, s>>>(S, lds, q, p, X, ldx, mrows);
  return cudaGetLastError();
}

__global__ void gather_u_kernel(const cplx* src, int lds, int pp, const int* perm,
                                const double* sigma, int use_sigma, int rho, cplx* X, int ldx,
                                int mrows, cplx* Ub, int ldub) {
  const size_t total = (size_t)mrows * rho;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % mrows), l = (int)(e / mrows);
    cplx v = mk(0, 0);
    if (r < pp) {
      const int col = perm[l];
      v = src[r + (size_t)lds * col];
      if (use_sigma) {
        const double sg = sigma[col];
        v = (sg > 0.0) ? cscale(v, 1.0 / sg) : mk(0, 0);
      }
      Ub[r + (size_t)ldub * l] = v;
    }
    X[r + (size_t)ldx * l] = v;
  }
}

cudaError_t gather_u(const cplx* src, int lds, int pp, const int* perm, const double* sigma,
                     int use_sigma, int rho, cplx* X, int ldx, int mrows, cplx* Ub, int ldub,
                     cudaStream_t s) {
  const size_t total = (size_t)mrows * rho;
  if (total == 0) return cudaSuccess;
  const int grid = std::min<size_t>(nblk(total, 256), (size_t)dev_info().sm_count * 8);
  gather_u_kernel<<<grid, 256, 0, s>>>(src, lds, pp, perm, sigma, use_sigma, rho, X, ldx, mrows,
                                       Ub, ldub);
  return cudaGetLastError();
}

// ---- moments ----------------------------------------------------------------------------
// vals layout: [0] Phi(0); [1+2k] Phi(+e_k), [2+2k] Phi(-e_k); then for each
// pair j < k (row-major order) four values Phi(+j+k), Phi(+j-k), Phi(-j+k),
// Phi(-j-k).
__global__ void moments_combine_kernel(const cplx* vals, int d, double da, double* mean,
                                       double* cov, double* imag_resid) {
  __shared__ double mshared[256];
  __shared__ double ires[256];
  const int t = threadIdx.x;
  double ir = 0.0;
  for (int k = t; k < d; k += blockDim.x) {
    const cplx p = vals[1 + 2 * k], m = vals[2 + 2 * k];
    // -i (p - m) / (2 da)
    const cplx dlt = csub(p, m);
    const double re = dlt.y / (2 * da), im = -dlt.x / (2 * da);
    mean[k] = re;
    mshared[k] = re;
    ir = fmax(ir, fabs(im));
  }
  __syncthreads();
  for (int e = t; e < d * d; e += blockDim.x) {
    const int j = e % d, k = e / d;
    cplx v;
    if (j == k) {
      const cplx p = vals[1 + 2 * k], m = vals[2 + 2 * k], z = vals[0];
      const cplx s2 = cadd(csub(p, cscale(z, 2.0)), m);
      v = cscale(s2, -1.0 / (da * da));
    } else {
      const int a = min(j, k), b = max(j, k);
      // pair index of (a, b), a < b, in row-major order over a
      const int pidx = a * d - a * (a + 1) / 2 + (b - a - 1);
      const cplx* f = vals + 1 + 2 * d + 4 * pidx;
      // f: (+a+b), (+a-b), (-a+b), (-a-b); symmetric in (j, k)
      const cplx s4 = csub(csub(f[0], f[1]), csub(f[2], f[3]));
      v = cscale(s4, -1.0 / (4 * da * da));
    }
    cov[e] = v.x - mshared[j] * mshared[k];
    ir = fmax(ir, fabs(v.y));
  }
  ires[t] = ir;
  __syncthreads();
  if (t == 0) {
    double mx = 0.0;
    for (int u = 0; u < blockDim.x; ++u) mx = fmax(mx, ires[u]);
    if (imag_resid) *imag_resid = mx;
  }
}

cudaError_t moments_combine(const cplx* vals, int d, double da, double* mean, double* cov,
                            double* imag_resid, cudaStream_t s) {
  if (d > 256) return cudaErrorInvalidValue;
  moments_combine_kernel<<<1, 256, 0, s>>>(vals, d, da, mean, cov, imag_resid);
  return cudaGetLastError();
}

// ---- dense helpers -------------------------------------------------------------------------
__global__ void conj_transpose_kernel(const cplx* __restrict__ A, int lda, int k, int m,
                                      cplx* __restrict__ B, int ldb) {
  // A is k x m; B (m x k) = A^H.  32 x 32 tiles through shared memory.
  __shared__ cplx tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;  // bx over m, by over k
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int col = bx + yy;        // column of A (index in m)
    const int row = by + threadIdx.x;  // row of A (index in k)
    if (row < k && col < m) tile[yy][threadIdx.x] = A[row + (size_t)lda * col];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int row = bx + threadIdx.x;  // row of B (index in m)
    const int col = by + yy;           // column of B (index in k)
    if (row < m && col < k) B[row + (size_t)ldb * col] = cconj(tile[threadIdx.x][yy]);
  }
}

cudaError_t conj_transpose(const cplx* A, int lda, int k, int m, cplx* B, int ldb,
                           cudaStream_t s) {
  if (k <= 0 || m <= 0) return cudaSuccess;
  dim3 grid((m + 31) / 32, (k + 31) / 32);
  conj_transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(A, lda, k, m, B, ldb);
  return cudaGetLastError();
}

__global__ void frob2_kernel(const cplx* A, int lda, int m, int k, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  const size_t total = (size_t)m * k;
  for (size_t e = threadIdx.x; e < total; e += blockDim.x) {
    const size_t i = e % m, j = e / m;
    acc += cabs2(A[i + (size_t)lda * j]);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *out = acc;
}

cudaError_t frob2(const cplx* A, int lda, int m, int k, double* out, cudaStream_t s) {
  frob2_kernel<<<1, 1024, 0, s>>>(A, lda, m, k, out);
  return cudaGetLastError();
}

cudaError_t fill_zero(cplx* A, size_t count, cudaStream_t s) {
  return cudaMemsetAsync(A, 0, count * sizeof(cplx), s);
}

__global__ void extract_r_kernel(const cplx* A, int lda, int p, int k, cplx* R, int ldr) {
  const size_t total = (size_t)p * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % p), j = (int)(e / p);
    R[i + (size_t)ldr * j] = (i <= j) ? A[i + (size_t)lda * j] : mk(0, 0);
  }
}

cudaError_t extract_r(const cplx* A, int lda, int p, int k, cplx* R, int ldr, cudaStream_t s) {
  const size_t total = (size_t)p * k;
  extract_r_kernel<<<std::max(1, std::min(nblk(total, 256), 1024)), 256, 0, s>>>(A, lda, p, k, R, ldr);
  return cudaGetLastError();
}

__global__ void check_finite_kernel(const cplx* x, size_t count, int* flag) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const cplx v = x[e];
    if (!isfinite(v.x) || !isfinite(v.y)) *flag = 1;
  }
}

cudaError_t check_finite(const cplx* x, size_t count, int* flag, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int grid = std::min<size_t>(nblk(count, 256), (size_t)dev_info().sm_count * 8);
  check_finite_kernel<<<grid, 256, 0, s>>>(x, count, flag);
  return cudaGetLastError();
}

// ---- FP64 complex GEMM (64 x 64 tiles, 4 x 4 outputs per thread) -------------------------
constexpr int GT = 64, GK = 16;

struct LoadA_N {  // A(i, t) = A[i + lda t]
  const cplx* A;
  int lda, M, K;
  __device__ cplx operator()(int i, int t) const {
    return (i < M && t < K) ? A[i + (size_t)lda * t] : mk(0, 0);
  }
};
struct LoadB_RH {  // B(t, j) = conj(R[j + ldr (coff + t)]) for j <= coff + t
  const cplx* R;    // (R upper trapezoidal; coff selects a block of columns)
  int ldr, K, N, coff;
  __device__ cplx operator()(int t, int j) const {
    return (t < K && j < N && j <= coff + t) ? cconj(R[j + (size_t)ldr * (coff + t)]) : mk(0, 0);
  }
};
struct LoadA_UH {  // A(i, t) = conj(U[t + ldu i])
  const cplx* U;
  int ldu, M, K;
  __device__ cplx operator()(int i, int t) const {
    return (i < M && t < K) ? cconj(U[t + (size_t)ldu * i]) : mk(0, 0);
  }
};
struct LoadB_N {  // B(t, j) = B[t + ldb j]
  const cplx* B;
  int ldb, K, N;
  __device__ cplx operator()(int t, int j) const {
    return (t < K && j < N) ? B[t + (size_t)ldb * j] : mk(0, 0);
  }
};
struct StoreC {  // mode 0: C[i + ldc j]; mode 1: conj into the H^H layout
  cplx* C;
  int ldc, M, N, mode, rl, n;
  __device__ void operator()(int i, int j, cplx v) const {
    if (i >= M || j >= N) return;
    if (mode == 0) {
      C[i + (size_t)ldc * j] = v;
    } else {
      const int ii = i % rl, mm = i / rl;
      C[(size_t)(mm + (size_t)n * j) + (size_t)ldc * ii] = cconj(v);
    }
  }
};

template <class LA, class LB, class ST>
__global__ void __launch_bounds__(256) gemm_kernel(LA la, LB lb, ST st, int M, int N, int K) {
  __shared__ cplx As[GK][GT + 1];
  __shared__ cplx Bs[GK][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  cplx acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = mk(0, 0);
  for (int t0 = 0; t0 < K; t0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      const int r = e % GT, kk = e / GT;
      As[kk][r] = la(i0 + r, t0 + kk);
      const int kk2 = e % GK, cc = e / GK;
      Bs[kk2][cc] = lb(t0 + kk2, j0 + cc);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      cplx av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = cfma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) st(i0 + tx + 16 * a, j0 + ty + 16 * b, acc[a][b]);
}

// Mixed-precision variant: operands split into double-float (hi, lo) when
// staged, products and sums in double-float arithmetic on the FP32 pipe,
// result stored in FP64.
template <class LA, class LB, class ST>
__global__ void __launch_bounds__(256) gemm_kernel_f(LA la, LB lb, ST st, int M, int N, int K) {
  __shared__ df2 As[GK][GT + 1];
  __shared__ df2 Bs[GK][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  df2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = df_zero();
  for (int t0 = 0; t0 < K; t0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      const int r = e % GT, kk = e / GT;
      As[kk][r] = df_from(la(i0 + r, t0 + kk));
      const int kk2 = e % GK, cc = e / GK;
      Bs[kk2][cc] = df_from(lb(t0 + kk2, j0 + cc));
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      df2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) df_cmac(acc[a][b], av[a], bv[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) st(i0 + tx + 16 * a, j0 + ty + 16 * b, df_to(acc[a][b]));
}

cudaError_t gemm_a_rh(const cplx* A, int lda, int M, int K, const cplx* R, int ldr, int N,
                      cplx* C, int ldc, int mode, int rl, int n, cudaStream_t s, int mixed) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((M + GT - 1) / GT, (N + GT - 1) / GT);
  if (mixed)
    gemm_kernel_f<<<grid, 256, 0, s>>>(LoadA_N{A, lda, M, K}, LoadB_RH{R, ldr, K, N, 0},
                                       StoreC{C, ldc, M, N, mode, rl, n}, M, N, K);
  else
    gemm_kernel<<<grid, 256, 0, s>>>(LoadA_N{A, lda, M, K}, LoadB_RH{R, ldr, K, N, 0},
                                     StoreC{C, ldc, M, N, mode, rl, n}, M, N, K);
  return cudaGetLastError();
}

cudaError_t gemm_a_rblk_h(const cplx* A, int lda, int M, int K, const cplx* R, int ldr, int coff,
                          int N, cplx* C, int ldc, cudaStream_t s, int mixed) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((M + GT - 1) / GT, (N + GT - 1) / GT);
  if (mixed)
    gemm_kernel_f<<<grid, 256, 0, s>>>(LoadA_N{A, lda, M, K}, LoadB_RH{R, ldr, K, N, coff},
                                       StoreC{C, ldc, M, N, 0, 1, 1}, M, N, K);
  else
    gemm_kernel<<<grid, 256, 0, s>>>(LoadA_N{A, lda, M, K}, LoadB_RH{R, ldr, K, N, coff},
                                     StoreC{C, ldc, M, N, 0, 1, 1}, M, N, K);
  return cudaGetLastError();
}

// out(alpha, i, m, q) = sum_beta W[alpha, beta] applied along m to
// T_beta[i, :, q] (T_beta: r x n x p, consecutive blocks of r n p).  Written
// in the V layout (mode 0: out[(alpha r + i) + Al r m + Al r n q]) or
// conj-transposed into the H^H layout of the next QR (mode 1:
// out[(m + n q) + ldo (alpha r + i)] = conj(value)).
__global__ void stencil_combine_kernel(const cplx* __restrict__ T, int r, int n, int p, int Bn,
                                       int Al, int Ar, const unsigned char* __restrict__ blocks,
                                       const cplx* __restrict__ coef, cplx* __restrict__ out,
                                       int mode, int ldo) {
  // grid y walks q, x the (alpha, i, m) plane: 32-bit index arithmetic
  const int rows = Al * r;
  const int plane = rows * n;
  const size_t blk = (size_t)r * n * p;
  for (int q = blockIdx.y; q < p; q += gridDim.y) {
    const cplx* Tq = T + (size_t)r * n * q;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < plane; idx += gridDim.x * blockDim.x) {
      const int m = idx / rows, pr = idx - m * rows;
      const int al = pr / r, i = pr - al * r;
      cplx v = mk(0, 0);
      for (int be = 0; be < Bn; ++be) {
        const int op = blocks[al * Ar + be];
        if (op == OP_NONE) continue;
        v = cadd(v, op_apply(coef, op, n, Tq + blk * be + i, (size_t)r, m));  // T_beta[i, :, q]
      }
      if (mode == 0) out[(size_t)idx + (size_t)plane * q] = v;
      else out[(size_t)(m + (size_t)n * q) + (size_t)ldo * pr] = cconj(v);
    }
  }
}

// Tiled form of the same sum for the conj-transposed layout (mode 1) and
// three-point operators.  One CTA per (q, 32 left-rank indices i, 16 grid
// points m): the T_beta[i, m - 1 .. m + 16, q] rows of every beta are staged
// in shared memory by cp.async (zero beyond the grid's edges), each thread
// forms all Al outputs of one (i, m) from the three taps of every beta with
// only the coefficient parts that are nonzero (the identity is an addition,
// a real diagonal two multiply-adds), and a warp writes 16 consecutive m of
// two output rows: 256-byte segments of the H^H layout.
constexpr int kStTM = 16;
constexpr int kStTI = 32;
constexpr int kStThreads = 256;
constexpr int kStLd = kStTI + 1;  // odd row stride: conflict-free reads along m

size_t stencil_tile_smem(int Bn) { return (size_t)Bn * (kStTM + 2) * kStLd * sizeof(cplx); }

DV void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

// acc += (op x)[m] from the taps xl = x[m-1], x0 = x[m], xu = x[m+1]
// (zero beyond the edges), using the parts of the coefficients that f marks.
DV void op_acc(const cplx* __restrict__ cf, int n, int m, unsigned f, const cplx& xl, const cplx& x0,
               const cplx& xu, cplx& acc) {
  if (f & 0x40) {
    acc.x += x0.x;
    acc.y += x0.y;
    return;
  }
  if (f & 0x03) {
    const cplx c = cf[m];
    if (f & 0x01) { acc.x = fma(c.x, xl.x, acc.x); acc.y = fma(c.x, xl.y, acc.y); }
    if (f & 0x02) { acc.x = fma(-c.y, xl.y, acc.x); acc.y = fma(c.y, xl.x, acc.y); }
  }
  if (f & 0x0C) {
    const cplx c = cf[n + m];
    if (f & 0x04) { acc.x = fma(c.x, x0.x, acc.x); acc.y = fma(c.x, x0.y, acc.y); }
    if (f & 0x08) { acc.x = fma(-c.y, x0.y, acc.x); acc.y = fma(c.y, x0.x, acc.y); }
  }
  if (f & 0x30) {
    const cplx c = cf[2 * n + m];
    if (f & 0x10) { acc.x = fma(c.x, xu.x, acc.x); acc.y = fma(c.x, xu.y, acc.y); }
    if (f & 0x20) { acc.x = fma(-c.y, xu.y, acc.x); acc.y = fma(c.y, xu.x, acc.y); }
  }
}

__global__ void __launch_bounds__(kStThreads, 3)
    stencil_tile_kernel(const cplx* __restrict__ T, int r, int n, int p, int Bn, int Al, int Ar,
                        const unsigned char* __restrict__ blocks, const cplx* __restrict__ coef,
                        unsigned long long forms, cplx* __restrict__ out, int ldo) {
  extern __shared__ cplx xs[];  // [Bn][kStTM + 2][kStLd]: T_beta[i0 + i, m0 - 1 + mm, q]
  __shared__ unsigned char blk[36];
  constexpr int rows = kStTM + 2;
  const int mt = (n + kStTM - 1) / kStTM, it = (r + kStTI - 1) / kStTI;
  int b = blockIdx.x;
  const int m0 = (b % mt) * kStTM;
  b /= mt;
  const int i0 = (b % it) * kStTI;
  const int q = b / it;
  const int ti = min(kStTI, r - i0);
  const size_t bstride = (size_t)r * n * p;
  if (threadIdx.x < Al * Ar) blk[threadIdx.x] = blocks[threadIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int row = w; row < Bn * rows; row += kStThreads / 32) {
    const int be = row / rows, mm = row - be * rows;
    const int m = m0 - 1 + mm;
    if (lane < ti) {
      cplx* dst = xs + row * kStLd + lane;
      if (m >= 0 && m < n) cp_async16(dst, T + bstride * be + (size_t)(i0 + lane) + (size_t)r * ((size_t)m + (size_t)n * q));
      else *dst = mk(0, 0);
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int mi = lane & 15, m = m0 + mi;
  if (m >= n) return;
  const size_t col = (size_t)m + (size_t)n * q;
  for (int i = 2 * w + (lane >> 4); i < ti; i += kStThreads / 16) {
    cplx acc[6];
#pragma unroll
    for (int al = 0; al < 6; ++al) acc[al] = mk(0, 0);
    for (int be = 0; be < Bn; ++be) {
      const cplx* x = xs + (be * rows + mi) * kStLd + i;  // row mi holds m - 1
      const cplx xl = x[0], x0 = x[kStLd], xu = x[2 * kStLd];
#pragma unroll
      for (int al = 0; al < 6; ++al) {
        if (al < Al) {
          const int op = blk[al * Ar + be];
          if (op != OP_NONE)
            op_acc(coef + (size_t)op * 3 * n, n, m, (unsigned)(forms >> (8 * op)) & 0xFFu, xl, x0, xu, acc[al]);
        }
      }
    }
#pragma unroll
    for (int al = 0; al < 6; ++al)
      if (al < Al) out[col + (size_t)ldo * (size_t)(al * r + i0 + i)] = cconj(acc[al]);
  }
}

cudaError_t stencil_combine(const cplx* T, int r, int n, int p, int Bn, int Al, int Ar,
                            const unsigned char* blocks_dev, const OpTable& ops, cplx* out,
                            int mode, int ldo, cudaStream_t s) {
  const size_t total = (size_t)Al * r * n * p;
  if (total == 0) return cudaSuccess;
  if (mode == 1 && (ops.forms >> 63) && Bn <= 6 && Al <= 6 && Al * Ar <= 36) {
    const size_t smem = stencil_tile_smem(Bn);
    cudaError_t e = allow_smem((const void*)stencil_tile_kernel, smem);
    if (e != cudaSuccess) return e;
    const size_t tiles = (size_t)((n + kStTM - 1) / kStTM) * ((r + kStTI - 1) / kStTI) * p;
    stencil_tile_kernel<<<(unsigned)tiles, kStThreads, smem, s>>>(T, r, n, p, Bn, Al, Ar, blocks_dev, ops.coef,
                                                                   ops.forms, out, ldo);
    return cudaGetLastError();
  }
  const size_t plane = (size_t)Al * r * n;
  if (plane >= (1u << 31)) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)std::min<size_t>(nblk(plane, 256), 1024), (unsigned)std::min(p, 65535));
  stencil_combine_kernel<<<grid, 256, 0, s>>>(T, r, n, p, Bn, Al, Ar, blocks_dev, ops.coef, out,
                                              mode, ldo);
  return cudaGetLastError();
}

cudaError_t gemm_uh_r(const cplx* U, int ldu, int M, int K, const cplx* R, int ldr, int N,
                      cplx* C, int ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((M + GT - 1) / GT, (N + GT - 1) / GT);
  gemm_kernel<<<grid, 256, 0, s>>>(LoadA_UH{U, ldu, M, K}, LoadB_N{R, ldr, K, N},
                                   StoreC{C, ldc, M, N, 0, 1, 1}, M, N, K);
  return cudaGetLastError();
}

// ---- watchdog check -----------------------------------------------------------
__global__ void watchdog_kernel(GridBar* bar) {
  if (blockIdx.x == 0) return;  // never arrives: the others' wait must expire
  GridSync gs{bar, 0u};
  grid_sync(gs);
}

cudaError_t watchdog_probe(const CoopWs& ws, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&ws.bar->count, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  GridBar* bar = ws.bar;
  void* args[] = {&bar};
  return cudaLaunchCooperativeKernel((void*)watchdog_kernel, dim3(2), dim3(32), args, 0, s);
}

}  // namespace hk
