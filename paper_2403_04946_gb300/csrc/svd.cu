// Small dense SVD for the truncation step, and the rank rule.
//
// After the QR of a core's vertical flattening, the truncated SVD is taken of
// the small triangular factor R (App. A: "R has the same singular values as
// A", the QR-then-SVD structure of Alg. 4).  The SVD here is the one-sided
// Jacobi method (Hestenes 1958; accuracy analysis Demmel & Veselic 1992),
// written for this library: columns are orthogonalised pairwise by complex
// plane rotations in round-robin order (each round is a perfect matching of
// the columns, so one round's rotations are independent and run on all SMs),
// sweeps repeat until no pair is rotated.  A pair is left alone once its
// columns are orthogonal to 2 nr eps (above the rounding floor of their
// computed inner product) or once its smaller column is negligible for the
// truncation (see theta below).  The CTAs meet at a bounded grid barrier
// between rounds.
#include <algorithm>
#include <cfloat>

#include "kernels.h"

namespace hk {

constexpr int kJacThreads = 256;

__device__ __forceinline__ void pair_of(int r, int q, int N, int* a, int* b) {
  // circle method: player N-1 fixed, others rotate
  if (q == 0) {
    *a = r;
    *b = N - 1;
  } else {
    *a = (r + q) % (N - 1);
    *b = (r - q + N - 1) % (N - 1);
  }
}

// One pair of columns per group of kGroup threads (two groups per CTA); each
// thread keeps its rows of both columns in registers, so a pair costs one
// round trip to L2 for the loads, one group reduction and one store.
constexpr int kGroup = 128;

template <int RPT>
__global__ void __launch_bounds__(kJacThreads, 1)
jacobi_kernel(cplx* M, int ldm, int nr, int nc, cplx* J, int ldj, int accumJ, double tol,
              int max_sweeps, const double* eps_hat, CoopWs ws) {
  __shared__ double red[2][4][2];  // [group][warp][ga.x, ga.y]
  const int G = gridDim.x, g = blockIdx.x;
  const int grp = threadIdx.x / kGroup, gt = threadIdx.x % kGroup;
  const int lane = gt & 31, gw = gt >> 5;
  const int wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int N = nc + (nc & 1);
  const int npairs = N / 2;
  GridSync gs{ws.bar, 0u};
  double* colnorm = ws.colnorm;
  unsigned int* colver = ws.colver;
  unsigned long long* pairchk = ws.pairchk;

  // exact squared column norms (also re-done at the start of every sweep),
  // column versions zeroed, no pair marked orthogonal yet
  auto column_norms = [&]() {
    for (int c = g * nwarp + wid; c < nc; c += G * nwarp) {
      const cplx* a = M + (size_t)ldm * c;
      double s = 0.0;
      for (int row = lane; row < nr; row += 32) s += cabs2(__ldcg(a + row));
      s = warp_sum(s);
      if (lane == 0) colnorm[c] = s;
    }
  };
  column_norms();
  for (int c = g * blockDim.x + threadIdx.x; c < nc; c += G * blockDim.x) colver[c] = 0u;
  for (size_t e = (size_t)g * blockDim.x + threadIdx.x; e < (size_t)nc * nc; e += (size_t)G * blockDim.x)
    pairchk[e] = ~0ull;
  grid_sync(gs);
  if (grid_failed(ws.bar)) return;
  double fro2 = 0.0;
  for (int c = 0; c < nc; ++c) fro2 += __ldcg(colnorm + c);
  // A pair is left alone once its smaller column is below theta: a column of
  // norm theta moves any other column (hence any kept singular vector) by at
  // most theta, and the discarded tail is the Frobenius norm of the columns
  // left over, which rotations do not change.  theta = max(1e-3 eps_hat,
  // 64 eps ||M||_F): far below the truncation error committed at this bond,
  // and at the rounding floor of the QR that produced M.
  // eps_hat == NULL asks for the exact method (no pair left out).
  const double eh = eps_hat ? __ldcg(eps_hat) : 0.0;
  const double floor_abs = 64.0 * DBL_EPSILON * sqrt(fro2);
  const double theta = eps_hat ? fmax(1e-3 * eh, floor_abs) : 0.0;
  const double negl2 = theta * theta;

  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps; ++sweep) {
    if (sweep > 0) {
      // the rotations below update the norms incrementally; start each sweep
      // from exact ones, so the final (rotation-free) sweep tests exactly
      column_norms();
      grid_sync(gs);
      if (grid_failed(ws.bar)) return;
    }
    for (int r = 0; r < N - 1; ++r) {
      for (int base = 2 * g; base < npairs; base += 2 * G) {
        const int q = base + grp;
        int i = 0, j = 0;
        bool active = q < npairs;
        unsigned long long key = 0ull;
        if (active) {
          pair_of(r, q, N, &i, &j);
          active = (i < nc && j < nc);
          if (i > j) {
            const int t = i;
            i = j;
            j = t;
          }
        }
        double al = 0.0, be = 0.0;
        if (active) {
          // skip the pair if neither column changed since it was last found
          // orthogonal (no column loads at all)
          key = ((unsigned long long)__ldcg(colver + i) << 32) | __ldcg(colver + j);
          if (__ldcg(pairchk + (size_t)i * nc + j) == key) active = false;
          // read before the group's barriers: thread 0 rewrites them below
          al = __ldcg(colnorm + i);
          be = __ldcg(colnorm + j);
        }
        cplx x[RPT], y[RPT];
        cplx ga = mk(0, 0);
        if (active) {
          const cplx* ai = M + (size_t)ldm * i;
          const cplx* aj = M + (size_t)ldm * j;
#pragma unroll
          for (int u = 0; u < RPT; ++u) {
            const int row = gt + u * kGroup;
            x[u] = (row < nr) ? __ldcg(ai + row) : mk(0, 0);
            y[u] = (row < nr) ? __ldcg(aj + row) : mk(0, 0);
          }
#pragma unroll
          for (int u = 0; u < RPT; ++u) ga = cfmac(x[u], y[u], ga);
        }
        ga = warp_sum(ga);
        if (lane == 0) {
          red[grp][gw][0] = ga.x;
          red[grp][gw][1] = ga.y;
        }
        __syncthreads();
        ga = mk(0, 0);
#pragma unroll
        for (int w = 0; w < kGroup / 32; ++w) {
          ga.x += red[grp][w][0];
          ga.y += red[grp][w][1];
        }
        __syncthreads();
        if (!active) continue;
        const double gabs = sqrt(cabs2(ga));
        const bool rot = gabs > 0.0 && gabs > tol * sqrt(al) * sqrt(be) && fmin(al, be) > negl2;
        if (rot) {
          const double zeta = (be - al) / (2.0 * gabs);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t);
          const double s = c * t;
          const cplx em = mk(ga.x / gabs, -ga.y / gabs);  // e^{-i phi}, e^{i phi} = ga/|ga|
          cplx* ai = M + (size_t)ldm * i;
          cplx* aj = M + (size_t)ldm * j;
#pragma unroll
          for (int u = 0; u < RPT; ++u) {
            const int row = gt + u * kGroup;
            if (row < nr) {
              const cplx xv = x[u];
              const cplx yv = cmul(y[u], em);
              ai[row] = mk(c * xv.x - s * yv.x, c * xv.y - s * yv.y);
              aj[row] = mk(s * xv.x + c * yv.x, s * xv.y + c * yv.y);
            }
          }
          if (accumJ) {
            cplx* ji = J + (size_t)ldj * i;
            cplx* jj = J + (size_t)ldj * j;
            for (int row = gt; row < nc; row += kGroup) {
              const cplx xv = __ldcg(ji + row);
              const cplx yv = cmul(__ldcg(jj + row), em);
              ji[row] = mk(c * xv.x - s * yv.x, c * xv.y - s * yv.y);
              jj[row] = mk(s * xv.x + c * yv.x, s * xv.y + c * yv.y);
            }
          }
          if (gt == 0) {
            // norms of the rotated pair (exact in exact arithmetic)
            colnorm[i] = fmax(al - t * gabs, 0.0);
            colnorm[j] = be + t * gabs;
            colver[i] += 1u;
            colver[j] += 1u;
            atomicAdd(ws.counters + (sweep & 31), 1);
          }
        } else if (gt == 0) {
          pairchk[(size_t)i * nc + j] = key;
        }
      }
      grid_sync(gs);
      if (grid_failed(ws.bar)) return;
    }
    // every CTA sees the same count after the last round's barrier
    const int rotations = __ldcg(ws.counters + (sweep & 31));
    if (rotations == 0) {
      converged = true;
      break;
    }
    // reset the counter two sweeps ahead (no CTA touches it before another
    // full round of barriers)
    if (g == 0 && threadIdx.x == 0) atomicExch(ws.counters + ((sweep + 2) & 31), 0);
  }
  if (g == 0 && threadIdx.x == 0) ws.counters[63] = converged ? sweep + 1 : -(sweep + 1);
}

__global__ void init_identity_kernel(cplx* J, int ldj, int nc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nc * nc) {
    const int r = i % nc, c = i / nc;
    J[r + (size_t)ldj * c] = mk(r == c ? 1.0 : 0.0, 0.0);
  }
}

cudaError_t jacobi_svd(cplx* M, int ldm, int nr, int nc, cplx* J, int ldj, int accumJ,
                       const double* eps_hat, int init_j, const CoopWs& ws, cudaStream_t s) {
  if (nc <= 0 || nr <= 0) return cudaSuccess;
  if (nc > ws.jac_cap) return cudaErrorInvalidValue;
  if (accumJ && init_j) {
    init_identity_kernel<<<(nc * nc + 255) / 256, 256, 0, s>>>(J, ldj, nc);
  }
  cudaError_t e = cudaMemsetAsync(ws.counters, 0, 32 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&ws.bar->count, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const DevInfo& di = dev_info();
  const int npairs = (nc + 1) / 2;
  // two pairs per CTA, as many CTAs as SMs allow
  const int G = std::max(1, std::min(coop_sms(ws), (npairs + 1) / 2));
  // Stop rotating a pair once |a_i^H a_j| <= tol |a_i| |a_j|.  The computed
  // inner product of two length-nr columns carries a rounding error of up
  // to about nr * eps relative to |a_i| |a_j|, so a threshold below that
  // floor can keep re-rotating noise forever (seen on factors whose singular
  // values span 16 decades); 2 nr eps sits above it.
  double tol = 2.0 * DBL_EPSILON * (double)nr;
  int max_sweeps = 80;
  CoopWs w = ws;
  void* args[] = {&M, &ldm, &nr, &nc, &J, &ldj, &accumJ, &tol, &max_sweeps, (void*)&eps_hat, &w};
  void* fn;
  if (nr <= 2 * kGroup) fn = (void*)jacobi_kernel<2>;
  else if (nr <= 4 * kGroup) fn = (void*)jacobi_kernel<4>;
  else if (nr <= 8 * kGroup) fn = (void*)jacobi_kernel<8>;
  else if (nr <= 16 * kGroup) fn = (void*)jacobi_kernel<16>;
  else return cudaErrorInvalidValue;  // columns longer than 2048
  return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kJacThreads), args, 0, s);
}

// ---- rank selection ---------------------------------------------------------

__global__ void rank_select_kernel(const cplx* M, int ldm, int nr, int nc,
                                   const double* eps_hat, int cap, int forced, double* sigma,
                                   int* perm, int* out_int, double* out_dbl, double* tail2) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < nc; c += nw) {
    double s = 0.0;
    for (int row = lane; row < nr; row += 32) s += cabs2(M[row + (size_t)ldm * c]);
    s = warp_sum(s);
    if (lane == 0) sigma[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const double sc = sigma[c];
    int rank = 0;
    for (int o = 0; o < nc; ++o) {
      const double so = sigma[o];
      rank += (so > sc) || (so == sc && o < c);
    }
    perm[rank] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // tail2[r] = sum_{i >= r} sigma_sorted[i]^2, accumulated from the smallest
    tail2[nc] = 0.0;
    for (int r = nc - 1; r >= 0; --r) {
      const double sv = sigma[perm[r]];
      tail2[r] = tail2[r + 1] + sv * sv;
    }
    const double eh = *eps_hat;
    int rho_tol = nc;
    for (int r = 1; r <= nc; ++r)
      if (sqrt(tail2[r]) <= eh) {
        rho_tol = r;
        break;
      }
    int rho = forced > 0 ? forced : (rho_tol < cap ? rho_tol : cap);
    if (rho < 1) rho = 1;
    if (rho > nc) rho = nc;
    out_int[0] = rho;
    out_int[1] = rho_tol;
    out_dbl[0] = sqrt(tail2[rho]);
    out_dbl[1] = sigma[perm[rho - 1]];  // smallest kept singular value
    out_dbl[2] = tail2[0];              // ||M||_F^2
  }
}

cudaError_t rank_select(const cplx* M, int ldm, int nr, int nc, const double* eps_hat, int cap,
                        int forced, double* sigma, int* perm, int* out_int, double* out_dbl,
                        cudaStream_t s) {
  // tail2 lives after sigma (caller sizes sigma for 2 * nc + 1 doubles)
  rank_select_kernel<<<1, 256, 0, s>>>(M, ldm, nr, nc, eps_hat, cap, forced, sigma, perm,
                                       out_int, out_dbl, sigma + nc);
  return cudaGetLastError();
}

}  // namespace hk
