// Internal interface between the C-ABI layer (hopf.cu) and the kernel
// translation units.  Every launcher enqueues work on `s` and returns the
// launch's cudaError_t; none synchronises.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace hk {

// ---- device properties ------------------------------------------------------
struct DevInfo {
  int sm_count;
  int max_smem_optin;
};
const DevInfo& dev_info();

// ---- workspaces for the cooperative QR / ormqr / SVD kernels ---------------
struct CoopWs {
  GridBar* bar;     // 1 barrier (zeroed)
  double* pr;       // [max_grid] real partials
  cplx* pc;         // complex partials, pc_elems
  size_t pc_elems;
  cplx* wfin;       // reduced values, wfin_elems
  size_t wfin_elems;
  cplx* scal;       // [8] scalars
  int* counters;    // [64] sweep counters
  // one-sided Jacobi state: squared column norms, column versions, and the
  // versions at which each pair was last found orthogonal (jac_cap columns)
  double* colnorm;
  unsigned int* colver;
  unsigned long long* pairchk;
  int jac_cap;
  // upper bound on the CTAs (one per SM) of every cooperative launch that
  // uses this workspace; 0 = all SMs.  Contexts limited to disjoint shares
  // of the SMs run their cooperative kernels concurrently.
  int max_ctas;
};
// SMs available to a cooperative launch on this workspace.
int coop_sms(const CoopWs& ws);
// Raises the kernel's dynamic shared-memory limit to the device maximum
// (opt-in size minus its static shared memory) once per function and
// checks that `need` bytes fit.  The attribute is process-wide, so it is
// never lowered: contexts on several host threads launch concurrently.
cudaError_t allow_smem(const void* fn, size_t need);

// Householder QR of the column-major m x k matrix A (lda >= m), in place:
// R on and above the diagonal, reflector tails below, tau[min(m,k)], and for
// every panel of width `nb` its reflectors' Gram matrix v_u^H v_s (strict
// upper triangle) with tau on the diagonal, in T (npanel x nb x nb); ormqr
// applies the panel from these.  Returns the panel width used through
// *nb_out.  mixed != 0: the matrix is held in double-float form (scaled by a
// power of two) during the factorisation, the Householder scalars in FP64.
cudaError_t geqrf(cplx* A, int lda, int m, int k, cplx* tau, cplx* T, int* nb_out,
                  const CoopWs& ws, cudaStream_t s, int mixed = 0);
// C <- Q C with Q = H_0 H_1 ... H_{p-1} from geqrf (A, lda, m, p, tau, T, nb);
// C is m x q column-major (ldc).
cudaError_t ormqr(const cplx* A, int lda, int m, int p, const cplx* tau, const cplx* T,
                  int nb, cplx* C, int ldc, int q, const CoopWs& ws, cudaStream_t s, int mixed = 0);

// One-sided Jacobi SVD of the nr x nc column-major matrix M (ldm), in place:
// on exit the columns of M are U_i * sigma_i (any order); if accumJ, J
// (nc x nc, ldj) accumulates the rotations (set to the identity first if
// init_j).  eps_hat (device scalar) is the truncation tolerance of this
// bond: pairs whose smaller column is below max(1e-3 eps_hat,
// 64 eps ||M||_F) are not rotated; eps_hat == NULL rotates every pair (the
// exact method, also usable to finish a run started with eps_hat).  Writes
// the number of sweeps to ws.counters[63] (negative if not converged).
cudaError_t jacobi_svd(cplx* M, int ldm, int nr, int nc, cplx* J, int ldj, int accumJ,
                       const double* eps_hat, int init_j, const CoopWs& ws, cudaStream_t s);

// Column norms of M -> sigma, sort descending (ties: lower index first),
// choose the rank (tolerance rule or forced) and the discarded tail.
// out_int[0] = rho, out_int[1] = rho by tolerance (before the cap);
// out_dbl[0] = discarded tail at rho, out_dbl[1] = smallest kept sigma,
// out_dbl[2] = ||M||_F^2.  perm[nc] = sorted order.
cudaError_t rank_select(const cplx* M, int ldm, int nr, int nc, const double* eps_hat,
                        int cap, int forced, double* sigma, int* perm, int* out_int,
                        double* out_dbl, cudaStream_t s);

// ---- SVD of a square factor through bidiagonalisation (bdsvd.cu) --------
// R (n x n, lda) = Q B P^H in place (LAPACK zgebrd layout: left reflector
// tails below the diagonal, right reflector tails right of the
// superdiagonal); B: diagonal d[n], superdiagonal e[n-1], both real.
// Cooperative launch, one grid barrier per column.
cudaError_t gebrd(cplx* A, int lda, int n, double* d, double* e, cplx* tauq, cplx* taup,
                  const CoopWs& ws, cudaStream_t s);
bool gebrd_fits(int n, const CoopWs& ws);  // shared-memory resident rows fit
// All singular values of B, sorted descending, into sig[n]; a2 (float2
// [2n]) and info (double [4]) are scratch kept for bd_vectors.
cudaError_t bd_sigma(const double* d, const double* e, int n, float2* a2, double* info, double* sig,
                     cudaStream_t s);
// Rank rule on sorted values: out_int[0] = rho, [1] = rho by tolerance,
// [2] = number of kept values above the noise level 2 n eps ||B||_F;
// out_dbl as rank_select; tail2[n+1] scratch.
cudaError_t bd_rank(const double* sig, int n, const double* eps_hat, int cap, int forced, int* out_int,
                    double* out_dbl, double* tail2, cudaStream_t s);
// Left singular vectors of B: columns k < kt by inverse iteration, columns
// kt..nvec-1 by orthonormal completion; X (n x nvec, ldx), real.
// Zs: nvec x 2n doubles of scratch (the T_GK eigenvectors).
cudaError_t bd_vectors(const double* d, const double* e, int n, const double* info, const double* sig,
                       int kt, int nvec, double* X, int ldx, double* Zs, cudaStream_t s);
// U = Q X -> U (n x nvec, ldu) and Xp (mrows x nvec, ldp, zero below row n).
cudaError_t bd_back(const cplx* A, int lda, const cplx* tauq, int n, const double* X, int ldx, int nvec,
                    cplx* U, int ldu, cplx* Xp, int ldp, int mrows, cudaStream_t s);

// ---- TT-cross construction of a Gaussian (cross.cu) --------------------------
// A (rl n x rr, column-major, row alpha + rl i) = Phi0(Il[alpha], i, Jr[beta])
// with the free index on mode kl; Il rl x kl, Jr rr x (d-kl-1) tuples.
cudaError_t gauss_fibers(const double* agrid, int n, int d, const double* m, const double* C, const int* Il,
                         int rl, int kl, const int* Jr, int rr, cplx* A, cudaStream_t s);
// Complete-pivoting elimination (cooperative): pivot rows[cnt], cols[cnt],
// *count = cnt, stopping at rel_tol of the first pivot; W: M x c scratch.
cudaError_t cross_pivots(const cplx* A, int M, int c, double rel_tol, cplx* W, int* rows, int* cols, int* count,
                         const CoopWs& ws, cudaStream_t s);
// out = A[:, cols] (M x cnt), eye = [I; 0] (M x cnt), seq = 0..cnt-1.
cudaError_t cross_gather(const cplx* A, int M, const int* cols, int cnt, cplx* out, cplx* eye, int* seq,
                         cudaStream_t s);
// core (M x cnt) = A[:, cols] * A[rows, cols]^-1; Gw, Gi: cnt x cnt scratch.
cudaError_t cross_core(const cplx* A, int M, const int* rows, const int* cols, int cnt, cplx* Gw, cplx* Gi,
                       cplx* core, cudaStream_t s);

// ---- dense helpers ------------------------------------------------------------
// B (m x k, ldb) = conj-transpose of the k x m matrix A (lda).
cudaError_t conj_transpose(const cplx* A, int lda, int k, int m, cplx* B, int ldb,
                           cudaStream_t s);
// Frobenius norm^2 of the m x k matrix A -> *out (device).
cudaError_t frob2(const cplx* A, int lda, int m, int k, double* out, cudaStream_t s);
cudaError_t fill_zero(cplx* A, size_t count, cudaStream_t s);
// Upper triangle of the top p x k block of A (lda) -> R (p x k, ldr), zeros below.
cudaError_t extract_r(const cplx* A, int lda, int p, int k, cplx* R, int ldr, cudaStream_t s);

// GEMM variants (FP64 complex, tiles of 64 x 64).
// C[M x N] = A[M x K] * R^H, R upper-trapezoidal N x K (ldr), A column-major (lda).
// mode 0: C column-major (ldc); mode 1: C written conj-transposed into the
// "H^H layout": row index i_all = i + rl * mm (i < rl), column j ->
// B[(mm + n * j) + ldb * i] = conj(C[i_all, j]).
cudaError_t gemm_a_rh(const cplx* A, int lda, int M, int K, const cplx* R, int ldr, int N,
                      cplx* C, int ldc, int mode, int rl, int n, cudaStream_t s, int mixed = 0);
// C[M x N] = A[M x K] * (columns coff..coff+K of R)^H, R upper trapezoidal
// (ldr): C[i, q] = sum_t A[i, t] conj(R[q, coff + t]) over q <= coff + t.
cudaError_t gemm_a_rblk_h(const cplx* A, int lda, int M, int K, const cplx* R, int ldr, int coff,
                          int N, cplx* C, int ldc, cudaStream_t s, int mixed = 0);
// C[M x N] = U[:, perm[0..M)]^H-gathered * R: C[i, j] = sum_t conj(U[t, i]) R[t, j].
cudaError_t gemm_uh_r(const cplx* U, int ldu, int M, int K, const cplx* R, int ldr, int N,
                      cplx* C, int ldc, cudaStream_t s);

// ---- TT-level kernels -------------------------------------------------------------
struct OpTable {
  // Tridiagonal coefficients (lo, di, up) of the per-mode operators
  // I, A, P, Q, Z (index op*3*n + {0,n,2n} + i), complex.
  cplx* coef;
  int n;
};
enum { OP_I = 0, OP_A = 1, OP_P = 2, OP_Q = 3, OP_Z = 4, OP_NONE = 7 };
// Operator blocks applied along the middle index and summed over beta:
// out(alpha, i, m, q) = sum_{beta < Bn} W[alpha*Ar + beta](T_beta[i, :, q])[m].
// mode 0: V layout, mode 1: conj-transposed H^H layout with leading dim ldo.
cudaError_t stencil_combine(const cplx* T, int r, int n, int p, int Bn, int Al, int Ar,
                            const unsigned char* blocks_dev, const OpTable& ops, cplx* out,
                            int mode, int ldo, cudaStream_t s);
// out core (Al*a) x n x (Ar*c) from in core a x n x c; blocks[alpha*Ar+beta]
// holds the op index (OP_NONE = zero block).
cudaError_t apply_core(const cplx* in, int a, int n, int c, cplx* out, int Al, int Ar,
                       const unsigned char* blocks_dev, const OpTable& ops, cudaStream_t s);
// Block concatenation of one core of a TT sum.  kind: 0 first, 1 interior,
// 2 last.  Term t has core pointer ptrs[t], dims (ra[t], n, rc[t]) and
// coefficient coef[t] (applied on the first core only).
struct SumTerm {
  const cplx* p;
  int ra, rc;
  cplx coef;
};
cudaError_t sum_core(const SumTerm* terms_dev, int nterms, int kind, int n, cplx* out,
                     int out_ra, int out_rc, cudaStream_t s);
// Phi at points: idx[npts*d] (device), cores via pointer array (device),
// ranks (device [d+1]).  vals[npts] complex.
cudaError_t eval_points(const cplx* const* cores_dev, const int* ranks_dev, int d, int n,
                        int maxr, int npts, const int* idx_dev, cplx* vals, cudaStream_t s);
// Gaussian set-up kernels.
cudaError_t gauss_rank1_core(const double* agrid, int n, double m, double c, cplx* core,
                             cudaStream_t s);
cudaError_t gauss_full_core(const double* agrid, int n, int d, int c, const double* m0,
                            const double* C0, cplx* core, cudaStream_t s);
cudaError_t identity_core(int n, int a, int b, int left, cplx* core, cudaStream_t s);
// alpha, beta (device [nmodes]), gl (device [2q]: nodes then weights of a
// q-point Gauss-Legendre rule on [0, 1]), m0 (device [d]), C0 (device [d*d]).
cudaError_t cell_moments(int d, int nmodes, const double* alpha, const double* beta,
                         double sigma, double ell, const double* gl, int q, double* m0,
                         double* C0, cudaStream_t s);
// X (mrows x q, ldx) = [S^H; 0] with S q x p (lds).
cudaError_t init_sh_pad(const cplx* S, int lds, int q, int p, cplx* X, int ldx, int mrows,
                        cudaStream_t s);
// Columns l < rho of U: src[:, perm[l]] (scaled by 1/sigma[perm[l]] if
// use_sigma), length pp.  Written to X (mrows x rho, ldx, zero below row pp)
// and to Ub (pp x rho, ldub).
cudaError_t gather_u(const cplx* src, int lds, int pp, const int* perm, const double* sigma,
                     int use_sigma, int rho, cplx* X, int ldx, int mrows, cplx* Ub, int ldub,
                     cudaStream_t s);
// Combine the point values of the moment stencil into mean/cov.
cudaError_t moments_combine(const cplx* vals, int d, double da, double* mean, double* cov,
                            double* imag_resid, cudaStream_t s);
// Any non-finite value in x[count]? sets *flag = 1.
cudaError_t check_finite(const cplx* x, size_t count, int* flag, cudaStream_t s);

}  // namespace hk
