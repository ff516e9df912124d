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
// rows_ws (may be NULL): gebrd_rows_elems(n) elements where the rows go when
// they do not fit in shared memory (L2-resident for the sizes met here).
cudaError_t gebrd(cplx* A, int lda, int n, double* d, double* e, cplx* tauq, cplx* taup,
                  const CoopWs& ws, cudaStream_t s, cplx* rows_ws = nullptr);
bool gebrd_fits(int n, const CoopWs& ws, bool have_rows_ws = false);
size_t gebrd_rows_elems(int n, int sms);
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
  // Coefficients (lo, di, up) of the per-mode operators in slots
  // I, A, P, Q, Z, K (index op*3*n + {0,n,2n} + i), complex (op_apply).
  cplx* coef;
  int n;
  // Per slot (8 bits at 8 * op): which coefficient parts are nonzero
  // anywhere (bits 0-5: lo re, lo im, di re, di im, up re, up im), bit 6 the
  // identity.  Bit 63 set: the table holds only such three-point operators
  // and the tiled apply may use these forms; 0: not computed.
  unsigned long long forms = 0;
};
enum { OP_I = 0, OP_A = 1, OP_P = 2, OP_Q = 3, OP_Z = 4, OP_K = 5, OP_NONE = 7 };
constexpr int kNumOps = 6;  // slots of the coefficient table
// (op x)[m] for the fiber x (stride s): a tridiagonal operator from its
// coefficients (lo, di, up) at coef + op * 3n; OP_K, the CDF equation's
// u - (trapezoidal integral from the lower edge), is di[m] x_m minus
// du (x_0 / 2 + x_1 + ... + x_{m-1} + x_m / 2), du stored in lo[0].
DV cplx op_apply(const cplx* coef, int op, int n, const cplx* x, size_t s, int m) {
  const cplx* cf = coef + (size_t)op * 3 * n;
  cplx v = cmul(cf[n + m], x[s * m]);
  if (op == OP_K) {
    cplx acc = mk(0, 0);
    for (int q = 0; q <= m; ++q) acc = cadd(acc, x[s * q]);
    acc = csub(acc, cscale(cadd(x[0], x[s * m]), 0.5));
    return csub(v, cscale(acc, cf[0].x));
  }
  if (m > 0) v = cfma(cf[m], x[s * (m - 1)], v);
  if (m + 1 < n) v = cfma(cf[2 * n + m], x[s * (m + 1)], v);
  return v;
}
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


// ---- complex products on the tensor cores (tc.cu) ---------------------------
// Logical R x K operand: element (r, k) = X[r * rs + k * ks] (conjugated if
// conj).  tri_mode 1: zero where r > k + tri (upper trapezoid); 2: rows are
// Householder reflectors s and columns their entries i, zero where
// k < r + tri, one where k == r + tri; 3: the same reflectors with rows i and
// columns s (zero where r < k + tri, one where r == k + tri).
struct TcOperandView {
  const cplx* X;
  long long rs, ks;
  int R, K, conj;
  int tri_mode, tri;
};
// Digit planes of an operand split for the tensor cores: 3 components
// (re, im, re + im) x S digits, each R x ldk BF16 (K contiguous), and the
// per-(component, K-chunk, row) power-of-two exponents.
struct TcOperand {
  void* planes;
  int* e;
  int R, K, S;
  long long ldk;
  int nchunks;
};
// Bytes of device memory an operand's digits take (planes + exponents).
size_t tc_operand_bytes(int R, int K, int S, int Kc);
int tc_chunk();       // K-chunk with exact FP32 accumulation (192)
int tc_max_digits();  // 5
// Splits the operand into S digit planes in `buf` (tc_operand_bytes).
cudaError_t tc_split(const TcOperandView& v, int S, TcOperand* out, void* buf, cudaStream_t s);
// out (M x N, column-major, ldo) = alpha * A B^T (+ out if accumulate), with
// alpha a signed power of two, A (M x K) and B (N x K) split operands, i.e. out[m, n] =
// alpha sum_k A(m, k) B(n, k).  K beyond one chunk: per-chunk partials in
// part (tc_part_elems), summed in a fixed order.  err: expiry record.
cudaError_t tc_zgemm(const TcOperand& A, const TcOperand& B, cplx* out, long long ldo, double alpha, int accumulate,
                     cplx* part, size_t part_elems, int* err, cudaStream_t s);
size_t tc_part_elems(int M, int N, int K);

// ---- blocked QR / Q application with tensor-core products (qrtc.cu) -------
// Optional per-phase timing: begin() before a phase's launches returns a
// slot, end() after them records the phase under a profile class (the
// caller's class numbering) with its algorithmic FLOPs.
struct PhaseTimer {
  void* user = nullptr;
  int (*begin)(void* user) = nullptr;
  void (*end)(void* user, int slot, int cls, double flops, int nlaunch) = nullptr;
  int cls_panel = 0, cls_tc = 0, cls_small = 0;
  int b() const { return begin ? begin(user) : -1; }
  void e(int slot, int cls, double flops, int nl) const {
    if (end) end(user, slot, cls, flops, nl);
  }
};
// Used by the mixed-precision rounding for tall factors (qr_tc_applies).
int tc_outer_panel();                                   // 128
bool qr_tc_applies(int m, int p);                       // m rows, p = min(m, k) reflectors
size_t qr_tc_scratch_bytes(int m, int k, int S);        // scratch of one call
size_t qr_tc_gram_elems(int k);                         // complex elements of Gout
// As geqrf (mixed), plus Gout: per outer panel j the Gram v_s^H v_u of its
// reflectors (128 x 128 block at Gout + j 128^2, leading dimension 128),
// which ormqr_tc needs.  T receives the inner panels' records as geqrf.
cudaError_t geqrf_tc(cplx* A, int lda, int m, int k, cplx* tau, cplx* T, cplx* Gout, void* scratch,
                     size_t scratch_bytes, const CoopWs& cws, int S, cudaStream_t s, const PhaseTimer& pt);
// C <- Q C for the Q of geqrf_tc (p reflectors).
cudaError_t ormqr_tc(const cplx* A, int lda, int m, int p, const cplx* tau, const cplx* Gin, cplx* C, int ldc, int q,
                     void* scratch, size_t scratch_bytes, int* err, int S, cudaStream_t s, const PhaseTimer& pt);

// ---- device memory of the library (hopf.cu) -----------------------------------
// Every device allocation of the solver and the surrogate goes through these:
// cudaMalloc / cudaFree, or the caller's functions set by hopf_set_allocator.
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);
// Contexts, tensors and networks alive (the allocator may change only at 0).
void live_add(int delta);

// Watchdog check: a cooperative launch of two CTAs in which CTA 0 never
// reaches the grid barrier, so CTA 1's bounded wait must expire (recorded
// in ws.bar->err after the context's wait limit).  Faults nothing.
cudaError_t watchdog_probe(const CoopWs& ws, cudaStream_t s);

}  // namespace hk
