/*
 * hopf.h -- C ABI of the GB300 (sm_103a) tensor-train solver for the
 * Burgers-Hopf characteristic-function PDE of Rodgers & Venturi, "Tensor
 * approximation of functional differential equations" (arXiv 2403.04946).
 *
 * What is solved.  Phi(a,t) = E[exp(i a . u(t))] for the d cell averages u of
 * the periodic Burgers solution (Sec. 5, Eq. burgers-rxn with alpha = 0 and
 * Eq. BHfde), projected on d cell-indicator functions (Eq. sense) so that it
 * obeys a linear PDE of the form of Eq. (hyper1):
 *     dPhi/dt = sum_k a_k sum_j [ (i/2) D1[k,j] d^2Phi/da_j^2
 *                                 + nu D2[k,j] dPhi/da_j ],
 * D1, D2 the periodic second-order difference matrices in x (text under
 * Eq. pdf-burgers).  Each a_j lives on a_i = (i - n/2) da, da = 2L/n,
 * i = 0..n-1; slot 0 (a = -L) is held at zero and a = +L is a zero ghost.
 * Phi is held in tensor-train format (App. A, "Tensor train decomposition")
 * and advanced by step-truncation RK4 (Eq. discrete-flow-trunc-intro).
 *
 * Conventions shared by every call.
 *  - Complex numbers are pairs of doubles (re, im), interleaved.
 *  - A TT core C_k has shape r_{k-1} x n x r_k with r_0 = r_d = 1 and is
 *    stored column-major, C[i,j,k] = v[i + a j + a b k] (App. A, the
 *    vectorisation under the flattening maps H and V).  Host arrays hold the
 *    d cores back to back in that layout.
 *  - All device work is ordered on the stream given to hopf_create (a
 *    cudaStream_t, e.g. PyTorch's current stream; NULL = legacy default
 *    stream).  Calls that return host data synchronise that stream.
 *  - The library allocates and owns all device memory it uses (contexts,
 *    tensors, workspaces; through the caller's allocator if one is set,
 *    hopf_set_allocator) and frees it in hopf_destroy / tt_free.  Host
 *    arrays passed in are read during the call only; host output arrays
 *    are caller-owned and written before the call returns.
 *  - Every call returns a hopf_status; nothing aborts.  On an error the
 *    context keeps a message (hopf_last_error) and tensors passed in are
 *    left in a valid state (their contents are unspecified after a failed
 *    device step).  A context must not be used from two threads at once.
 *  - Device waits inside the library's cooperative kernels are bounded (a
 *    few seconds of wall time); expiry returns HOPF_ETIMEOUT.
 */
#ifndef HOPF_H
#define HOPF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hopf_ctx hopf_ctx; /* stream, model parameters, workspaces */
typedef struct hopf_tt hopf_tt;   /* one TT on the device: cores + ranks   */

typedef enum {
  HOPF_OK = 0,
  HOPF_EINVAL = 1,   /* bad argument (message in hopf_last_error)          */
  HOPF_ENOMEM = 2,   /* device or host allocation failed                   */
  HOPF_ECUDA = 3,    /* a CUDA call failed                                 */
  HOPF_ENUMERIC = 4, /* NaN/Inf met, or the Jacobi SVD did not converge    */
  HOPF_ETIMEOUT = 5, /* a bounded device-side wait expired                 */
  HOPF_ERANKCAP = 6  /* informational: the rank cap bound, so the error   */
                     /* exceeds the tolerance by the discarded norm        */
} hopf_status;

enum { HOPF_FP64 = 0, HOPF_MIXED = 1 };

typedef struct {
  int d;          /* number of cells / tensor modes, d >= 3               */
  int n;          /* grid points per mode, n >= 4, even                   */
  double nu;      /* viscosity                                            */
  double L;       /* half-width of the a-box; <= 0: set by                */
                  /* hopf_init_gaussian to sqrt(36.8 / min_k C0_kk)       */
  double tol;     /* relative rounding tolerance used by hopf_step        */
  int rank_cap;   /* rank cap used by hopf_step                           */
  int precision;  /* HOPF_FP64: every step in FP64.  HOPF_MIXED: the    */
                  /* dense products of the rounding (QR trailing updates,  */
                  /* Q applications, merges, U^H R) run on the tensor     */
                  /* cores as digit-split BF16 products with exact FP32   */
                  /* accumulation, and the QR panels in double-float      */
                  /* arithmetic (hopf_set_qr_method); Householder         */
                  /* scalars, the SVD that sets the ranks and all storage */
                  /* stay FP64.                                           */
  int nonlinear;  /* 1: full Burgers generator; 0: drop the (i/2) D1 term */
} hopf_params;

/* ---- context ------------------------------------------------------------ */

/* Device memory.  By default the library allocates with cudaMalloc and
 * releases with cudaFree.  hopf_set_allocator routes every device
 * allocation of the library (contexts, tensors, workspaces, networks)
 * through the caller's functions instead, e.g. a framework's caching
 * allocator, so that the solver's memory is accounted and reused with the
 * rest of the process's.  alloc(bytes, user) returns a device pointer
 * aligned to at least 256 bytes, or NULL when it cannot serve the request
 * (the calling entry point then returns HOPF_ENOMEM and leaves its objects
 * valid); free(ptr, user) releases a pointer alloc returned.  Both NULL
 * restores cudaMalloc / cudaFree.  The allocator can change only while no
 * context, tensor or network exists (so that every pointer is released by
 * the functions that allocated it): HOPF_EINVAL otherwise, or when exactly
 * one of the two functions is NULL.  Pinned host staging buffers are not
 * affected. */
typedef void* (*hopf_alloc_fn)(size_t bytes, void* user);
typedef void (*hopf_free_fn)(void* ptr, void* user);
hopf_status hopf_set_allocator(hopf_alloc_fn alloc, hopf_free_fn free, void* user);

/* Creates a context bound to `stream` (cudaStream_t or NULL) on the current
 * device.  `p` is copied.  Errors: HOPF_EINVAL (d < 3 or > 64, n < 4 or odd,
 * rank_cap < 1, tol < 0, unknown precision), HOPF_ENOMEM, HOPF_ECUDA. */
hopf_status hopf_create(const hopf_params* p, void* stream, hopf_ctx** out);
void hopf_destroy(hopf_ctx* ctx);
/* Message of the last failed call on ctx ("" if none).  Owned by ctx. */
const char* hopf_last_error(const hopf_ctx* ctx);
/* Sets / reads the a-box half-width L (> 0; 0 leaves it unset, so that the
 * next hopf_init_gaussian picks it from its covariance). */
hopf_status hopf_set_L(hopf_ctx* ctx, double L);
hopf_status hopf_get_L(const hopf_ctx* ctx, double* L);
/* Changes the viscosity nu (>= 0) of the generator, so that one context
 * (and its workspaces) serves a sequence of solves with different nu. */
hopf_status hopf_set_nu(hopf_ctx* ctx, double nu);
/* Method of the small SVDs of the truncation (App. A, Alg. 4: the SVD of
 * the triangular factor R of each bond).  HOPF_SVD_AUTO (the default):
 * Householder bidiagonalisation, Sturm bisection and inverse iteration
 * (a wide factor through its LQ, whose square triangle has the same
 * singular values and left singular vectors).
 * HOPF_SVD_JACOBI: one-sided Jacobi for every factor.  Both give the same
 * truncation up to rounding.  Errors: HOPF_EINVAL (unknown method). */
enum { HOPF_SVD_AUTO = 0, HOPF_SVD_JACOBI = 1 };
hopf_status hopf_set_svd_method(hopf_ctx* ctx, int method);
/* Limit of the bounded device-side waits of this context's cooperative
 * kernels (the grid barriers of the QR, Q application, SVD and cross
 * kernels): a wait longer than the limit records an expiry, every CTA of
 * the launch leaves, and the call returns HOPF_ETIMEOUT (the context stays
 * usable; the tensors involved have unspecified contents).  seconds in
 * (0, 60]; 0 restores the default of 4 s.  A short limit also serves to
 * check a caller's handling of the expiry path without a fault.  Errors:
 * HOPF_EINVAL (out of range). */
hopf_status hopf_set_wait_limit(hopf_ctx* ctx, double seconds);
/* Exercises the expiry path: launches a two-CTA cooperative kernel whose
 * grid barrier cannot complete (one CTA never arrives), so the other's
 * bounded wait runs out after the context's wait limit.  Returns
 * HOPF_ETIMEOUT when the watchdog works (the context stays usable), or a
 * CUDA error.  Nothing faults; the call blocks for the wait limit. */
hopf_status hopf_check_watchdog(hopf_ctx* ctx);
/* How the mixed-precision rounding factors its tall flattenings (QR of
 * n p x K matrices, App. A Alg. 1/2; in HOPF_FP64 every QR is FP64).
 * HOPF_QR_TENSOR (the default): for factors of at least 4096 rows,
 * blocked Householder in outer panels of 128 columns whose Gram, trailing
 * products and Q applications run on the tensor cores (digit-split BF16
 * products with exact FP32 accumulation, see hopf_tc_zgemm; about 1e-9
 * relative per step), as do the merge products of the orthogonalisation
 * sweep and the projections U^H R of the truncation; each panel by the
 * cooperative kernel below.  1.2x the step rate of the alternative on the
 * d = 32, n = 128, rank-64 workload.
 * HOPF_QR_DOUBLEFLOAT: one cooperative Householder kernel per factor in
 * double-float arithmetic (about 1e-13 relative per step).
 * Errors: HOPF_EINVAL (unknown method). */
enum { HOPF_QR_DOUBLEFLOAT = 0, HOPF_QR_TENSOR = 1 };
hopf_status hopf_set_qr_method(hopf_ctx* ctx, int method);
/* Autotuning of the mixed-precision tall-factor QR (no counterpart in the
 * paper; the factorisations themselves are App. A Alg. 1/2).  With enable =
 * 1, the first QR of every new shape (m rows, p = min(m, k) reflectors, for
 * factors the tensor-core form applies to) times four configurations on
 * copies of the matrix, two runs each: tensor-core products or double-float
 * kernel alone (hopf_set_qr_method) x the cooperative panel kernel on all
 * the context's SMs or half of them; the fastest is used from then on for
 * that shape, for the factorisation and the application of its Q alike.
 * Results differ between configurations at the mixed path's rounding level
 * (about 1e-9 relative per step), so a tuned run is reproducible only with
 * the same table.  The first QR of a shape costs about nine times one QR
 * and two temporary copies of the matrix in device memory.  enable = 0
 * clears the table (the hopf_set_qr_method choice applies everywhere).
 * Errors: HOPF_EINVAL. */
hopf_status hopf_set_autotune(hopf_ctx* ctx, int enable);
/* The autotuning table: *count receives the number of tuned shapes; the
 * first min(cap, *count) entries are written as shapes[4 i ..] = (m, p,
 * method chosen, CTAs chosen: 0 = all) and ms[4 i ..] = the candidates'
 * times in milliseconds (tensor-core on all SMs, tensor-core on half,
 * double-float on all, double-float on half; +inf for a candidate that was
 * not run).  Host arrays, caller-owned.  Errors: HOPF_EINVAL. */
hopf_status hopf_get_autotune(const hopf_ctx* ctx, int* shapes, float* ms, int cap, int* count);
/* Limits every cooperative kernel launched by this context to max_ctas
 * CTAs, one per SM (0, the default: all SMs).  Several contexts whose
 * limits add up to at most the SM count run their solves concurrently on
 * their own streams (one host thread per context): an ensemble of
 * independent initial states, each too small to fill the GPU, advances in
 * parallel.  The paper solves one state at a time; this is a scheduling
 * option only, results are unchanged.  Errors: HOPF_EINVAL (negative). */
hopf_status hopf_set_max_ctas(hopf_ctx* ctx, int max_ctas);

/* Selects the equation the context's generator stands for.
 * HOPF_EQ_PHI (the default): the characteristic-function PDE above, box
 * half-width L (box = L; 0 leaves it unset).
 * HOPF_EQ_CDF: the paper's CDF equation of the same Burgers dynamics
 * (Sec. 5, Eq. cdf-burgers, reaction alpha = 0) for the joint CDF
 * F(u_1..u_d) of the d grid values, on u_k = -box + k du, du = 2 box/(n-1),
 * k = 0..n-1 (both box edges on the grid; the paper's box is 1.3): centred
 * differences with dF/du = 0 on the box boundary (outflow), trapezoidal
 * integrals from the lower edge, viscosity gamma = the context's nu.  Its
 * operator has the same bond structure as the PDE's (each neighbour pair
 * (m, m+1) contributes P+_m K_{m+1} + K_m P-_{m+1}, K = u - integral), so
 * hopf_apply_op, tt_round and the step schemes serve it unchanged.
 * The paper's numerical-diffusion stabiliser is not part of it (its
 * coefficient is not given).  hopf_eval_moments and hopf_init_gaussian
 * refuse a CDF context.  Errors: HOPF_EINVAL (unknown equation, box <= 0
 * for the CDF). */
enum { HOPF_EQ_PHI = 0, HOPF_EQ_CDF = 1 };
hopf_status hopf_set_equation(hopf_ctx* ctx, int equation, double box);
/* Initial state of the CDF equation (Sec. 5): F(u, 0) = prod_k g(u_k - mu_k),
 * g(u) = (1 + erf(u / (sigma sqrt 2))) / 2, a rank-1 TT with zero imaginary
 * parts (the paper: sigma = 0.25, mu = 0).  mu: host [d] or NULL (zero).
 * *out has capacity rank_cap.  Errors: HOPF_EINVAL (not a CDF context,
 * sigma <= 0). */
hopf_status hopf_init_cdf(hopf_ctx* ctx, double sigma, const double* mu, hopf_tt** out);

/* ---- model set-up -------------------------------------------------------- */

/* Projection of the Gaussian initial state on the cell-indicator basis
 * (Eq. sense): m0_k = (1/h) int_{I_k} mu, C0_jk = (1/h^2) int int K, with
 * mu(x) = sum_{m=1}^{nmodes} alpha[m-1] cos(m x) + beta[m-1] sin(m x) and
 * the periodic squared-exponential kernel
 * K(x,y) = sigma^2 exp(-2 sin^2((x-y)/2) / ell^2), by 12-point tensor
 * Gauss-Legendre quadrature per cell, computed on the device.
 * m0: host [d]; C0: host [d*d] (symmetric).  Errors: HOPF_EINVAL. */
hopf_status hopf_cell_moments(hopf_ctx* ctx, int nmodes, const double* alpha,
                              const double* beta, double sigma, double ell,
                              double* m0, double* C0);

/* ---- tensors ------------------------------------------------------------- */

/* Uploads a TT: ranks[d+1] (ranks[0] = ranks[d] = 1, each <= max_rank),
 * cores as described above (2 * sum_k r_{k-1} n r_k doubles).  `max_rank`
 * (>= every rank) fixes the device capacity of every core.  The TT has the
 * context's d and n.  Errors: HOPF_EINVAL, HOPF_ENOMEM, HOPF_ECUDA. */
hopf_status tt_from_host(hopf_ctx* ctx, const int* ranks, const double* cores,
                         int max_rank, hopf_tt** out);
/* Allocates an empty TT (all ranks 1, cores zero) with capacity max_rank. */
hopf_status tt_create(hopf_ctx* ctx, int max_rank, hopf_tt** out);
/* Copies ranks[d+1] to the host. */
hopf_status tt_get_ranks(const hopf_tt* t, int* ranks);
/* Number of doubles tt_to_host writes: 2 * sum_k r_{k-1} n r_k. */
hopf_status tt_size(const hopf_tt* t, size_t* ndoubles);
/* Downloads the cores (layout above) into `cores` (capacity `cap_doubles`).
 * Errors: HOPF_EINVAL if the capacity is too small. */
hopf_status tt_to_host(const hopf_tt* t, double* cores, size_t cap_doubles);
/* dst <- src (dst capacity must hold src's ranks). */
hopf_status tt_copy(hopf_ctx* ctx, const hopf_tt* src, hopf_tt* dst);
void tt_free(hopf_tt* t);

/* ---- the hot path (Sec. 4.1 and App. A) ---------------------------------- */

/* Builds the TT of Phi0(a) = exp(i a.m0 - a^T C0 a / 2), zero on the
 * boundary slot, rounded to the context's tol and rank_cap (Sec. 5's
 * Gaussian random initial state).  m0: host [d], C0: host [d*d]
 * (column-major, symmetric positive definite).  If the context's L <= 0 it
 * is set first to sqrt(36.8 / min_k C0_kk).  Diagonal C0 gives the exact
 * rank-1 product for any d.  A correlated C0 is built by rounding the exact
 * full-grid TT when n^d <= 2^20, and otherwise by TT-cross interpolation
 * (exact at the cross points, ranks up to rank_cap <= 256, two alternating
 * sweeps) followed by the rounding.  HOPF_ERANKCAP: the cap bound.
 * *out is allocated with capacity rank_cap. */
hopf_status hopf_init_gaussian(hopf_ctx* ctx, const double* m0,
                               const double* C0, hopf_tt** out);

/* out <- G(in): the generator applied core by core as a matrix product
 * operator of bond dimension 6 (Eq. hyper1 for 1-D Burgers; rank growth
 * under operator application, Sec. 4.1): out ranks are 6 r_k (interior).
 * `out` must have capacity >= 6 * max rank of `in`; it is not rounded. */
hopf_status hopf_apply_op(hopf_ctx* ctx, const hopf_tt* in, hopf_tt* out);

/* In-place TT rounding (App. A, Alg. 2 in its mirrored form with the
 * factor-then-SVD structure of Alg. 4): right-to-left Householder LQ sweep
 * (Alg. 1 mirrored), then left-to-right truncated SVDs of the small
 * triangular factors with per-SVD tolerance tol * ||f||_F / sqrt(d-1); each
 * rank is the smallest rho >= 1 whose discarded tail norm is <= that
 * tolerance, then capped at rank_cap.  forced_ranks: NULL, or host [d+1]
 * ranks to use instead of the tolerance rule (ranks replay).
 * discarded_norm (may be NULL): sqrt(sum of squared discarded tails), a
 * bound on ||g - f||_F.  Returns HOPF_ERANKCAP (result valid) when the cap
 * overrode the tolerance rule. */
hopf_status tt_round(hopf_ctx* ctx, hopf_tt* inout, double tol, int rank_cap,
                     const int* forced_ranks, double* discarded_norm);

/* out <- sum_t coef[t] * term[t] by block concatenation (App. A, TT sum and
 * scalar multiplication).  coef: host [2*nterms] complex.  `out` must not
 * alias a term and needs capacity >= sum of the terms' ranks. */
hopf_status tt_sum(hopf_ctx* ctx, int nterms, const hopf_tt* const* terms,
                   const double* coef, hopf_tt* out);

/* nsteps step-truncation RK4 steps (Eq. discrete-flow-trunc-intro with the
 * classical RK4 increment): K_s = T[G Y_s], Y_2 = T[f + dt/2 K_1],
 * Y_3 = T[f + dt/2 K_2], Y_4 = T[f + dt K_3],
 * f <- T[f + dt/6 (K_1 + 2 K_2 + 2 K_3 + K_4)], every T at the context's
 * tol and rank_cap.  `inout` needs capacity >= rank_cap.
 * discarded_norm_sum (may be NULL): sum of the 8 * nsteps discarded norms.
 * rank_log (may be NULL): host [8 * nsteps * (d+1)] ints receiving the ranks
 * after every rounding (for ranks replay).  forced_log (may be NULL): host
 * ranks to replay, same layout.  Returns HOPF_ERANKCAP if the cap bound. */
hopf_status hopf_step(hopf_ctx* ctx, hopf_tt* inout, double dt, int nsteps,
                      double* discarded_norm_sum, int* rank_log,
                      const int* forced_log);

/* Step-truncation schemes (Sec. 4, "Step-truncation tensor methods"):
 *  HOPF_RK4       classical RK4 increment, 8 roundings per step (hopf_step);
 *  HOPF_EULER     truncated explicit Euler, Eq. (adaptive-euler-method):
 *                 f <- T[f + dt T[G f]], 2 roundings per step;
 *  HOPF_MIDPOINT  truncated explicit midpoint, Eq. (adaptive-midpoint-method):
 *                 f <- T[f + dt T[G(f + dt/2 T[G f])]], 3 roundings per step,
 *                 the inner sum untruncated as printed (the operator then acts
 *                 on ranks up to 2 rank_cap).
 * Every T at the context's tol and rank_cap.  Arguments as hopf_step, with
 * rank_log / forced_log holding (roundings per step) x nsteps x (d+1) ints.
 * Errors as hopf_step, HOPF_EINVAL for an unknown scheme. */
enum { HOPF_RK4 = 0, HOPF_EULER = 1, HOPF_MIDPOINT = 2 };
hopf_status hopf_step_scheme(hopf_ctx* ctx, hopf_tt* inout, int scheme, double dt, int nsteps,
                             double* discarded_norm_sum, int* rank_log, const int* forced_log);

/* Advances an ensemble of independent states (Sec. 5: the Gaussian random
 * initial states are solved one at a time in the paper; here several are in
 * flight at once): hopf_step(ctxs[a], tts[a], dt[a], nsteps) for every a,
 * each on its own host thread and its context's stream and device.  The
 * contexts must be distinct and should have hopf_set_max_ctas limits that
 * add up to at most the SM count so that their cooperative kernels run
 * side by side.  statuses: host [count], per-member status.  Returns the
 * first failure, else HOPF_ERANKCAP if any cap bound, else HOPF_OK. */
hopf_status hopf_step_ensemble(int count, hopf_ctx* const* ctxs, hopf_tt* const* tts,
                               const double* dt, int nsteps, hopf_status* statuses);

/* Mean and covariance of u from central differences of Phi at a = 0
 * (Sec. 1: moments are functional derivatives of Phi at theta = 0):
 * mean_k = Re[-i (Phi(+da e_k) - Phi(-da e_k)) / (2 da)],
 * E[u_j u_k] = -(mixed central difference) for j != k, -(second difference)
 * for j == k, cov = E[u u^T] - mean mean^T.  mean: host [d]; cov: host
 * [d*d]; imag_resid (may be NULL): host [1], the largest imaginary part met
 * (diagnostic; exactly zero for a Hermitian-symmetric Phi). */
hopf_status hopf_eval_moments(hopf_ctx* ctx, const hopf_tt* t, double* mean,
                              double* cov, double* imag_resid);

/* Phi at npts grid multi-indices idx (host [npts*d], row-major, each in
 * [0, n)).  vals: host [2*npts] complex.  Device staging is kept by the
 * context between calls (grown to the largest request). */
hopf_status hopf_eval_points(hopf_ctx* ctx, const hopf_tt* t, int npts,
                             const int* idx, double* vals);

/* Allocation-free variant of hopf_eval_points (the paper has no counterpart;
 * it exists for callers that cannot allocate device memory).
 *
 * hopf_eval_points allocates its device staging buffers with cudaMalloc and
 * releases them with cudaFree on every call.  cudaFree waits for all work on
 * the device, so a caller that probes Phi between solver steps while other
 * streams keep the GPU busy would stall them; and a process whose device
 * memory is fully reserved by another allocator may not be able to allocate
 * at all.  This call stages the same data in two fixed arrays inside the
 * library's device image instead (HOPF_NOALLOC_MAX_POINTS points of at most
 * HOPF_NOALLOC_MAX_D modes: 512 KiB of indices and 32 KiB of results,
 * reserved on every GPU that loads the library until the process exits).
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Arguments and results are those of hopf_eval_points (the tensor's context
 * and stream are used).  npts > HOPF_NOALLOC_MAX_POINTS or d >
 * HOPF_NOALLOC_MAX_D returns HOPF_EINVAL.  The work runs on the device of
 * the tensor's context: the call makes that device current for its duration
 * and restores the caller's current device before it returns.  The first
 * call on a device looks up the arrays' device addresses there; make that
 * first call before any stream capture.  All calls share the two arrays:
 * calls whose GPU work overlaps (on different streams or contexts) race on
 * them and must be serialised by the caller. */
#define HOPF_NOALLOC_MAX_POINTS 2048
#define HOPF_NOALLOC_MAX_D 64
hopf_status hopf_eval_points_noalloc(const hopf_tt* t, int npts, const int* idx, double* vals);

/* Checkpoint and resume.  tt_save writes the TT (d, n, ranks, the cores in
 * the layout above as FP64) and a time stamp to `path` in this machine's
 * byte order: 8 bytes "HOPFTT\0\1", int32 d, int32 n, int32 ranks[d+1],
 * double time, then 2 sum_k r_{k-1} n r_k doubles.  tt_load reads such a
 * file into a new tensor of ctx (capacity max(max_rank, largest rank)) and
 * its time stamp into *time (may be NULL).  The kernels reduce in a fixed
 * order, so stepping a loaded tensor gives bitwise the same result as
 * stepping the saved one.  Errors: HOPF_EINVAL (cannot open or write, not
 * such a file, another d or n), HOPF_ENOMEM, HOPF_ECUDA. */
hopf_status tt_save(const hopf_tt* t, const char* path, double time);
hopf_status tt_load(hopf_ctx* ctx, const char* path, int max_rank, hopf_tt** out, double* time);

/* ||t||_F (by orthogonalisation, computed on the device). */
hopf_status tt_norm(hopf_ctx* ctx, const hopf_tt* t, double* norm);

/* Overwrites t with host cores (same layout and rules as tt_from_host; the
 * ranks must fit t's capacity).  No device allocation. */
hopf_status tt_set_from_host(hopf_tt* t, const int* ranks, const double* cores);

/* ---- learned surrogate: a small multilayer perceptron ------------------- */
/* Not part of the paper's method: a network that maps the parameters of a
 * Gaussian initial state (nu, sigma, ell, Fourier coefficients of the mean,
 * horizon T) to the mean and covariance of the cell averages at T, trained
 * only on outputs of this solver, with the solver as its fallback.
 *
 * Network.  Linear layers l = 0..depth over the widths
 * [n_in, width (depth times), n_out]; every hidden layer is followed by
 * GELU(z) = z Phi(z) (Phi the standard normal CDF, Hendrycks & Gimpel 2016),
 * the last layer is linear.  Parameters of one member, packed: for each
 * layer W_l (fan_out x fan_in, row-major) then b_l (fan_out); P floats per
 * member, `members` members back to back ([members][P]).  The library keeps
 * FP32 master parameters and Adam moments; products read BF16 copies of the
 * weights (round to nearest even) with FP32 activations and FP32
 * accumulation; biases stay FP32.  The products run on the tensor cores
 * (BF16 x BF16 -> FP32): an FP32 operand enters as three BF16 parts
 * (hi + mid + lo, 24 significant bits), so the result is the FP32 product
 * up to FP32 accumulation rounding.  A bounded wait that expires inside
 * them returns HOPF_ETIMEOUT. 
 *
 * Normalisation.  hopf_mlp_set_data stores a data set and its per-column
 * mean and population standard deviation (1 for a constant column).  The
 * network sees x_hat = (x - mu_x) / sd_x and is trained on
 * y_hat = (y - mu_y) / sd_y with the mean-squared error over batch and
 * outputs; predictions are mapped back to y = mu_y + sd_y * net(x_hat).
 *
 * Ensemble and error bound.  The members are trained independently (their
 * own initial parameters and batches) in the same launches.  A prediction
 * is the member mean ybar, and its error bound is
 * kappa * ||s||_2 / ||ybar||_2, s the per-output standard deviation over the
 * members: the caller calibrates kappa on held-out solves and sends every
 * query whose bound is too large to the solver.
 *
 * Training runs Adam (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8)
 * as one CUDA graph per step, replayed `iters` times on the library's own
 * stream (ordered after the context's stream; the call returns when done).
 * Random draws (initial parameters, batch indices) are inputs. */
typedef struct hopf_mlp hopf_mlp;
typedef struct {
  int n_in, width, depth, n_out; /* depth >= 0 hidden layers; sizes 1..4096 */
  int members;                   /* 1..64 networks in the ensemble         */
  int max_batch;                 /* largest training batch, and the chunk  */
                                 /* size of hopf_mlp_predict               */
} hopf_mlp_params;

/* Creates a network on the context's device with initial parameters `init`
 * (host [members][P] floats, P from hopf_mlp_param_count).  Errors:
 * HOPF_EINVAL, HOPF_ENOMEM, HOPF_ECUDA. */
hopf_status hopf_mlp_create(hopf_ctx* ctx, const hopf_mlp_params* p,
                            const float* init, hopf_mlp** out);
/* P, the number of parameters of one member. */
hopf_status hopf_mlp_param_count(const hopf_mlp_params* p, long long* P);
/* Copies the FP32 master parameters to host [members][P]. */
hopf_status hopf_mlp_get_params(hopf_mlp* m, float* out);
/* Stores nsamples (x, y) pairs (host, row-major [nsamples][n_in] and
 * [nsamples][n_out], doubles) on the device and computes the normalisation
 * statistics from them; stats (may be NULL) receives host
 * [2 (n_in + n_out)] = mu_x, sd_x, mu_y, sd_y.  Errors: HOPF_EINVAL for
 * nsamples < 1 or non-finite data. */
hopf_status hopf_mlp_set_data(hopf_mlp* m, int nsamples, const double* x,
                              const double* y, double* stats);
/* Runs `iters` Adam steps.  idx: host [iters][members][batch] sample
 * indices in [0, nsamples); lr: host [iters] learning rates; loss (may be
 * NULL): host [iters][members], the batch loss before each step.  Errors:
 * HOPF_EINVAL (no data, batch outside [1, max_batch], index out of range),
 * HOPF_ECUDA. */
hopf_status hopf_mlp_train(hopf_mlp* m, int iters, int batch, const int* idx,
                           const float* lr, float* loss);
/* Loss and gradient at the current parameters for one batch per member
 * (idx: host [members][batch]), without an update.  loss: host [members];
 * grad: host [members][P] (FP32). */
hopf_status hopf_mlp_loss_grad(hopf_mlp* m, int batch, const int* idx,
                               float* loss, float* grad);
/* Ensemble prediction for nq queries x (host [nq][n_in]).  Member m
 * answers y_m = base + scale * (mu_y + sd_y * net_m(x_hat)), with base
 * (host [nq][n_out], may be NULL: 0) and scale (host [nq], may be NULL: 1)
 * per query, so that a network trained on a rate or an increment answers in
 * the units of the full quantity.  y: host [nq][n_out], the member mean;
 * bound: host [nq], kappa ||s||_2 / ||y||_2 with s the per-output standard
 * deviation of y_m over the members; members_y (may be NULL): host
 * [members][nq][n_out].  Errors: HOPF_EINVAL (no statistics yet, nq < 0,
 * kappa < 0). */
hopf_status hopf_mlp_predict(hopf_mlp* m, int nq, const double* x,
                             const double* base, const double* scale,
                             double kappa, double* y, double* bound,
                             double* members_y);
void hopf_mlp_free(hopf_mlp* m);

/* ---- tensor-core products (diagnostic) ------------------------------------ */

/* C = op(A) op(B) for complex matrices through the library's tensor-core
 * path: the digit-split (Ozaki-style) BF16 products with exact FP32
 * accumulation that the mixed-precision rounding uses for its dense
 * contractions (App. A, Alg. 4's products), with three real products per
 * complex one.  op(X) = X (op 0) or X^H (op 1).  A: host, column-major,
 * op(A) is M x K (A itself is M x K with lda >= M, or K x M with lda >= K);
 * B likewise with op(B) K x N; C: host M x N, ldc >= M.  digits: 1..5
 * (each 8 bits of every operand row, relative to the row's largest
 * entry; 5 digits give about 5e-12 of |op(A)| |op(B)|).  Exposed so that the
 * products can be checked directly; the solver calls the same kernels.
 * Errors: HOPF_EINVAL (sizes, digits), HOPF_ENOMEM, HOPF_ETIMEOUT, HOPF_ECUDA. */
hopf_status hopf_tc_zgemm(hopf_ctx* ctx, int M, int N, int K, const double* A, int lda, int opA,
                          const double* B, int ldb, int opB, int digits, double* C, int ldc);

/* ---- instrumentation ----------------------------------------------------- */

/* Kernel classes of the profile record. */
enum {
  HOPF_K_QR = 0,      /* Householder QR panels + trailing updates           */
  HOPF_K_APPLYQ = 1,  /* application of Householder Q factors               */
  HOPF_K_SVD = 2,     /* one-sided Jacobi SVD                               */
  HOPF_K_APPLY = 3,   /* operator apply (MPO x TT)                          */
  HOPF_K_GEMM = 4,    /* small dense products (merges, projections)         */
  HOPF_K_SUM = 5,     /* TT sums, copies, transposes                        */
  HOPF_K_SMALL = 6,   /* rank selection, gathers, norms, set-up             */
  HOPF_K_TC = 7,      /* tensor-core products of the mixed precision (digit */
                      /* splitting included); flops counted as FP64-       */
                      /* equivalent complex products, 8 per multiply-add   */
  HOPF_K_NCLASS = 8
};
typedef struct {
  double ms[HOPF_K_NCLASS];        /* device time (CUDA events around each */
                                   /* launch on the context's stream)      */
  double flops[HOPF_K_NCLASS];     /* algorithmic real FLOPs               */
  double bytes[HOPF_K_NCLASS];     /* algorithmic DRAM bytes (apply, sums) */
  long long launches[HOPF_K_NCLASS]; /* kernels launched                   */
  long long timed_launches[HOPF_K_NCLASS]; /* launches covered by ms      */
  long long svd_count;             /* Jacobi SVDs run                      */
  long long svd_sweeps;            /* their sweeps, summed                 */
} hopf_profile;

/* Turns per-launch event timing on or off (launch counting is always on).
 * Timing adds two event records per launch on the context's stream. */
hopf_status hopf_profile_enable(hopf_ctx* ctx, int on);
/* Copies the accumulated record into *out (synchronises the stream);
 * reset != 0 zeroes it afterwards. */
hopf_status hopf_profile_read(hopf_ctx* ctx, hopf_profile* out, int reset);

#ifdef __cplusplus
}
#endif
#endif /* HOPF_H */
