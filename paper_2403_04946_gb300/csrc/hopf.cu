// C ABI of the solver (include/hopf.h): contexts, tensors, and the host
// orchestration of the hot path.  All arithmetic runs in the kernels of
// qr.cu, svd.cu and tt.cu; the host keeps the TT ranks, launches kernels with
// exact dimensions, and reads back one small record per truncation (the rank
// chosen for the next core depends on the singular values just computed).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <set>
#include <thread>
#include <atomic>
#include <vector>

#include "../../include/hopf.h"
#include "kernels.h"

// cplx (double2) comes from common.cuh

struct hopf_tt {
  hopf_ctx* ctx = nullptr;
  int d = 0, n = 0, cap_rank = 0;
  std::vector<size_t> core_cap;  // capacity (elements) of each core buffer
  std::vector<cplx*> cores;
  std::vector<int> ranks;        // host copy, authoritative
  cplx** d_ptrs = nullptr;       // device copy of `cores`
  int* d_ranks = nullptr;        // device copy of `ranks`
};

struct RoundWs {
  size_t elems = 0;  // capacity of each big buffer (elements)
  int d = 0;
  int kcap = 0;      // largest rank the workspace serves
  std::vector<cplx*> B;   // per-core QR buffers (phase 1)
  cplx* W1 = nullptr;     // phase-2 scratch
  cplx* tau = nullptr;    // d * kcap
  cplx* T = nullptr;      // d * tstride
  size_t tstride = 0;
  cplx* tau2 = nullptr;   // kcap
  cplx* T2 = nullptr;     // tstride
  cplx* Rb = nullptr;     // kcap * kcap
  cplx* Mb = nullptr;     // kcap * kcap
  cplx* Jb = nullptr;     // kcap * kcap
  cplx* Ub = nullptr;     // kcap * kcap
  cplx* Sb = nullptr;     // kcap * kcap
  double* sig = nullptr;  // 2 * kcap + 2
  int* perm = nullptr;    // kcap
  // bidiagonal SVD of square factors
  double* bd_d = nullptr;     // kcap
  double* bd_e = nullptr;     // kcap
  cplx* bd_tauq = nullptr;    // kcap
  cplx* bd_taup = nullptr;    // kcap
  float2* bd_a2 = nullptr;    // 2 * kcap
  double* bd_info = nullptr;  // 4
  double* bd_X = nullptr;     // kcap * kcap
  double* bd_Zs = nullptr;    // kcap * 2 kcap
  // mixed precision, tensor-core QR: per core the Gram blocks of the
  // phase-1 reflectors (gstride elements each), and those of phase 2's QR
  cplx* G = nullptr;
  size_t gstride = 0;
  cplx* G2 = nullptr;
  // rows of a bidiagonalisation too large for shared memory
  cplx* bd_rows = nullptr;
};

struct hopf_ctx {
  hopf_params p{};
  cudaStream_t stream = nullptr;
  std::string err;
  double L = 0.0;      // a-box half-width (Phi), or the u-box half-width U (CDF)
  int equation = HOPF_EQ_PHI;
  // operator tables
  cplx* d_coef = nullptr;             // kNumOps ops x 3 x n
  unsigned char* d_blocks = nullptr;  // 3 site kinds x 36
  unsigned long long op_forms = 0;    // hk::OpTable::forms of d_coef (0: apply untiled)
  double* d_agrid = nullptr;          // n
  std::vector<double> agrid;
  // cooperative-kernel workspace
  hk::CoopWs coop{};
  int coop_kcap = 0;
  int device = 0;
  int svd_method = HOPF_SVD_AUTO;
  int qr_method = HOPF_QR_TENSOR;
  // per-shape choice of the tall-factor QR configuration (hopf_set_autotune)
  struct QrTune {
    int m, p, method, ctas;
    float ms[4];
  };
  int autotune = 0;
  std::vector<QrTune> tune;
  unsigned int wait_limit_us = 0;  // grid-barrier wait limit (0: the default)
  // persistent staging of point / moment evaluation (grown on demand)
  int* ev_idx = nullptr;
  cplx* ev_vals = nullptr;
  double* ev_out = nullptr;
  size_t ev_idx_cap = 0, ev_vals_cap = 0, ev_out_cap = 0;
  // small device scalars and pinned mirrors
  double* d_dbl = nullptr;  // [16]
  int* d_int = nullptr;     // [16]
  double* h_dbl = nullptr;  // pinned [16]
  int* h_int = nullptr;     // pinned [16]
  RoundWs rw;
  // scratch of the tensor-core QR / Q application (grown on demand)
  void* tcbuf = nullptr;
  size_t tcbytes = 0;
  // hopf_step workspace
  hopf_tt* big = nullptr;
  hopf_tt* kst[4] = {nullptr, nullptr, nullptr, nullptr};
  hopf_tt* ytmp = nullptr;
  int step_scheme = -1;            // scheme the step workspace was sized for
  hk::SumTerm* d_terms = nullptr;  // [16]
  std::vector<void*> extra;        // other device allocations to free
  // launch instrumentation
  struct ProfRec {
    int cls, slot;
    double flops, bytes;
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;  // 2 per slot
  std::vector<ProfRec> prof_recs;
  hopf_profile prof{};
};

// ---------------------------------------------------------------------------
// Library-wide device allocator (hopf_set_allocator) and the count of live
// contexts and tensors, which must be zero while the allocator changes.
namespace {
hopf_alloc_fn g_alloc = nullptr;
hopf_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;
std::atomic<long long> g_live{0};
}  // namespace

namespace hk {
cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  if (g_alloc) {
    *p = g_alloc(bytes, g_alloc_user);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}
void dev_free(void* p) {
  if (!p) return;
  if (g_free) g_free(p, g_alloc_user);
  else cudaFree(p);
}
void live_add(int delta) { g_live += delta; }
}  // namespace hk

namespace {

hopf_status fail(hopf_ctx* c, hopf_status st, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return st;
}

#define CK(expr)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      if (e_ == cudaErrorMemoryAllocation) {                                        \
        cudaGetLastError();                                                         \
        return fail(ctx, HOPF_ENOMEM, "%s: %s", #expr, cudaGetErrorString(e_));     \
      }                                                                             \
      return fail(ctx, HOPF_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));        \
    }                                                                               \
  } while (0)

// Mixed precision: FP32 trailing updates and products in QR / apply-Q /
// merges; FP64 Householder panels and Jacobi SVD.
#define MIXED_FLAG (ctx->p.precision == HOPF_MIXED ? 1 : 0)

#define TRY(expr)                        \
  do {                                   \
    hopf_status s_ = (expr);             \
    if (s_ != HOPF_OK) return s_;        \
  } while (0)

// ---- launch instrumentation ----------------------------------------------------
constexpr int kProfSlots = 4096;

hopf_status prof_flush(hopf_ctx* ctx) {
  if (ctx->prof_recs.empty()) return HOPF_OK;
  CK(cudaEventSynchronize(ctx->prof_ev[2 * ctx->prof_recs.back().slot + 1]));
  for (const auto& r : ctx->prof_recs) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->prof_ev[2 * r.slot], ctx->prof_ev[2 * r.slot + 1]));
    ctx->prof.ms[r.cls] += ms;
    ctx->prof.timed_launches[r.cls] += 1;
  }
  ctx->prof_recs.clear();
  return HOPF_OK;
}

int prof_begin(hopf_ctx* ctx) {
  if (!ctx->prof_on) return -1;
  if ((int)ctx->prof_recs.size() >= kProfSlots && prof_flush(ctx) != HOPF_OK) return -1;
  const int slot = (int)ctx->prof_recs.size();
  if (cudaEventRecord(ctx->prof_ev[2 * slot], ctx->stream) != cudaSuccess) return -1;
  return slot;
}

void prof_end(hopf_ctx* ctx, int slot, int cls, double flops, double bytes, int nlaunch) {
  ctx->prof.launches[cls] += nlaunch;
  ctx->prof.flops[cls] += flops;
  ctx->prof.bytes[cls] += bytes;
  if (slot < 0) return;
  if (cudaEventRecord(ctx->prof_ev[2 * slot + 1], ctx->stream) != cudaSuccess) return;
  ctx->prof_recs.push_back({cls, slot, flops, bytes});
}

// Launch `expr` (a kernel launcher returning cudaError_t) as one profiled
// unit of class `cls` with algorithmic flops/bytes and `nl` kernels.
#define LAUNCH(cls, flops, bytes, nl, expr)                 \
  do {                                                      \
    const int ps_ = prof_begin(ctx);                        \
    CK(expr);                                               \
    prof_end(ctx, ps_, (cls), (flops), (bytes), (nl));      \
  } while (0)

// Algorithmic real FLOPs (complex = 4 real multiplies + adds per MAC pair):
// Householder QR of m x k (LAPACK count for the complex case).
double qr_flops(double m, double k) {
  return (m >= k) ? 8.0 * m * k * k - 8.0 * k * k * k / 3.0 : 8.0 * k * m * m - 8.0 * m * m * m / 3.0;
}
// Bidiagonalisation of a square n x n complex matrix (LAPACK count).
double gebrd_flops(double n) { return 32.0 * n * n * n / 3.0; }
// Q (m x m, p reflectors) applied to an m x q block.
double applyq_flops(double m, double q, double p) { return 16.0 * m * q * p - 8.0 * q * p * p; }
// C = A R^H with R upper trapezoidal N x K: sum_j (K - j) MACs per row.
double arh_flops(double M, double K, double N) {
  const double Nn = std::min(N, K);
  return 8.0 * M * (Nn * K - Nn * (Nn - 1) / 2.0);
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return hk::dev_alloc((void**)p, count * sizeof(T));
}
inline void dfree(void* p) { hk::dev_free(p); }

// ---- per-mode operator coefficients ------------------------------------------
// (op x)[i] = lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1] on a_i = (i - n/2) da,
// slot 0 with zero row and column for A, D, S (and so for P, Q, Z).
hopf_status build_ops_cdf(hopf_ctx* ctx);

// hk::OpTable::forms of a coefficient table of three-point operators.
unsigned long long op_forms(const std::vector<cplx>& coef, int n) {
  unsigned long long f = 1ull << 63;
  for (int op = 0; op < hk::kNumOps; ++op) {
    unsigned b = 0;
    bool ident = true;
    for (int w = 0; w < 3; ++w)
      for (int i = 0; i < n; ++i) {
        const cplx c = coef[(size_t)op * 3 * n + (size_t)w * n + i];
        if (c.x != 0.0) b |= 1u << (2 * w);
        if (c.y != 0.0) b |= 2u << (2 * w);
        if (c.y != 0.0 || c.x != (w == 1 ? 1.0 : 0.0)) ident = false;
      }
    f |= (unsigned long long)(ident ? 0x40u : b) << (8 * op);
  }
  return f;
}

hopf_status build_ops(hopf_ctx* ctx) {
  if (ctx->equation == HOPF_EQ_CDF) return build_ops_cdf(ctx);
  const int n = ctx->p.n, d = ctx->p.d;
  const double L = ctx->L;
  const double da = 2.0 * L / n;
  const double h = 2.0 * M_PI / d;
  ctx->agrid.assign(n, 0.0);
  for (int i = 0; i < n; ++i) ctx->agrid[i] = (i - n / 2) * da;
  std::vector<cplx> coef((size_t)hk::kNumOps * 3 * n, cplx{0.0, 0.0});
  auto set = [&](int op, int which, int i, cplx v) { coef[(size_t)op * 3 * n + (size_t)which * n + i] = v; };
  const cplx cS = ctx->p.nonlinear ? cplx{0.0, 1.0 / (4.0 * h)} : cplx{0.0, 0.0};
  const double e = ctx->p.nu / (h * h);
  for (int i = 0; i < n; ++i) {
    // identity keeps every slot
    set(hk::OP_I, 1, i, cplx{1.0, 0.0});
    if (i == 0) continue;
    const double a = ctx->agrid[i];
    set(hk::OP_A, 1, i, cplx{a, 0.0});
    // D: -1/(2da) on the left (column >= 1), +1/(2da) on the right (column < n)
    const double dlo = (i >= 2) ? -1.0 / (2 * da) : 0.0;
    const double dup = (i + 1 < n) ? 1.0 / (2 * da) : 0.0;
    // S: (1, -2, 1)/da^2
    const double slo = (i >= 2) ? 1.0 / (da * da) : 0.0;
    const double sdi = -2.0 / (da * da);
    const double sup = (i + 1 < n) ? 1.0 / (da * da) : 0.0;
    // P = cS + eD, Q = -cS + eD (c purely imaginary)
    set(hk::OP_P, 0, i, cplx{e * dlo, cS.y * slo});
    set(hk::OP_P, 1, i, cplx{0.0, cS.y * sdi});
    set(hk::OP_P, 2, i, cplx{e * dup, cS.y * sup});
    set(hk::OP_Q, 0, i, cplx{e * dlo, -cS.y * slo});
    set(hk::OP_Q, 1, i, cplx{0.0, -cS.y * sdi});
    set(hk::OP_Q, 2, i, cplx{e * dup, -cS.y * sup});
    // Z = -2e A D
    set(hk::OP_Z, 0, i, cplx{-2.0 * e * a * dlo, 0.0});
    set(hk::OP_Z, 2, i, cplx{-2.0 * e * a * dup, 0.0});
  }
  ctx->op_forms = op_forms(coef, n);  // the Phi equation's operators are all three-point
  CK(cudaMemcpyAsync(ctx->d_coef, coef.data(), coef.size() * sizeof(cplx), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_agrid, ctx->agrid.data(), n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return HOPF_OK;
}

// Per-variable operators of the CDF equation (Sec. 5, Eq. cdf-burgers with
// alpha = 0) on u_k = -U + k du, du = 2U/(n-1), k = 0..n-1:
// D centred differences with dF/du = 0 on the two boundary rows (outflow),
// A = diag(u), and in the table's slots
//   A <- P+ = (A D)/(2h) - (gamma/h^2) D,   Q <- P- = -(A D)/(2h) - (gamma/h^2) D,
//   Z <- (2 gamma/h^2) A D,                 K <- A - J (J the trapezoidal
// integral from the lower edge, op_apply), gamma = nu.  Each cyclic pair
// (m, m+1) of the x grid contributes P+_m K_{m+1} + K_m P-_{m+1}.
hopf_status build_ops_cdf(hopf_ctx* ctx) {
  const int n = ctx->p.n, d = ctx->p.d;
  const double U = ctx->L;
  const double du = 2.0 * U / (n - 1);
  const double h = 2.0 * M_PI / d;
  ctx->agrid.assign(n, 0.0);
  for (int k = 0; k < n; ++k) ctx->agrid[k] = -U + k * du;
  ctx->op_forms = 0;  // K integrates along the grid: the untiled apply
  std::vector<cplx> coef((size_t)hk::kNumOps * 3 * n, cplx{0.0, 0.0});
  auto set = [&](int op, int which, int i, double v) { coef[(size_t)op * 3 * n + (size_t)which * n + i] = cplx{v, 0.0}; };
  const double c = ctx->p.nonlinear ? 1.0 / (2.0 * h) : 0.0;
  const double e = ctx->p.nu / (h * h);
  for (int k = 0; k < n; ++k) {
    set(hk::OP_I, 1, k, 1.0);
    set(hk::OP_K, 1, k, ctx->agrid[k]);
    if (k == 0 || k == n - 1) continue;  // outflow rows
    const double u = ctx->agrid[k];
    const double dlo = -1.0 / (2 * du), dup = 1.0 / (2 * du);
    set(hk::OP_A, 0, k, c * u * dlo - e * dlo);
    set(hk::OP_A, 2, k, c * u * dup - e * dup);
    set(hk::OP_Q, 0, k, -c * u * dlo - e * dlo);
    set(hk::OP_Q, 2, k, -c * u * dup - e * dup);
    set(hk::OP_Z, 0, k, 2.0 * e * u * dlo);
    set(hk::OP_Z, 2, k, 2.0 * e * u * dup);
  }
  set(hk::OP_K, 0, 0, du);  // weight of the cumulative integral (op_apply)
  CK(cudaMemcpyAsync(ctx->d_coef, coef.data(), coef.size() * sizeof(cplx), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_agrid, ctx->agrid.data(), n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return HOPF_OK;
}

// MPO block tables: kind 0 first site (row), 1 interior, 2 last site (column).
void mpo_tables_cdf(unsigned char out[3][36]);
void mpo_tables(unsigned char out[3][36], int equation) {
  if (equation == HOPF_EQ_CDF) return mpo_tables_cdf(out);
  for (int k = 0; k < 3; ++k)
    for (int e = 0; e < 36; ++e) out[k][e] = hk::OP_NONE;
  using namespace hk;
  // bond states: 0 idle, 1 A placed (P pending), 2 Q placed (A pending), 3 done,
  // 4 wrap P at site 1 (A pending at d), 5 wrap A at site 1 (Q pending at d)
  const unsigned char first[6] = {OP_I, OP_A, OP_Q, OP_Z, OP_P, OP_A};
  for (int b = 0; b < 6; ++b) out[0][b] = first[b];  // Al = 1, Ar = 6
  auto I6 = [&](int a, int b, unsigned char op) { out[1][a * 6 + b] = op; };
  I6(0, 0, OP_I); I6(0, 1, OP_A); I6(0, 2, OP_Q); I6(0, 3, OP_Z);
  I6(1, 3, OP_P); I6(2, 3, OP_A); I6(3, 3, OP_I); I6(4, 4, OP_I); I6(5, 5, OP_I);
  const unsigned char last[6] = {OP_Z, OP_P, OP_A, OP_I, OP_A, OP_Q};
  for (int a = 0; a < 6; ++a) out[2][a] = last[a];  // Al = 6, Ar = 1
}

// The same bond states for the CDF equation: the first operator of the pair
// type "A then P" is P+ (slot A) and its second K; the pair type "Q then A"
// becomes K then P- (slot Q).
void mpo_tables_cdf(unsigned char out[3][36]) {
  for (int k = 0; k < 3; ++k)
    for (int e = 0; e < 36; ++e) out[k][e] = hk::OP_NONE;
  using namespace hk;
  const unsigned char first[6] = {OP_I, OP_A, OP_K, OP_Z, OP_K, OP_Q};
  for (int b = 0; b < 6; ++b) out[0][b] = first[b];
  auto I6 = [&](int a, int b, unsigned char op) { out[1][a * 6 + b] = op; };
  I6(0, 0, OP_I); I6(0, 1, OP_A); I6(0, 2, OP_K); I6(0, 3, OP_Z);
  I6(1, 3, OP_K); I6(2, 3, OP_Q); I6(3, 3, OP_I); I6(4, 4, OP_I); I6(5, 5, OP_I);
  const unsigned char last[6] = {OP_Z, OP_K, OP_Q, OP_I, OP_A, OP_K};
  for (int a = 0; a < 6; ++a) out[2][a] = last[a];
}

hopf_status coop_reserve(hopf_ctx* ctx, int kcap) {
  if (kcap <= ctx->coop_kcap) return HOPF_OK;
  kcap = std::max(kcap, 64);
  hk::CoopWs& w = ctx->coop;
  dfree(w.pc);
  dfree(w.wfin);
  dfree(w.colnorm);
  dfree(w.colver);
  dfree(w.pairchk);
  w.pc = nullptr;
  w.wfin = nullptr;
  w.colnorm = nullptr;
  w.colver = nullptr;
  w.pairchk = nullptr;
  const int G = hk::dev_info().sm_count;
  w.pc_elems = (size_t)G * 32 * (size_t)(kcap + 64);
  w.wfin_elems = (size_t)32 * (size_t)(kcap + 64);
  CK(dalloc(&w.pc, w.pc_elems));
  CK(dalloc(&w.wfin, w.wfin_elems));
  CK(dalloc(&w.colnorm, (size_t)kcap));
  CK(dalloc(&w.colver, (size_t)kcap));
  CK(dalloc(&w.pairchk, (size_t)kcap * kcap));
  w.jac_cap = kcap;
  ctx->coop_kcap = kcap;
  return HOPF_OK;
}

hopf_status round_reserve(hopf_ctx* ctx, const hopf_tt* t) {
  size_t need = 0;
  for (size_t c : t->core_cap) need = std::max(need, c);
  const int kcap = t->cap_rank;
  RoundWs& w = ctx->rw;
  if (w.elems >= need && w.kcap >= kcap && w.d >= t->d) return HOPF_OK;
  for (cplx* b : w.B) dfree(b);
  dfree(w.W1); dfree(w.tau); dfree(w.T); dfree(w.tau2); dfree(w.T2);
  dfree(w.Rb); dfree(w.Mb); dfree(w.Jb); dfree(w.Ub); dfree(w.Sb);
  dfree(w.sig); dfree(w.perm);
  dfree(w.bd_d); dfree(w.bd_e); dfree(w.bd_tauq); dfree(w.bd_taup); dfree(w.bd_a2);
  dfree(w.bd_info); dfree(w.bd_X); dfree(w.bd_Zs);
  dfree(w.G); dfree(w.G2); dfree(w.bd_rows);
  w = RoundWs{};
  const size_t elems = std::max(need, w.elems);
  const int d = t->d;
  const int K = std::max(kcap, t->n);  // ranks may reach n at the ends
  w.B.assign(d, nullptr);
  for (int c = 0; c < d; ++c) CK(dalloc(&w.B[c], elems));
  CK(dalloc(&w.W1, elems));
  w.tstride = (size_t)(K / 8 + 2) * 32 * 32;
  CK(dalloc(&w.tau, (size_t)d * K));
  CK(dalloc(&w.T, (size_t)d * w.tstride));
  CK(dalloc(&w.tau2, (size_t)K));
  CK(dalloc(&w.T2, w.tstride));
  CK(dalloc(&w.Rb, (size_t)K * K));
  CK(dalloc(&w.Mb, (size_t)K * K));
  CK(dalloc(&w.Jb, (size_t)K * K));
  CK(dalloc(&w.Ub, (size_t)K * K));
  CK(dalloc(&w.Sb, (size_t)K * K));
  CK(dalloc(&w.sig, (size_t)2 * K + 2));
  CK(dalloc(&w.perm, (size_t)K));
  CK(dalloc(&w.bd_d, (size_t)K));
  CK(dalloc(&w.bd_e, (size_t)K));
  CK(dalloc(&w.bd_tauq, (size_t)K));
  CK(dalloc(&w.bd_taup, (size_t)K));
  CK(dalloc(&w.bd_a2, (size_t)2 * K));
  CK(dalloc(&w.bd_info, 4));
  CK(dalloc(&w.bd_X, (size_t)K * K));
  CK(dalloc(&w.bd_Zs, (size_t)2 * K * K));
  w.gstride = hk::qr_tc_gram_elems(K);
  CK(dalloc(&w.G, (size_t)d * w.gstride));
  CK(dalloc(&w.G2, w.gstride));
  CK(dalloc(&w.bd_rows, hk::gebrd_rows_elems(K, hk::dev_info().sm_count)));
  w.elems = elems;
  w.d = d;
  w.kcap = K;
  return coop_reserve(ctx, K);
}

hopf_status tt_alloc(hopf_ctx* ctx, int cap_rank, hopf_tt** out) {
  hopf_tt* t = new (std::nothrow) hopf_tt();
  if (!t) return fail(ctx, HOPF_ENOMEM, "host allocation failed");
  t->ctx = ctx;
  t->d = ctx->p.d;
  t->n = ctx->p.n;
  t->cap_rank = cap_rank;
  t->core_cap.resize(t->d);
  t->cores.assign(t->d, nullptr);
  t->ranks.assign(t->d + 1, 1);
  auto cleanup = [&]() {
    for (cplx* c : t->cores) dfree(c);
    dfree(t->d_ptrs);
    dfree(t->d_ranks);
    delete t;
  };
  for (int k = 0; k < t->d; ++k) {
    const size_t rl = (k == 0) ? 1 : (size_t)cap_rank;
    const size_t rr = (k == t->d - 1) ? 1 : (size_t)cap_rank;
    t->core_cap[k] = rl * t->n * rr;
    cudaError_t e = dalloc(&t->cores[k], t->core_cap[k]);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cleanup();
      return fail(ctx, HOPF_ENOMEM, "tensor allocation (%zu bytes per core): %s",
                  t->core_cap[k] * sizeof(cplx), cudaGetErrorString(e));
    }
  }
  if (dalloc(&t->d_ptrs, t->d) != cudaSuccess || dalloc(&t->d_ranks, t->d + 1) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(ctx, HOPF_ENOMEM, "tensor metadata allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(t->d_ptrs, t->cores.data(), t->d * sizeof(cplx*), cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) {
    cleanup();
    return fail(ctx, HOPF_ECUDA, "%s", cudaGetErrorString(e));
  }
  hk::live_add(1);
  *out = t;
  return HOPF_OK;
}

hopf_status sync_meta(hopf_ctx* ctx, hopf_tt* t) {
  CK(cudaMemcpyAsync(t->d_ranks, t->ranks.data(), (t->d + 1) * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  return HOPF_OK;
}

size_t core_elems(const hopf_tt* t, int k) { return (size_t)t->ranks[k] * t->n * t->ranks[k + 1]; }

hopf_status check_fit(hopf_ctx* ctx, const hopf_tt* t, const std::vector<int>& r) {
  for (int k = 0; k < t->d; ++k)
    if ((size_t)r[k] * t->n * r[k + 1] > t->core_cap[k])
      return fail(ctx, HOPF_EINVAL, "core %d of size %d x %d x %d exceeds the tensor's capacity (max rank %d)",
                  k, r[k], t->n, r[k + 1], t->cap_rank);
  return HOPF_OK;
}

hopf_status read_small(hopf_ctx* ctx, int nint, int ndbl) {
  if (nint) CK(cudaMemcpyAsync(ctx->h_int, ctx->d_int, nint * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (ndbl) CK(cudaMemcpyAsync(ctx->h_dbl, ctx->d_dbl, ndbl * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return HOPF_OK;
}

// Barrier record back to its initial state (count 0, no expiry) with the
// context's wait limit.  Pageable host source: staged before the call returns.
void reset_barrier(hopf_ctx* ctx) {
  const GridBar hb{0u, ctx->wait_limit_us, 0, 0};
  cudaMemcpyAsync(ctx->coop.bar, &hb, sizeof hb, cudaMemcpyHostToDevice, ctx->stream);
}

// read_small and check_barrier with one synchronisation: the barrier record
// comes back in the last four ints of the pinned int buffer.
static_assert(sizeof(GridBar) == 4 * sizeof(int), "barrier record size");
hopf_status read_small_checked(hopf_ctx* ctx, int nint, int ndbl) {
  CK(cudaMemcpyAsync(ctx->h_int + 12, ctx->coop.bar, sizeof(GridBar), cudaMemcpyDeviceToHost, ctx->stream));
  TRY(read_small(ctx, nint, ndbl));
  GridBar hb;
  std::memcpy(&hb, ctx->h_int + 12, sizeof hb);
  if (hb.err) {
    reset_barrier(ctx);
    return fail(ctx, HOPF_ETIMEOUT, "a grid barrier wait expired");
  }
  return HOPF_OK;
}

hopf_status check_barrier(hopf_ctx* ctx) {
  GridBar hb;
  CK(cudaMemcpyAsync(&hb, ctx->coop.bar, sizeof(GridBar), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hb.err) {
    reset_barrier(ctx);
    return fail(ctx, HOPF_ETIMEOUT, "a grid barrier wait expired");
  }
  return HOPF_OK;
}

// Digits of the tensor-core products in mixed precision (about 5e-12 of
// |A||B| per product).
constexpr int kTcDigits = 5;

bool use_tc(const hopf_ctx* ctx, int m, int p) {
  return ctx->p.precision == HOPF_MIXED && ctx->qr_method == HOPF_QR_TENSOR && hk::qr_tc_applies(m, p);
}

hopf_status tc_reserve_bytes(hopf_ctx* ctx, size_t need) {
  if (need <= ctx->tcbytes) return HOPF_OK;
  dfree(ctx->tcbuf);
  dfree(ctx->ev_idx); dfree(ctx->ev_vals); dfree(ctx->ev_out);
  ctx->tcbuf = nullptr;
  ctx->tcbytes = 0;
  CK(hk::dev_alloc(&ctx->tcbuf, need));
  ctx->tcbytes = need;
  return HOPF_OK;
}

hopf_status tc_reserve(hopf_ctx* ctx, int m, int k) { return tc_reserve_bytes(ctx, hk::qr_tc_scratch_bytes(m, k, kTcDigits)); }

// out (a.R x b.R, column-major, ldo) = A B^T of two operand views on the
// tensor cores (digit splits in the context's scratch), profiled as one
// HOPF_K_TC phase with the given FLOP count.
hopf_status tc_product(hopf_ctx* ctx, const hk::TcOperandView& a, const hk::TcOperandView& b, cplx* out, long long ldo,
                       double flops) {
  const int Kc = hk::tc_chunk();
  const size_t ba = (hk::tc_operand_bytes(a.R, a.K, kTcDigits, Kc) + 255) & ~(size_t)255;
  const size_t bb = (hk::tc_operand_bytes(b.R, b.K, kTcDigits, Kc) + 255) & ~(size_t)255;
  const size_t np = hk::tc_part_elems(a.R, b.R, a.K);
  TRY(tc_reserve_bytes(ctx, ba + bb + np * sizeof(cplx) + 256));
  unsigned char* buf = static_cast<unsigned char*>(ctx->tcbuf);
  hk::TcOperand oa, ob;
  const int slot = prof_begin(ctx);
  CK(hk::tc_split(a, kTcDigits, &oa, buf, ctx->stream));
  CK(hk::tc_split(b, kTcDigits, &ob, buf + ba, ctx->stream));
  CK(hk::tc_zgemm(oa, ob, out, ldo, 1.0, 0, np ? reinterpret_cast<cplx*>(buf + ba + bb) : nullptr, np,
                  &ctx->coop.bar->err, ctx->stream));
  prof_end(ctx, slot, HOPF_K_TC, flops, 0.0, np ? 4 : 3);
  return HOPF_OK;
}

// Profile hooks for the phases of the tensor-core QR (PhaseTimer).
int pt_begin(void* user) { return prof_begin(static_cast<hopf_ctx*>(user)); }
void pt_end(void* user, int slot, int cls, double flops, int nl) {
  prof_end(static_cast<hopf_ctx*>(user), slot, cls, flops, 0.0, nl);
}
hk::PhaseTimer phase_timer(hopf_ctx* ctx, int cls_panel) {
  hk::PhaseTimer pt;
  pt.user = ctx;
  pt.begin = pt_begin;
  pt.end = pt_end;
  pt.cls_panel = cls_panel;
  pt.cls_tc = HOPF_K_TC;
  pt.cls_small = HOPF_K_SMALL;
  return pt;
}

// A configuration of the tall-factor QR: how the products run (the
// tensor-core blocked form or the double-float kernel alone) and how many
// CTAs (SMs) the cooperative panel kernel spreads over (0: all the
// context's).  The factorisation and the application of its Q must use
// the same one (the panel layout depends on the CTA count).
struct QrConf {
  int method, ctas;
};

const hopf_ctx::QrTune* tune_find(const hopf_ctx* ctx, int m, int p) {
  for (const auto& t : ctx->tune)
    if (t.m == m && t.p == p) return &t;
  return nullptr;
}

QrConf qr_conf(const hopf_ctx* ctx, int m, int p) {
  if (ctx->autotune)
    if (const hopf_ctx::QrTune* t = tune_find(ctx, m, p)) return QrConf{t->method, t->ctas};
  return QrConf{ctx->qr_method, 0};
}

// Limits the context's cooperative kernels to `ctas` CTAs while in scope.
struct CtaCap {
  hopf_ctx* ctx;
  int saved;
  CtaCap(hopf_ctx* c, int ctas) : ctx(c), saved(c->coop.max_ctas) {
    if (ctas > 0) ctx->coop.max_ctas = ctas;
  }
  ~CtaCap() { ctx->coop.max_ctas = saved; }
};

bool conf_tc(const hopf_ctx* ctx, const QrConf& c, int m, int p) {
  return ctx->p.precision == HOPF_MIXED && c.method == HOPF_QR_TENSOR && hk::qr_tc_applies(m, p);
}

hopf_status qr_factor_conf(hopf_ctx* ctx, const QrConf& c, cplx* A, int lda, int m, int k, cplx* tau, cplx* T,
                           int* nb, cplx* G) {
  CtaCap cap(ctx, c.ctas);
  if (conf_tc(ctx, c, m, std::min(m, k))) {
    TRY(tc_reserve(ctx, m, k));
    *nb = 32;
    CK(hk::geqrf_tc(A, lda, m, k, tau, T, G, ctx->tcbuf, ctx->tcbytes, ctx->coop, kTcDigits, ctx->stream,
                    phase_timer(ctx, HOPF_K_QR)));
    return HOPF_OK;
  }
  LAUNCH(HOPF_K_QR, qr_flops(m, k), 0, 1, hk::geqrf(A, lda, m, k, tau, T, nb, ctx->coop, ctx->stream, MIXED_FLAG));
  return HOPF_OK;
}

// Times every candidate configuration on copies of A (two runs each, the
// faster counts) and records the fastest for the shape (m, min(m, k)).
// Device scratch for the copies and outputs is taken for the duration.
hopf_status tune_qr(hopf_ctx* ctx, const cplx* A, int lda, int m, int k) {
  const int p = std::min(m, k);
  const size_t elems = (size_t)m * k;
  const int all = hk::coop_sms(ctx->coop);
  const QrConf cand[4] = {{HOPF_QR_TENSOR, 0}, {HOPF_QR_TENSOR, std::max(1, all / 2)}, {HOPF_QR_DOUBLEFLOAT, 0},
                          {HOPF_QR_DOUBLEFLOAT, std::max(1, all / 2)}};
  cplx *orig = nullptr, *work = nullptr, *tau = nullptr, *T = nullptr, *G = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hopf_status st = HOPF_OK;
  hopf_ctx::QrTune tu{m, p, ctx->qr_method, 0, {INFINITY, INFINITY, INFINITY, INFINITY}};
  // the candidates' launches are not part of the caller's profile
  const bool prof_was = ctx->prof_on;
  const hopf_profile prof_saved = ctx->prof;
  ctx->prof_on = false;
  auto run = [&]() -> hopf_status {
    CK(dalloc(&orig, elems));
    CK(dalloc(&work, elems));
    CK(dalloc(&tau, (size_t)k));
    CK(dalloc(&T, (size_t)((k + 31) / 32) * 32 * 32));
    CK(dalloc(&G, hk::qr_tc_gram_elems(k)));
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaMemcpy2DAsync(orig, (size_t)m * sizeof(cplx), A, (size_t)lda * sizeof(cplx), (size_t)m * sizeof(cplx), k,
                         cudaMemcpyDeviceToDevice, ctx->stream));
    for (int i = 0; i < 4; ++i) {
      if (i % 2 == 1 && cand[i].ctas >= all) continue;  // no smaller share to try
      float best = INFINITY;
      for (int rep = 0; rep < 2; ++rep) {
        CK(cudaMemcpyAsync(work, orig, elems * sizeof(cplx), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaEventRecord(e0, ctx->stream));
        int nb = 32;
        const hopf_status r = qr_factor_conf(ctx, cand[i], work, m, m, k, tau, T, &nb, G);
        if (r != HOPF_OK) return r;
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        TRY(check_barrier(ctx));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
      }
      tu.ms[i] = best;
    }
    int bi = -1;
    for (int i = 0; i < 4; ++i)
      if (std::isfinite(tu.ms[i]) && (bi < 0 || tu.ms[i] < tu.ms[bi])) bi = i;
    if (bi >= 0) {
      tu.method = cand[bi].method;
      tu.ctas = cand[bi].ctas;
    }
    return HOPF_OK;
  };
  st = run();
  ctx->prof_on = prof_was;
  ctx->prof = prof_saved;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(ctx->stream);
  dfree(orig);
  dfree(work);
  dfree(tau);
  dfree(T);
  dfree(G);
  if (st == HOPF_OK) ctx->tune.push_back(tu);
  return st;
}

// Householder QR of the m x k matrix A (lda) in place: in mixed precision
// and for tall factors the blocked form with tensor-core products (G
// receives its panel Grams), otherwise the cooperative kernel alone; with
// autotuning on, the configuration measured fastest for the shape.
hopf_status qr_factor(hopf_ctx* ctx, cplx* A, int lda, int m, int k, cplx* tau, cplx* T, int* nb, cplx* G) {
  const int p = std::min(m, k);
  if (ctx->autotune && ctx->p.precision == HOPF_MIXED && hk::qr_tc_applies(m, p) && !tune_find(ctx, m, p))
    TRY(tune_qr(ctx, A, lda, m, k));
  return qr_factor_conf(ctx, qr_conf(ctx, m, p), A, lda, m, k, tau, T, nb, G);
}

// C <- Q C with the Q of qr_factor (same m and p = min(m, k), same
// configuration).
hopf_status qr_apply(hopf_ctx* ctx, const cplx* A, int lda, int m, int p, const cplx* tau, const cplx* T, int nb,
                     const cplx* G, cplx* C, int ldc, int q) {
  const QrConf c = qr_conf(ctx, m, p);
  CtaCap cap(ctx, c.ctas);
  if (conf_tc(ctx, c, m, p)) {
    TRY(tc_reserve(ctx, m, q));
    CK(hk::ormqr_tc(A, lda, m, p, tau, G, C, ldc, q, ctx->tcbuf, ctx->tcbytes, &ctx->coop.bar->err, kTcDigits,
                    ctx->stream, phase_timer(ctx, HOPF_K_APPLYQ)));
    return HOPF_OK;
  }
  LAUNCH(HOPF_K_APPLYQ, applyq_flops(m, q, p), 0, 1,
         hk::ormqr(A, lda, m, p, tau, T, nb, C, ldc, q, ctx->coop, ctx->stream, MIXED_FLAG));
  return HOPF_OK;
}

// Persistent device staging of point / moment evaluation, grown on demand
// (no per-call allocation once large enough).
hopf_status ev_reserve(hopf_ctx* ctx, size_t nidx, size_t nvals, size_t nout) {
  if (nidx > ctx->ev_idx_cap) {
    dfree(ctx->ev_idx);
    ctx->ev_idx = nullptr;
    ctx->ev_idx_cap = 0;
    CK(dalloc(&ctx->ev_idx, nidx));
    ctx->ev_idx_cap = nidx;
  }
  if (nvals > ctx->ev_vals_cap) {
    dfree(ctx->ev_vals);
    ctx->ev_vals = nullptr;
    ctx->ev_vals_cap = 0;
    CK(dalloc(&ctx->ev_vals, nvals));
    ctx->ev_vals_cap = nvals;
  }
  if (nout > ctx->ev_out_cap) {
    dfree(ctx->ev_out);
    ctx->ev_out = nullptr;
    ctx->ev_out_cap = 0;
    CK(dalloc(&ctx->ev_out, nout));
    ctx->ev_out_cap = nout;
  }
  return HOPF_OK;
}

// Phase 1 of the rounding: right-to-left Householder LQ sweep (App. A,
// Alg. 1 mirrored).  Reads the cores of t (unchanged), leaves B_c = the
// factored H(Y_c)^H with its reflectors for c >= 1 and B_0 = V(Y_0 L_1)
// explicitly; p[c] = rank after orthogonalisation at bond c.  Returns
// ||f||_F^2 in ctx->d_dbl[0].
hopf_status orth_sweep(hopf_ctx* ctx, const hopf_tt* t, std::vector<int>& p, std::vector<int>& nbv) {
  RoundWs& w = ctx->rw;
  const int d = t->d, n = t->n;
  const std::vector<int>& r = t->ranks;
  p.assign(d + 1, 1);
  nbv.assign(d, 32);
  // B_{d-1} = H(X_{d-1})^H: X_{d-1} is r[d-1] x n (x 1)
  LAUNCH(HOPF_K_SUM, 0, 32.0 * r[d - 1] * n, 1, hk::conj_transpose(t->cores[d - 1], r[d - 1], r[d - 1], n, w.B[d - 1], n, ctx->stream));
  for (int c = d - 1; c >= 1; --c) {
    const int m = n * p[c + 1], k = r[c];
    TRY(qr_factor(ctx, w.B[c], m, m, k, w.tau + (size_t)c * w.kcap, w.T + (size_t)c * w.tstride, &nbv[c],
                  w.G + (size_t)c * w.gstride));
    p[c] = std::min(m, k);
    // merge L_c = R_c^H into core c-1
    const int rl = r[c - 1];
    if (c - 1 >= 1 && use_tc(ctx, rl * n, 64)) {
      // on the tensor cores: C = X_{c-1} R^H into the scratch W1
      // (column-major), then H(Y)^H into the next factor's buffer
      TRY(tc_product(ctx, hk::TcOperandView{t->cores[c - 1], 1, (long long)rl * n, rl * n, k, 0, 0, 0},
                     hk::TcOperandView{w.B[c], 1, m, p[c], k, 1, 1, 0}, w.W1, (long long)rl * n,
                     arh_flops((double)rl * n, k, p[c])));
      LAUNCH(HOPF_K_SUM, 0, 32.0 * rl * n * p[c], 1,
             hk::conj_transpose(w.W1, rl, rl, n * p[c], w.B[c - 1], n * p[c], ctx->stream));
    } else if (c - 1 >= 1) {
      LAUNCH(HOPF_K_GEMM, arh_flops((double)rl * n, k, p[c]), 0, 1, hk::gemm_a_rh(t->cores[c - 1], rl * n, rl * n, k, w.B[c], m, p[c], w.B[c - 1], n * p[c], 1, rl, n, ctx->stream, MIXED_FLAG));
    } else {
      LAUNCH(HOPF_K_GEMM, arh_flops(n, k, p[1]), 0, 1, hk::gemm_a_rh(t->cores[0], n, n, k, w.B[1], m, p[1], w.B[0], n, 0, 1, n, ctx->stream, MIXED_FLAG));
    }
  }
  LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::frob2(w.B[0], n, n, p[1], ctx->d_dbl, ctx->stream));
  return HOPF_OK;
}

// Phase 2 of the rounding (left-to-right truncated SVDs, App. A Alg. 2
// mirrored, factor-then-SVD as in Alg. 4), after a phase-1 sweep left the
// factored flattenings in the workspace.  Writes the new cores into t.
hopf_status phase2(hopf_ctx* ctx, hopf_tt* t, const std::vector<int>& p, const std::vector<int>& nbv,
                   double tol, int cap, const int* forced, double* disc_out, bool* capped) {
  const int d = t->d, n = t->n;
  RoundWs& w = ctx->rw;
  TRY(read_small_checked(ctx, 0, 1));
  const double nrm2 = ctx->h_dbl[0];
  if (!std::isfinite(nrm2)) return fail(ctx, HOPF_ENUMERIC, "non-finite norm in rounding");
  const double eps_hat = tol * std::sqrt(nrm2) / std::sqrt((double)(d - 1));
  ctx->h_dbl[1] = eps_hat;
  CK(cudaMemcpyAsync(ctx->d_dbl + 1, ctx->h_dbl + 1, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));

  std::vector<int> rho(d + 1, 1);
  double disc2 = 0.0;
  bool cap_hit = false;
  for (int c = 0; c <= d - 2; ++c) {
    cplx* Z;
    const int Mrows = rho[c] * n, cols = p[c + 1];
    if (c == 0) {
      Z = w.B[0];
    } else {
      const int mc = n * p[c + 1];
      LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::init_sh_pad(w.Sb, rho[c], rho[c], p[c], t->cores[c], mc, mc, ctx->stream));
      TRY(qr_apply(ctx, w.B[c], mc, mc, p[c], w.tau + (size_t)c * w.kcap, w.T + (size_t)c * w.tstride, nbv[c],
                   w.G + (size_t)c * w.gstride, t->cores[c], mc, rho[c]));
      LAUNCH(HOPF_K_SUM, 0, 32.0 * mc * rho[c], 1, hk::conj_transpose(t->cores[c], mc, mc, rho[c], w.W1, rho[c], ctx->stream));
      Z = w.W1;
    }
    int nb2 = 32;
    TRY(qr_factor(ctx, Z, Mrows, Mrows, cols, w.tau2, w.T2, &nb2, w.G2));
    const int pp = std::min(Mrows, cols);
    LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::extract_r(Z, Mrows, pp, cols, w.Rb, pp, ctx->stream));
    const int forced_c = forced ? forced[c + 1] : 0;
    const bool case1 = (pp >= cols);
    const int nsv = case1 ? cols : pp;
    if (forced && (forced_c < 1 || forced_c > nsv))
      return fail(ctx, HOPF_EINVAL, "forced rank %d at bond %d outside [1, %d]", forced_c, c + 1, nsv);
    // Square factors: bidiagonalisation, bisection and inverse iteration.
    // A wide factor (pp < cols) goes the same way through its LQ:
    // R = L Q' with L = R_f^H, R^H = Q_h R_f, so R and the square L share
    // their singular values and left singular vectors, which is all the
    // truncation uses (the projection below is S = U^H R).  The LQ is FP64
    // like the SVD, on the reflector slot c that this step no longer needs.
    const bool use_bd = ctx->svd_method != HOPF_SVD_JACOBI && hk::gebrd_fits(pp, ctx->coop, true);
    if (use_bd) {
      if (case1) {
        CK(cudaMemcpyAsync(w.Mb, w.Rb, (size_t)pp * cols * sizeof(cplx), cudaMemcpyDeviceToDevice, ctx->stream));
      } else {
        int nbl = 32;
        LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::conj_transpose(w.Rb, pp, pp, cols, w.Mb, cols, ctx->stream));
        LAUNCH(HOPF_K_SVD, qr_flops(cols, pp), 0, 1, hk::geqrf(w.Mb, cols, cols, pp, w.tau + (size_t)c * w.kcap, w.T + (size_t)c * w.tstride, &nbl, ctx->coop, ctx->stream, 0));
        LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::extract_r(w.Mb, cols, pp, pp, w.Jb, pp, ctx->stream));
        LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::conj_transpose(w.Jb, pp, pp, pp, w.Mb, pp, ctx->stream));
      }
      LAUNCH(HOPF_K_SVD, gebrd_flops(pp), 0, 1, hk::gebrd(w.Mb, pp, pp, w.bd_d, w.bd_e, w.bd_tauq, w.bd_taup, ctx->coop, ctx->stream, w.bd_rows));
      LAUNCH(HOPF_K_SVD, 0, 0, 2, hk::bd_sigma(w.bd_d, w.bd_e, pp, w.bd_a2, w.bd_info, w.sig, ctx->stream));
      LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::bd_rank(w.sig, pp, ctx->d_dbl + 1, cap, forced_c, ctx->d_int, ctx->d_dbl + 2, w.sig + pp, ctx->stream));
      TRY(read_small_checked(ctx, 3, 5));
      ctx->prof.svd_count += 1;
    }
    // Jacobi leaves out pairs far below the truncation tolerance (theta);
    // if the rank kept reaches below theta, finish the SVD exactly so that
    // every kept singular vector is orthogonal to all others.
    for (int pass = 0; pass < 2 && !use_bd; ++pass) {
      const double* eh = (pass == 0) ? ctx->d_dbl + 1 : nullptr;
      if (case1) {
        if (pass == 0)
          CK(cudaMemcpyAsync(w.Mb, w.Rb, (size_t)pp * cols * sizeof(cplx), cudaMemcpyDeviceToDevice, ctx->stream));
        LAUNCH(HOPF_K_SVD, 0, 0, 1, hk::jacobi_svd(w.Mb, pp, pp, cols, nullptr, 1, 0, eh, 0, ctx->coop, ctx->stream));
        LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::rank_select(w.Mb, pp, pp, cols, ctx->d_dbl + 1, cap, forced_c, w.sig, w.perm, ctx->d_int, ctx->d_dbl + 2, ctx->stream));
      } else {
        if (pass == 0) LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::conj_transpose(w.Rb, pp, pp, cols, w.Mb, cols, ctx->stream));
        LAUNCH(HOPF_K_SVD, 0, 0, pass == 0 ? 2 : 1,
               hk::jacobi_svd(w.Mb, cols, cols, pp, w.Jb, pp, 1, eh, pass == 0, ctx->coop, ctx->stream));
        LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::rank_select(w.Mb, cols, cols, pp, ctx->d_dbl + 1, cap, forced_c, w.sig, w.perm, ctx->d_int, ctx->d_dbl + 2, ctx->stream));
      }
      CK(cudaMemcpyAsync(ctx->d_int + 2, ctx->coop.counters + 63, sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
      TRY(read_small_checked(ctx, 3, 5));
      if (ctx->h_int[2] < 0) return fail(ctx, HOPF_ENUMERIC, "Jacobi SVD did not converge at bond %d", c + 1);
      ctx->prof.svd_count += 1;
      ctx->prof.svd_sweeps += ctx->h_int[2];
      const double theta = std::max(1e-3 * eps_hat, 64.0 * 2.220446049250313e-16 * std::sqrt(ctx->h_dbl[4]));
      if (pass == 0 && !(ctx->h_dbl[3] > theta)) continue;  // smallest kept sigma below theta
      break;
    }
    const int rnew = ctx->h_int[0];
    const int rtol = ctx->h_int[1];
    const double delta = ctx->h_dbl[2];
    if (!std::isfinite(delta)) return fail(ctx, HOPF_ENUMERIC, "non-finite singular values at bond %d", c + 1);
    if (!forced && rtol > cap) cap_hit = true;
    // the new core must fit the tensor's capacity
    if ((size_t)rho[c] * n * rnew > t->core_cap[c])
      return fail(ctx, HOPF_EINVAL, "rank %d at bond %d exceeds the tensor's capacity", rnew, c + 1);
    rho[c + 1] = rnew;
    disc2 += delta * delta;
    // new core c = Q [U_rho; 0]
    if (use_bd) {
      const int kt = std::min(ctx->h_int[2], rnew);
      LAUNCH(HOPF_K_SVD, 0, 0, (kt > 0) + (kt < rnew), hk::bd_vectors(w.bd_d, w.bd_e, pp, w.bd_info, w.sig, kt, rnew, w.bd_X, pp, w.bd_Zs, ctx->stream));
      LAUNCH(HOPF_K_SVD, 0, 0, 1, hk::bd_back(w.Mb, pp, w.bd_tauq, pp, w.bd_X, pp, rnew, w.Ub, pp, t->cores[c], Mrows, Mrows, ctx->stream));
    } else if (case1) {
      LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::gather_u(w.Mb, pp, pp, w.perm, w.sig, 1, rnew, t->cores[c], Mrows, Mrows, w.Ub, pp, ctx->stream));
    } else {
      LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::gather_u(w.Jb, pp, pp, w.perm, w.sig, 0, rnew, t->cores[c], Mrows, Mrows, w.Ub, pp, ctx->stream));
    }
    TRY(qr_apply(ctx, Z, Mrows, Mrows, pp, w.tau2, w.T2, nb2, w.G2, t->cores[c], Mrows, rnew));
    // S = U_rho^H R (rho x cols)
    if (use_tc(ctx, 4096, pp)) {
      TRY(tc_product(ctx, hk::TcOperandView{w.Ub, pp, 1, rnew, pp, 1, 0, 0}, hk::TcOperandView{w.Rb, pp, 1, cols, pp, 0, 0, 0},
                     w.Sb, rnew, 8.0 * rnew * pp * cols));
    } else {
      LAUNCH(HOPF_K_GEMM, 8.0 * rnew * pp * cols, 0, 1, hk::gemm_uh_r(w.Ub, pp, rnew, pp, w.Rb, pp, cols, w.Sb, rnew, ctx->stream));
    }
  }
  // last core: C = Q_{B,d-1} [S^H; 0] (n x rho), core = C^H
  {
    const int c = d - 1;
    LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::init_sh_pad(w.Sb, rho[c], rho[c], p[c], w.W1, n, n, ctx->stream));
    TRY(qr_apply(ctx, w.B[c], n, n, p[c], w.tau + (size_t)c * w.kcap, w.T + (size_t)c * w.tstride, nbv[c],
                 w.G + (size_t)c * w.gstride, w.W1, n, rho[c]));
    LAUNCH(HOPF_K_SUM, 0, 32.0 * n * rho[c], 1, hk::conj_transpose(w.W1, n, n, rho[c], t->cores[c], rho[c], ctx->stream));
  }
  rho[d] = 1;
  t->ranks = rho;
  TRY(sync_meta(ctx, t));
  if (disc_out) *disc_out = std::sqrt(disc2);
  if (capped) *capped = cap_hit;
  return HOPF_OK;
}

hopf_status round_impl(hopf_ctx* ctx, hopf_tt* t, double tol, int cap, const int* forced,
                       double* disc_out, bool* capped) {
  TRY(round_reserve(ctx, t));
  std::vector<int> p, nbv;
  TRY(orth_sweep(ctx, t, p, nbv));
  return phase2(ctx, t, p, nbv, tol, cap, forced, disc_out, capped);
}

// FLOPs of C = A (columns coff..coff+K of R)^H with R upper trapezoidal.
double rblk_flops(double M, int K, int N, int coff) {
  double s = 0.0;
  for (int t = 0; t < K; ++t) s += std::min(N, coff + t + 1);
  return 8.0 * M * s;
}

// Phase 1 for the rounding of Y = G X without forming Y: the LQ factor L_c
// of core c is merged into core c-1 as
//   Y'_{c-1}(alpha, i, m, q) = sum_beta W[alpha, beta] along m of
//                              (X_{c-1} x_3 L_c[beta-block])(i, m, q),
// i.e. six r x r x p products (one per MPO bond state beta) and one stencil
// pass, instead of one (6r) x (6r) x p product on the materialised apply.
// The stencil pass writes the next QR's input layout directly.
hopf_status orth_sweep_apply(hopf_ctx* ctx, const hopf_tt* X, std::vector<int>& p, std::vector<int>& nbv) {
  RoundWs& w = ctx->rw;
  const int d = X->d, n = X->n;
  const std::vector<int>& r = X->ranks;
  const hk::OpTable ops{ctx->d_coef, n, ctx->op_forms};
  p.assign(d + 1, 1);
  nbv.assign(d, 32);
  {
    const double rd = (double)r[d - 1] * n;
    LAUNCH(HOPF_K_APPLY, 0, 16.0 * rd * 7.0, 1,
           hk::stencil_combine(X->cores[d - 1], r[d - 1], n, 1, 1, 6, 1, ctx->d_blocks + 72, ops, w.B[d - 1], 1, n,
                               ctx->stream));
  }
  for (int c = d - 1; c >= 1; --c) {
    const int m = n * p[c + 1], k = 6 * r[c];
    TRY(qr_factor(ctx, w.B[c], m, m, k, w.tau + (size_t)c * w.kcap, w.T + (size_t)c * w.tstride, &nbv[c],
                  w.G + (size_t)c * w.gstride));
    p[c] = std::min(m, k);
    const int rl = r[c - 1];
    const size_t blk = (size_t)rl * n * p[c];
    if (use_tc(ctx, rl * n, 64)) {
      // the six products on the tensor cores: X_{c-1} (rl n x r) split once,
      // each block of R^H (conjugated, upper trapezoid) split in turn
      const int Kc = hk::tc_chunk();
      const size_t ba = (hk::tc_operand_bytes(rl * n, r[c], kTcDigits, Kc) + 255) & ~(size_t)255;
      const size_t bb = (hk::tc_operand_bytes(p[c], r[c], kTcDigits, Kc) + 255) & ~(size_t)255;
      const size_t np = hk::tc_part_elems(rl * n, p[c], r[c]);
      TRY(tc_reserve_bytes(ctx, ba + bb + np * sizeof(cplx) + 256));
      unsigned char* buf = static_cast<unsigned char*>(ctx->tcbuf);
      cplx* part = np ? reinterpret_cast<cplx*>(buf + ba + bb) : nullptr;
      hk::TcOperand oX, oR;
      int slot = prof_begin(ctx);
      CK(hk::tc_split(hk::TcOperandView{X->cores[c - 1], 1, (long long)rl * n, rl * n, r[c], 0, 0, 0}, kTcDigits, &oX, buf,
                      ctx->stream));
      prof_end(ctx, slot, HOPF_K_TC, 0.0, 0.0, 1);
      for (int be = 0; be < 6; ++be) {
        slot = prof_begin(ctx);
        CK(hk::tc_split(hk::TcOperandView{w.B[c] + (size_t)m * be * r[c], 1, m, p[c], r[c], 1, 1, be * r[c]}, kTcDigits,
                        &oR, buf + ba, ctx->stream));
        CK(hk::tc_zgemm(oX, oR, w.W1 + be * blk, rl * n, 1.0, 0, part, np, &ctx->coop.bar->err, ctx->stream));
        prof_end(ctx, slot, HOPF_K_TC, rblk_flops((double)rl * n, r[c], p[c], be * r[c]), 0.0, np ? 3 : 2);
      }
    } else {
      for (int be = 0; be < 6; ++be) {
        LAUNCH(HOPF_K_GEMM, rblk_flops((double)rl * n, r[c], p[c], be * r[c]), 0, 1,
               hk::gemm_a_rblk_h(X->cores[c - 1], rl * n, rl * n, r[c], w.B[c], m, be * r[c], p[c], w.W1 + be * blk,
                                 rl * n, ctx->stream, MIXED_FLAG));
      }
    }
    const int Al = (c - 1 == 0) ? 1 : 6;
    const int kind = (c - 1 == 0) ? 0 : 1;
    LAUNCH(HOPF_K_APPLY, 0, 16.0 * (double)blk * (6.0 + Al), 1,
           hk::stencil_combine(w.W1, rl, n, p[c], 6, Al, 6, ctx->d_blocks + 36 * kind, ops, w.B[c - 1],
                               (c - 1 == 0) ? 0 : 1, n * p[c], ctx->stream));
  }
  LAUNCH(HOPF_K_SMALL, 0, 0, 1, hk::frob2(w.B[0], n, n, p[1], ctx->d_dbl, ctx->stream));
  return HOPF_OK;
}

// out <- T[G X] (hopf_apply_op followed by tt_round, without the apply).
hopf_status round_apply_impl(hopf_ctx* ctx, const hopf_tt* X, hopf_tt* out, double tol, int cap,
                             const int* forced, double* disc_out, bool* capped) {
  std::vector<int> r(X->d + 1, 1);
  for (int k = 1; k < X->d; ++k) r[k] = 6 * X->ranks[k];
  TRY(check_fit(ctx, out, r));
  TRY(round_reserve(ctx, out));
  std::vector<int> p, nbv;
  TRY(orth_sweep_apply(ctx, X, p, nbv));
  return phase2(ctx, out, p, nbv, tol, cap, forced, disc_out, capped);
}

hopf_status apply_impl(hopf_ctx* ctx, const hopf_tt* in, hopf_tt* out) {
  const int d = in->d, n = in->n;
  std::vector<int> r(d + 1, 1);
  for (int k = 1; k < d; ++k) r[k] = 6 * in->ranks[k];
  TRY(check_fit(ctx, out, r));
  hk::OpTable ops{ctx->d_coef, n};
  for (int k = 0; k < d; ++k) {
    const int kind = (k == 0) ? 0 : (k == d - 1 ? 2 : 1);
    const int Al = (k == 0) ? 1 : 6, Ar = (k == d - 1) ? 1 : 6;
    const double rd = (double)in->ranks[k] * n * in->ranks[k + 1];
    LAUNCH(HOPF_K_APPLY, 0, 16.0 * rd * (1.0 + (double)Al * Ar), 1,
           hk::apply_core(in->cores[k], in->ranks[k], n, in->ranks[k + 1], out->cores[k], Al, Ar,
                          ctx->d_blocks + 36 * kind, ops, ctx->stream));
  }
  out->ranks = r;
  return sync_meta(ctx, out);
}

hopf_status sum_impl(hopf_ctx* ctx, int nterms, const hopf_tt* const* terms, const double* coef,
                     hopf_tt* out) {
  const int d = out->d, n = out->n;
  if (nterms < 1 || nterms > 16) return fail(ctx, HOPF_EINVAL, "tt_sum takes 1..16 terms");
  std::vector<int> r(d + 1, 1);
  for (int t = 0; t < nterms; ++t) {
    if (!terms[t] || terms[t]->d != d || terms[t]->n != n) return fail(ctx, HOPF_EINVAL, "tt_sum: term %d has another shape", t);
    if (terms[t] == out) return fail(ctx, HOPF_EINVAL, "tt_sum: output aliases term %d", t);
  }
  for (int k = 1; k < d; ++k) {
    int s = 0;
    for (int t = 0; t < nterms; ++t) s += terms[t]->ranks[k];
    r[k] = s;
  }
  TRY(check_fit(ctx, out, r));
  std::vector<hk::SumTerm> host((size_t)nterms * d);
  for (int k = 0; k < d; ++k)
    for (int t = 0; t < nterms; ++t) {
      hk::SumTerm& s = host[(size_t)k * nterms + t];
      s.p = terms[t]->cores[k];
      s.ra = terms[t]->ranks[k];
      s.rc = terms[t]->ranks[k + 1];
      s.coef = cplx{coef[2 * t], coef[2 * t + 1]};
    }
  // pageable source: the copy is staged before the call returns, and stream
  // order keeps earlier sums' kernels ahead of this overwrite
  hk::SumTerm* dt = ctx->d_terms;
  CK(cudaMemcpyAsync(dt, host.data(), host.size() * sizeof(hk::SumTerm), cudaMemcpyHostToDevice, ctx->stream));
  for (int k = 0; k < d; ++k) {
    const int kind = (k == 0) ? 0 : (k == d - 1 ? 2 : 1);
    double in_elems = 0.0;
    for (int t = 0; t < nterms; ++t) in_elems += (double)terms[t]->ranks[k] * n * terms[t]->ranks[k + 1];
    LAUNCH(HOPF_K_SUM, 0, 16.0 * (in_elems + (double)r[k] * n * r[k + 1]), 1,
           hk::sum_core(dt + (size_t)k * nterms, nterms, kind, n, out->cores[k], r[k], r[k + 1], ctx->stream));
  }
  out->ranks = r;
  return sync_meta(ctx, out);
}

hopf_status copy_impl(hopf_ctx* ctx, const hopf_tt* src, hopf_tt* dst) {
  TRY(check_fit(ctx, dst, src->ranks));
  for (int k = 0; k < src->d; ++k)
    CK(cudaMemcpyAsync(dst->cores[k], src->cores[k], core_elems(src, k) * sizeof(cplx), cudaMemcpyDeviceToDevice, ctx->stream));
  dst->ranks = src->ranks;
  return sync_meta(ctx, dst);
}

// Step workspace: `big` takes an operator output (6 x the input rank; the
// midpoint scheme applies the operator to an untruncated sum of rank 2 cap),
// `ytmp` the stage inputs (rank 2 cap for the midpoint's sum).
hopf_status ensure_step_ws(hopf_ctx* ctx, int cap, int scheme) {
  const int mult = (scheme == HOPF_MIDPOINT) ? 2 : 1;
  if (ctx->big && ctx->big->cap_rank >= 6 * mult * cap && ctx->kst[0]->cap_rank >= cap &&
      ctx->ytmp->cap_rank >= mult * cap)
    return HOPF_OK;
  if (ctx->big) tt_free(ctx->big);
  for (auto& k : ctx->kst)
    if (k) tt_free(k);
  if (ctx->ytmp) tt_free(ctx->ytmp);
  ctx->big = ctx->ytmp = nullptr;
  for (auto& k : ctx->kst) k = nullptr;
  TRY(tt_alloc(ctx, 6 * mult * cap, &ctx->big));
  for (auto& k : ctx->kst) TRY(tt_alloc(ctx, cap, &k));
  TRY(tt_alloc(ctx, mult * cap, &ctx->ytmp));
  return HOPF_OK;
}

std::vector<double> gauss_legendre01(int q) {
  // nodes by Newton's method on P_q, then mapped to [0, 1]
  std::vector<double> out(2 * q);
  for (int i = 0; i < q; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= q; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= q; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = q * (x * p1 - p0) / (x * x - 1.0);
    out[i] = 0.5 * (x + 1.0);
    out[q + i] = 1.0 / ((1.0 - x * x) * dp * dp);  // weight on [-1,1] halved
  }
  return out;
}

// ---- TT-cross construction of a correlated Gaussian initial state ------------
// Index sets are tuples of grid indices (row-major, one tuple per rank
// index).  A left-to-right sweep over the modes in `order` builds, at each
// bond, the next left set from the pivots of the fiber matrix and, when
// `cores` is set, the interpolating core.  The right-to-left sweeps are
// left-to-right sweeps of the mode-reversed problem.
struct CrossBufs {
  cplx* A = nullptr;     // fiber matrix, cap n x cap
  cplx* W = nullptr;     // pivoting copy
  cplx* Gw = nullptr;    // cap x cap
  cplx* Gi = nullptr;    // cap x cap
  int* il = nullptr;     // cap x d
  int* jr = nullptr;     // cap x d
  int* piv = nullptr;    // rows[cap], cols[cap], count
  int* seq = nullptr;    // 0..cap-1
  double* mc = nullptr;  // m (d), C (d x d)
  cplx* Q = nullptr;     // chosen columns, then their orthonormal basis (cap n x cap)
  cplx* tau = nullptr;   // cap
  cplx* T = nullptr;     // panel Grams of the QR
  void release() {
    dfree(A); dfree(W); dfree(Gw); dfree(Gi); dfree(il); dfree(jr); dfree(piv); dfree(mc);
    dfree(seq); dfree(Q); dfree(tau); dfree(T);
  }
};

hopf_status cross_sweep(hopf_ctx* ctx, CrossBufs& B, int cap, const std::vector<double>& m,
                        const std::vector<double>& C, const std::vector<std::vector<int>>& R,
                        std::vector<std::vector<int>>& L, hopf_tt* cores) {
  const int d = ctx->p.d, n = ctx->p.n;
  CK(cudaMemcpyAsync(B.mc, m.data(), d * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(B.mc + d, C.data(), (size_t)d * d * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  L.assign(d + 1, {});
  std::vector<int> ranks(d + 1, 1);
  std::vector<int> hp(2 * cap + 1);
  for (int k = 0; k < d; ++k) {
    const int rl = (k == 0) ? 1 : (int)(L[k].size() / k);
    const int kr = d - k - 1;
    const int rr = (k == d - 1) ? 1 : (int)(R[k + 1].size() / kr);
    if (k > 0) CK(cudaMemcpyAsync(B.il, L[k].data(), L[k].size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    if (kr > 0) CK(cudaMemcpyAsync(B.jr, R[k + 1].data(), R[k + 1].size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    const int M = rl * n;
    if (rl < 1 || rl > cap || rr < 1 || rr > cap)
      return fail(ctx, HOPF_EINVAL, "cross: index set of size %d x %d at mode %d outside [1, %d]", rl, rr, k, cap);
    if (k == d - 1) {
      if (cores) CK(hk::gauss_fibers(ctx->d_agrid, n, d, B.mc, B.mc + d, B.il, rl, k, B.jr, 1, cores->cores[k], ctx->stream));
      ranks[k] = rl;
      break;
    }
    CK(hk::gauss_fibers(ctx->d_agrid, n, d, B.mc, B.mc + d, B.il, rl, k, B.jr, rr, B.A, ctx->stream));
    CK(hk::cross_pivots(B.A, M, rr, 1e-14, B.W, B.piv, B.piv + cap, B.piv + 2 * cap, ctx->coop, ctx->stream));
    CK(cudaMemcpyAsync(hp.data(), B.piv, (2 * cap + 1) * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    TRY(check_barrier(ctx));
    const int cnt = hp[2 * cap];
    if (cnt < 1) return fail(ctx, HOPF_ENUMERIC, "cross: no pivot at bond %d", k + 1);
    if (cores) {
      // core = A[:, cols] A[rows, cols]^-1, formed stably as Q Q[rows, :]^-1
      // with Q an orthonormal basis of A[:, cols] (the same matrix: the
      // triangular factor cancels), so near-singular pivots cost no accuracy
      if ((size_t)M * cnt > cores->core_cap[k]) return fail(ctx, HOPF_EINVAL, "cross: core %d exceeds capacity", k);
      CK(hk::cross_gather(B.A, M, B.piv + cap, cnt, B.Q, B.W, B.seq, ctx->stream));
      int nb = 32;
      CK(hk::geqrf(B.Q, M, M, cnt, B.tau, B.T, &nb, ctx->coop, ctx->stream, 0));
      CK(hk::ormqr(B.Q, M, M, cnt, B.tau, B.T, nb, B.W, M, cnt, ctx->coop, ctx->stream, 0));
      TRY(check_barrier(ctx));
      CK(hk::cross_core(B.W, M, B.piv, B.seq, cnt, B.Gw, B.Gi, cores->cores[k], ctx->stream));
    }
    ranks[k] = rl;
    // next left set: (L[k][alpha], i) for each pivot row alpha + rl i
    std::vector<int> nl((size_t)cnt * (k + 1));
    for (int b = 0; b < cnt; ++b) {
      const int row = hp[b], alpha = row % rl, i = row / rl;
      for (int t = 0; t < k; ++t) nl[(size_t)b * (k + 1) + t] = L[k][(size_t)alpha * k + t];
      nl[(size_t)b * (k + 1) + k] = i;
    }
    L[k + 1] = std::move(nl);
  }
  if (cores) {
    std::vector<int> r(d + 1, 1);
    for (int k = 1; k < d; ++k) r[k] = (int)(L[k].size() / k);
    cores->ranks = r;
    TRY(sync_meta(ctx, cores));
  }
  return HOPF_OK;
}

// reverses the mode order of tuple sets: set over modes k..d-1 of the
// forward problem <-> set over modes 0..d-k-1 of the reversed problem
std::vector<std::vector<int>> cross_mirror(const std::vector<std::vector<int>>& S, int d, bool from_left) {
  std::vector<std::vector<int>> out(d + 1);
  for (int k = 1; k < d; ++k) {
    const int len = from_left ? k : d - k;  // tuple length in S at bond k
    const std::vector<int>& src = S[k];
    if (src.empty() || len == 0) continue;
    const int cnt = (int)(src.size() / len);
    std::vector<int> t((size_t)cnt * len);
    for (int b = 0; b < cnt; ++b)
      for (int q = 0; q < len; ++q) t[(size_t)b * len + q] = src[(size_t)b * len + (len - 1 - q)];
    out[d - k] = std::move(t);
  }
  return out;
}

// Pads every set S[k] (tuples over modes k..d-1) with distinct pseudo-random
// tuples up to min(cap, (n-1)^(d-k)), so that the ranks found by the next
// sweep can grow up to the cap (pivoting alone can only keep or lower them).
// Index q of a tuple is drawn around the grid centre with standard
// deviation sd[k+q] grid points, where |Phi0| is not negligible: uniform
// tuples in many modes land where Phi0 underflows to zero.
void cross_pad(std::vector<std::vector<int>>& S, int d, int n, int cap, const std::vector<double>& sd,
               unsigned long long& st) {
  auto unif = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return ((double)(st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (int k = 1; k < d; ++k) {
    const int len = d - k;
    double full = 1.0;
    for (int q = 0; q < len && full <= cap; ++q) full *= (n - 1);
    const size_t want = (size_t)std::min<double>(cap, full);
    // keep the distinct tuples already present (first occurrence, at most
    // `want`), then add fresh ones
    std::set<std::vector<int>> have;
    std::vector<int> v;
    const std::vector<int>& old = S[k];
    for (size_t b = 0; b < old.size() / len && have.size() < want; ++b) {
      std::vector<int> t(old.begin() + b * len, old.begin() + (b + 1) * len);
      if (have.insert(t).second) v.insert(v.end(), t.begin(), t.end());
    }
    size_t guard = 0;
    while (have.size() < want && guard++ < 100 * want + 100) {
      std::vector<int> t(len);
      for (int q = 0; q < len; ++q) {
        // Box-Muller normal deviate
        const double g = std::sqrt(-2.0 * std::log(unif())) * std::cos(6.283185307179586 * unif());
        int x = n / 2 + (int)std::lround(g * sd[k + q]);
        t[q] = std::min(n - 1, std::max(1, x));
      }
      if (have.insert(t).second) v.insert(v.end(), t.begin(), t.end());
    }
    S[k] = std::move(v);
  }
}

hopf_status init_cross(hopf_ctx* ctx, const double* m0, const double* C0, hopf_tt** out, bool* capped) {
  const int d = ctx->p.d, n = ctx->p.n, cap = ctx->p.rank_cap;
  if (cap > 256) return fail(ctx, HOPF_EINVAL, "cross construction supports rank_cap <= 256");
  TRY(coop_reserve(ctx, std::max(64, cap)));
  CrossBufs B;
  auto done = [&](hopf_status st) {
    B.release();
    return st;
  };
  const size_t Acap = (size_t)cap * n * cap;
  if (dalloc(&B.A, Acap) != cudaSuccess || dalloc(&B.W, Acap) != cudaSuccess ||
      dalloc(&B.Gw, (size_t)cap * cap) != cudaSuccess || dalloc(&B.Gi, (size_t)cap * cap) != cudaSuccess ||
      dalloc(&B.il, (size_t)cap * d) != cudaSuccess || dalloc(&B.jr, (size_t)cap * d) != cudaSuccess ||
      dalloc(&B.piv, (size_t)2 * cap + 1) != cudaSuccess || dalloc(&B.mc, (size_t)d + (size_t)d * d) != cudaSuccess ||
      dalloc(&B.seq, (size_t)cap) != cudaSuccess || dalloc(&B.Q, Acap) != cudaSuccess ||
      dalloc(&B.tau, (size_t)cap) != cudaSuccess || dalloc(&B.T, (size_t)(cap / 8 + 2) * 32 * 32) != cudaSuccess) {
    cudaGetLastError();
    return done(fail(ctx, HOPF_ENOMEM, "cross: workspace allocation failed"));
  }
  std::vector<double> m(m0, m0 + d), C(C0, C0 + (size_t)d * d), mr(d), Cr((size_t)d * d);
  for (int s = 0; s < d; ++s) {
    mr[s] = m[d - 1 - s];
    for (int t = 0; t < d; ++t) Cr[s + (size_t)d * t] = C[(d - 1 - s) + (size_t)d * (d - 1 - t)];
  }
  // sampling widths in grid points: |Phi0| ~ exp(-C_kk a_k^2 / 2) along mode k
  const double da = 2.0 * ctx->L / n;
  std::vector<double> sd(d), sdr(d);
  for (int k = 0; k < d; ++k) sd[k] = 1.0 / (std::sqrt(C[k + (size_t)d * k]) * da);
  for (int k = 0; k < d; ++k) sdr[k] = sd[d - 1 - k];
  // initial right sets: distinct pseudo-random tuples (cross_pad)
  std::vector<std::vector<int>> R(d + 1), L, Lm;
  unsigned long long st = 0x9E3779B97F4A7C15ull;
  hopf_status s = HOPF_OK;
  for (int it = 0; it < 2 && s == HOPF_OK; ++it) {
    cross_pad(R, d, n, cap, sd, st);
    s = cross_sweep(ctx, B, cap, m, C, R, L, nullptr);  // left sets
    if (s != HOPF_OK) break;
    std::vector<std::vector<int>> Rm = cross_mirror(L, d, true);
    cross_pad(Rm, d, n, cap, sdr, st);
    s = cross_sweep(ctx, B, cap, mr, Cr, Rm, Lm, nullptr);
    if (s == HOPF_OK) R = cross_mirror(Lm, d, true);  // right sets
  }
  if (s == HOPF_OK) cross_pad(R, d, n, cap, sd, st);
  hopf_tt* t = nullptr;
  if (s == HOPF_OK) s = tt_alloc(ctx, cap, &t);
  if (s == HOPF_OK) s = cross_sweep(ctx, B, cap, m, C, R, L, t);
  if (s == HOPF_OK) s = round_impl(ctx, t, ctx->p.tol, cap, nullptr, nullptr, capped);
  if (s != HOPF_OK) {
    tt_free(t);
    return done(s);
  }
  *out = t;
  return done(HOPF_OK);
}

}  // namespace

// Accessors for the allocation-free entry point (noalloc.cu).
hopf_ctx* hopf_internal_tt_ctx(const hopf_tt* t) { return t->ctx; }
cudaStream_t hopf_internal_stream(const hopf_ctx* ctx) { return ctx->stream; }
int hopf_internal_device(const hopf_ctx* ctx) { return ctx->device; }
int* hopf_internal_wait_record(hopf_ctx* ctx) { return &ctx->coop.bar->err; }
hopf_status hopf_internal_check_waits(hopf_ctx* ctx) { return check_barrier(ctx); }
hopf_status hopf_internal_tt_view(const hopf_tt* t, const double2* const** d_ptrs, const int** d_ranks,
                                  int* d, int* n, int* maxr) {
  *d_ptrs = t->d_ptrs;
  *d_ranks = t->d_ranks;
  *d = t->d;
  *n = t->n;
  int m = 1;
  for (int r : t->ranks) m = std::max(m, r);
  *maxr = m;
  return HOPF_OK;
}
void hopf_internal_set_error(hopf_ctx* ctx, const char* msg) {
  if (ctx) ctx->err = msg;
}

// ===========================================================================
extern "C" {

hopf_status hopf_create(const hopf_params* p, void* stream, hopf_ctx** out) {
  if (!p || !out) return HOPF_EINVAL;
  *out = nullptr;
  if (p->d < 3 || p->d > 64 || p->n < 4 || (p->n & 1) || p->rank_cap < 1 || !(p->tol >= 0.0) ||
      (p->precision != HOPF_FP64 && p->precision != HOPF_MIXED) || !(p->nu >= 0.0))
    return HOPF_EINVAL;
  hopf_ctx* ctx = new (std::nothrow) hopf_ctx();
  if (!ctx) return HOPF_ENOMEM;
  hk::live_add(1);  // hopf_destroy (also on the failure paths below) takes it back
  ctx->p = *p;
  ctx->stream = (cudaStream_t)stream;
  cudaGetDevice(&ctx->device);
  ctx->L = p->L;
  auto bad = [&](hopf_status st) {
    hopf_destroy(ctx);
    return st;
  };
  if (dalloc(&ctx->d_coef, (size_t)3 * hk::kNumOps * p->n) != cudaSuccess || dalloc(&ctx->d_blocks, 3 * 36) != cudaSuccess ||
      dalloc(&ctx->d_agrid, p->n) != cudaSuccess || dalloc(&ctx->d_dbl, 16) != cudaSuccess ||
      dalloc(&ctx->d_int, 16) != cudaSuccess || dalloc(&ctx->coop.bar, 1) != cudaSuccess ||
      dalloc(&ctx->coop.pr, 1024) != cudaSuccess || dalloc(&ctx->coop.scal, 8) != cudaSuccess ||
      dalloc(&ctx->coop.counters, 64) != cudaSuccess || dalloc(&ctx->d_terms, 16 * 64) != cudaSuccess)
    return bad(HOPF_ENOMEM);
  if (cudaMallocHost((void**)&ctx->h_dbl, 16 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_int, 16 * sizeof(int)) != cudaSuccess)
    return bad(HOPF_ENOMEM);
  if (cudaMemsetAsync(ctx->coop.bar, 0, sizeof(GridBar), ctx->stream) != cudaSuccess) return bad(HOPF_ECUDA);
  unsigned char tab[3][36];
  mpo_tables(tab, HOPF_EQ_PHI);
  if (cudaMemcpyAsync(ctx->d_blocks, tab, sizeof tab, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    return bad(HOPF_ECUDA);
  if (ctx->L > 0.0 && build_ops(ctx) != HOPF_OK) return bad(HOPF_ECUDA);
  if (coop_reserve(ctx, 64) != HOPF_OK) return bad(HOPF_ENOMEM);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return bad(HOPF_ECUDA);
  *out = ctx;
  return HOPF_OK;
}

hopf_status hopf_set_allocator(hopf_alloc_fn alloc, hopf_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return HOPF_EINVAL;
  if (g_live.load() != 0) return HOPF_EINVAL;
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_user = user;
  return HOPF_OK;
}

void tt_free(hopf_tt* t) {
  if (!t) return;
  hk::live_add(-1);
  for (cplx* c : t->cores) dfree(c);
  dfree(t->d_ptrs);
  dfree(t->d_ranks);
  delete t;
}

void hopf_destroy(hopf_ctx* ctx) {
  if (!ctx) return;
  hk::live_add(-1);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  tt_free(ctx->big);
  for (auto k : ctx->kst) tt_free(k);
  tt_free(ctx->ytmp);
  RoundWs& w = ctx->rw;
  for (cplx* b : w.B) dfree(b);
  dfree(w.W1); dfree(w.tau); dfree(w.T); dfree(w.tau2); dfree(w.T2);
  dfree(w.Rb); dfree(w.Mb); dfree(w.Jb); dfree(w.Ub); dfree(w.Sb);
  dfree(w.sig); dfree(w.perm);
  dfree(w.bd_d); dfree(w.bd_e); dfree(w.bd_tauq); dfree(w.bd_taup); dfree(w.bd_a2);
  dfree(w.bd_info); dfree(w.bd_X); dfree(w.bd_Zs);
  dfree(w.G); dfree(w.G2); dfree(w.bd_rows);
  dfree(ctx->tcbuf);
  dfree(ctx->ev_idx); dfree(ctx->ev_vals); dfree(ctx->ev_out);
  dfree(ctx->coop.bar); dfree(ctx->coop.pr); dfree(ctx->coop.pc);
  dfree(ctx->coop.wfin); dfree(ctx->coop.scal); dfree(ctx->coop.counters);
  dfree(ctx->coop.colnorm); dfree(ctx->coop.colver); dfree(ctx->coop.pairchk);
  dfree(ctx->d_coef); dfree(ctx->d_blocks); dfree(ctx->d_agrid);
  dfree(ctx->d_dbl); dfree(ctx->d_int); dfree(ctx->d_terms);
  for (void* p : ctx->extra) dfree(p);
  for (auto e : ctx->prof_ev) cudaEventDestroy(e);
  if (ctx->h_dbl) cudaFreeHost(ctx->h_dbl);
  if (ctx->h_int) cudaFreeHost(ctx->h_int);
  delete ctx;
}

const char* hopf_last_error(const hopf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

hopf_status hopf_set_L(hopf_ctx* ctx, double L) {
  if (!ctx) return HOPF_EINVAL;
  if (!(L >= 0.0) || !std::isfinite(L)) return fail(ctx, HOPF_EINVAL, "L must be positive (or 0: unset)");
  ctx->L = L;
  return L > 0.0 ? build_ops(ctx) : HOPF_OK;
}

hopf_status hopf_set_nu(hopf_ctx* ctx, double nu) {
  if (!ctx) return HOPF_EINVAL;
  if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(ctx, HOPF_EINVAL, "nu must be >= 0");
  ctx->p.nu = nu;
  return ctx->L > 0.0 ? build_ops(ctx) : HOPF_OK;
}

hopf_status hopf_set_max_ctas(hopf_ctx* ctx, int max_ctas) {
  if (!ctx) return HOPF_EINVAL;
  if (max_ctas < 0) return fail(ctx, HOPF_EINVAL, "max_ctas must be >= 0");
  ctx->coop.max_ctas = max_ctas;
  return HOPF_OK;
}

hopf_status hopf_check_watchdog(hopf_ctx* ctx) {
  if (!ctx) return HOPF_EINVAL;
  CK(hk::watchdog_probe(ctx->coop, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_barrier(ctx);
}

hopf_status hopf_set_wait_limit(hopf_ctx* ctx, double seconds) {
  if (!ctx) return HOPF_EINVAL;
  if (!(seconds >= 0.0) || seconds > 60.0) return fail(ctx, HOPF_EINVAL, "wait limit must be in [0, 60] s");
  ctx->wait_limit_us = seconds == 0.0 ? 0u : (unsigned int)std::max(1.0, std::round(seconds * 1e6));
  reset_barrier(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  return HOPF_OK;
}

namespace {
constexpr char kTtMagic[8] = {'H', 'O', 'P', 'F', 'T', 'T', '\0', '\1'};
}

hopf_status tt_save(const hopf_tt* t, const char* path, double time) {
  if (!t || !path) return HOPF_EINVAL;
  hopf_ctx* ctx = t->ctx;
  size_t nd = 0;
  tt_size(t, &nd);
  std::vector<double> buf(nd);
  TRY(tt_to_host(t, buf.data(), nd));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, HOPF_EINVAL, "tt_save: cannot open %s", path);
  const int hdr[2] = {t->d, t->n};
  bool ok = std::fwrite(kTtMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int), 2, f) == 2 &&
            std::fwrite(t->ranks.data(), sizeof(int), t->d + 1, f) == (size_t)(t->d + 1) &&
            std::fwrite(&time, sizeof(double), 1, f) == 1 && std::fwrite(buf.data(), sizeof(double), nd, f) == nd;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(ctx, HOPF_EINVAL, "tt_save: write to %s failed", path);
  return HOPF_OK;
}

hopf_status tt_load(hopf_ctx* ctx, const char* path, int max_rank, hopf_tt** out, double* time) {
  if (!ctx || !path || !out) return ctx ? fail(ctx, HOPF_EINVAL, "tt_load: null argument") : HOPF_EINVAL;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, HOPF_EINVAL, "tt_load: cannot open %s", path);
  char magic[8];
  int hdr[2] = {0, 0};
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kTtMagic, 8) == 0 &&
            std::fread(hdr, sizeof(int), 2, f) == 2 && hdr[0] == ctx->p.d && hdr[1] == ctx->p.n;
  std::vector<int> ranks(ctx->p.d + 1);
  double tm = 0.0;
  ok = ok && std::fread(ranks.data(), sizeof(int), ranks.size(), f) == ranks.size() &&
       std::fread(&tm, sizeof(double), 1, f) == 1;
  size_t nd = 0;
  if (ok) {
    for (int k = 0; k < ctx->p.d && ok; ++k) {
      ok = ranks[k] >= 1 && ranks[k + 1] >= 1 && ranks[k] <= (1 << 20) && ranks[k + 1] <= (1 << 20);
      nd += 2 * (size_t)ranks[k] * ctx->p.n * ranks[k + 1];
    }
  }
  std::vector<double> buf(ok ? nd : 0);
  ok = ok && std::fread(buf.data(), sizeof(double), nd, f) == nd;
  std::fclose(f);
  if (!ok) return fail(ctx, HOPF_EINVAL, "tt_load: %s is not a TT of this context's d and n (or is truncated)", path);
  const int cap = max_rank > 0 ? max_rank : *std::max_element(ranks.begin(), ranks.end());
  TRY(tt_from_host(ctx, ranks.data(), buf.data(), cap, out));
  if (time) *time = tm;
  return HOPF_OK;
}

hopf_status hopf_set_qr_method(hopf_ctx* ctx, int method) {
  if (!ctx) return HOPF_EINVAL;
  if (method != HOPF_QR_DOUBLEFLOAT && method != HOPF_QR_TENSOR) return fail(ctx, HOPF_EINVAL, "unknown QR method %d", method);
  ctx->qr_method = method;
  return HOPF_OK;
}

hopf_status hopf_set_autotune(hopf_ctx* ctx, int enable) {
  if (!ctx) return HOPF_EINVAL;
  if (enable != 0 && enable != 1) return fail(ctx, HOPF_EINVAL, "enable must be 0 or 1");
  ctx->autotune = enable;
  if (!enable) ctx->tune.clear();
  return HOPF_OK;
}

hopf_status hopf_get_autotune(const hopf_ctx* ctx, int* shapes, float* ms, int cap, int* count) {
  if (!ctx || !count || cap < 0 || (cap > 0 && (!shapes || !ms))) return HOPF_EINVAL;
  *count = (int)ctx->tune.size();
  const int n = std::min(cap, *count);
  for (int i = 0; i < n; ++i) {
    const hopf_ctx::QrTune& t = ctx->tune[i];
    shapes[4 * i + 0] = t.m;
    shapes[4 * i + 1] = t.p;
    shapes[4 * i + 2] = t.method;
    shapes[4 * i + 3] = t.ctas;
    for (int j = 0; j < 4; ++j) ms[4 * i + j] = t.ms[j];
  }
  return HOPF_OK;
}

hopf_status hopf_set_svd_method(hopf_ctx* ctx, int method) {
  if (!ctx) return HOPF_EINVAL;
  if (method != HOPF_SVD_AUTO && method != HOPF_SVD_JACOBI) return fail(ctx, HOPF_EINVAL, "unknown SVD method %d", method);
  ctx->svd_method = method;
  return HOPF_OK;
}

hopf_status hopf_get_L(const hopf_ctx* ctx, double* L) {
  if (!ctx || !L) return HOPF_EINVAL;
  *L = ctx->L;
  return HOPF_OK;
}

hopf_status hopf_cell_moments(hopf_ctx* ctx, int nmodes, const double* alpha, const double* beta,
                              double sigma, double ell, double* m0, double* C0) {
  if (!ctx) return HOPF_EINVAL;
  if (nmodes < 0 || nmodes > 64 || (nmodes && (!alpha || !beta)) || !m0 || !C0 || !(ell > 0.0) || !(sigma >= 0.0))
    return fail(ctx, HOPF_EINVAL, "hopf_cell_moments: bad arguments");
  const int d = ctx->p.d, q = 12;
  std::vector<double> host(2 * 64 + 2 * q, 0.0);
  for (int i = 0; i < nmodes; ++i) {
    host[i] = alpha[i];
    host[64 + i] = beta[i];
  }
  const std::vector<double> gl = gauss_legendre01(q);
  std::copy(gl.begin(), gl.end(), host.begin() + 128);
  double* dbuf = nullptr;
  CK(dalloc(&dbuf, host.size() + d + (size_t)d * d));
  CK(cudaMemcpyAsync(dbuf, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  double* dm0 = dbuf + host.size();
  double* dC0 = dm0 + d;
  cudaError_t e = hk::cell_moments(d, nmodes, dbuf, dbuf + 64, sigma, ell, dbuf + 128, q, dm0, dC0, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m0, dm0, d * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(C0, dC0, (size_t)d * d * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  dfree(dbuf);
  if (e != cudaSuccess) return fail(ctx, HOPF_ECUDA, "hopf_cell_moments: %s", cudaGetErrorString(e));
  for (int j = 0; j < d; ++j)
    for (int k = j + 1; k < d; ++k) {
      const double s = 0.5 * (C0[j + d * k] + C0[k + d * j]);
      C0[j + d * k] = C0[k + d * j] = s;
    }
  return HOPF_OK;
}

hopf_status tt_create(hopf_ctx* ctx, int max_rank, hopf_tt** out) {
  if (!ctx || !out || max_rank < 1) return ctx ? fail(ctx, HOPF_EINVAL, "tt_create: bad arguments") : HOPF_EINVAL;
  TRY(tt_alloc(ctx, max_rank, out));
  hopf_tt* t = *out;
  for (int k = 0; k < t->d; ++k) CK(cudaMemsetAsync(t->cores[k], 0, t->core_cap[k] * sizeof(cplx), ctx->stream));
  return sync_meta(ctx, t);
}

hopf_status tt_from_host(hopf_ctx* ctx, const int* ranks, const double* cores, int max_rank, hopf_tt** out) {
  if (!ctx || !ranks || !cores || !out) return ctx ? fail(ctx, HOPF_EINVAL, "tt_from_host: null argument") : HOPF_EINVAL;
  const int d = ctx->p.d, n = ctx->p.n;
  if (ranks[0] != 1 || ranks[d] != 1) return fail(ctx, HOPF_EINVAL, "boundary ranks must be 1");
  for (int k = 0; k <= d; ++k)
    if (ranks[k] < 1 || ranks[k] > max_rank) return fail(ctx, HOPF_EINVAL, "rank %d = %d outside [1, max_rank=%d]", k, ranks[k], max_rank);
  hopf_tt* t = nullptr;
  TRY(tt_alloc(ctx, max_rank, &t));
  size_t off = 0;
  for (int k = 0; k < d; ++k) {
    const size_t ne = (size_t)ranks[k] * n * ranks[k + 1];
    cudaError_t e = cudaMemcpyAsync(t->cores[k], cores + 2 * off, ne * sizeof(cplx), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
      tt_free(t);
      return fail(ctx, HOPF_ECUDA, "%s", cudaGetErrorString(e));
    }
    off += ne;
  }
  t->ranks.assign(ranks, ranks + d + 1);
  hopf_status st = sync_meta(ctx, t);
  if (st == HOPF_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = fail(ctx, HOPF_ECUDA, "upload failed");
  if (st != HOPF_OK) {
    tt_free(t);
    return st;
  }
  *out = t;
  return HOPF_OK;
}

hopf_status tt_get_ranks(const hopf_tt* t, int* ranks) {
  if (!t || !ranks) return HOPF_EINVAL;
  std::copy(t->ranks.begin(), t->ranks.end(), ranks);
  return HOPF_OK;
}

hopf_status tt_size(const hopf_tt* t, size_t* nd) {
  if (!t || !nd) return HOPF_EINVAL;
  size_t s = 0;
  for (int k = 0; k < t->d; ++k) s += core_elems(t, k);
  *nd = 2 * s;
  return HOPF_OK;
}

hopf_status tt_to_host(const hopf_tt* t, double* cores, size_t cap_doubles) {
  if (!t || !cores) return HOPF_EINVAL;
  hopf_ctx* ctx = t->ctx;
  size_t need = 0;
  tt_size(t, &need);
  if (cap_doubles < need) return fail(ctx, HOPF_EINVAL, "tt_to_host: buffer holds %zu doubles, %zu needed", cap_doubles, need);
  size_t off = 0;
  for (int k = 0; k < t->d; ++k) {
    const size_t ne = core_elems(t, k);
    CK(cudaMemcpyAsync(cores + 2 * off, t->cores[k], ne * sizeof(cplx), cudaMemcpyDeviceToHost, ctx->stream));
    off += ne;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return HOPF_OK;
}

hopf_status tt_copy(hopf_ctx* ctx, const hopf_tt* src, hopf_tt* dst) {
  if (!ctx || !src || !dst) return ctx ? fail(ctx, HOPF_EINVAL, "tt_copy: null argument") : HOPF_EINVAL;
  if (src == dst) return HOPF_OK;
  return copy_impl(ctx, src, dst);
}

hopf_status hopf_apply_op(hopf_ctx* ctx, const hopf_tt* in, hopf_tt* out) {
  if (!ctx || !in || !out || in == out) return ctx ? fail(ctx, HOPF_EINVAL, "hopf_apply_op: bad arguments") : HOPF_EINVAL;
  if (!(ctx->L > 0.0)) return fail(ctx, HOPF_EINVAL, "L is not set (hopf_set_L or hopf_init_gaussian)");
  return apply_impl(ctx, in, out);
}

hopf_status tt_round(hopf_ctx* ctx, hopf_tt* t, double tol, int cap, const int* forced, double* disc) {
  if (!ctx || !t) return ctx ? fail(ctx, HOPF_EINVAL, "tt_round: null argument") : HOPF_EINVAL;
  if (!(tol >= 0.0) || cap < 1) return fail(ctx, HOPF_EINVAL, "tt_round: tol must be >= 0 and cap >= 1");
  if (forced && (forced[0] != 1 || forced[t->d] != 1)) return fail(ctx, HOPF_EINVAL, "forced boundary ranks must be 1");
  bool capped = false;
  TRY(round_impl(ctx, t, tol, cap, forced, disc, &capped));
  return capped ? HOPF_ERANKCAP : HOPF_OK;
}

hopf_status tt_sum(hopf_ctx* ctx, int nterms, const hopf_tt* const* terms, const double* coef, hopf_tt* out) {
  if (!ctx || !terms || !coef || !out) return ctx ? fail(ctx, HOPF_EINVAL, "tt_sum: null argument") : HOPF_EINVAL;
  return sum_impl(ctx, nterms, terms, coef, out);
}

hopf_status hopf_profile_enable(hopf_ctx* ctx, int on) {
  if (!ctx) return HOPF_EINVAL;
  if (on && ctx->prof_ev.empty()) {
    ctx->prof_ev.resize(2 * kProfSlots);
    for (auto& e : ctx->prof_ev) CK(cudaEventCreate(&e));
  }
  if (!on) TRY(prof_flush(ctx));
  ctx->prof_on = on != 0;
  return HOPF_OK;
}

hopf_status hopf_profile_read(hopf_ctx* ctx, hopf_profile* out, int reset) {
  if (!ctx || !out) return HOPF_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  TRY(prof_flush(ctx));
  *out = ctx->prof;
  if (reset) ctx->prof = hopf_profile{};
  return HOPF_OK;
}

hopf_status tt_set_from_host(hopf_tt* t, const int* ranks, const double* cores) {
  if (!t || !ranks || !cores) return HOPF_EINVAL;
  hopf_ctx* ctx = t->ctx;
  const int d = t->d, n = t->n;
  std::vector<int> r(ranks, ranks + d + 1);
  if (r[0] != 1 || r[d] != 1) return fail(ctx, HOPF_EINVAL, "boundary ranks must be 1");
  for (int k = 0; k <= d; ++k)
    if (r[k] < 1) return fail(ctx, HOPF_EINVAL, "rank %d = %d < 1", k, r[k]);
  TRY(check_fit(ctx, t, r));
  size_t off = 0;
  for (int k = 0; k < d; ++k) {
    const size_t ne = (size_t)r[k] * n * r[k + 1];
    CK(cudaMemcpyAsync(t->cores[k], cores + 2 * off, ne * sizeof(cplx), cudaMemcpyHostToDevice, ctx->stream));
    off += ne;
  }
  t->ranks = r;
  return sync_meta(ctx, t);
}

hopf_status tt_norm(hopf_ctx* ctx, const hopf_tt* t, double* norm) {
  if (!ctx || !t || !norm) return ctx ? fail(ctx, HOPF_EINVAL, "tt_norm: null argument") : HOPF_EINVAL;
  TRY(round_reserve(ctx, t));
  std::vector<int> p, nbv;
  TRY(orth_sweep(ctx, t, p, nbv));
  TRY(read_small_checked(ctx, 0, 1));
  *norm = std::sqrt(ctx->h_dbl[0]);
  return HOPF_OK;
}

// Roundings per step of each scheme (the layout of rank logs).
int scheme_roundings(int scheme) { return scheme == HOPF_EULER ? 2 : scheme == HOPF_MIDPOINT ? 3 : 8; }

hopf_status hopf_step_scheme(hopf_ctx* ctx, hopf_tt* f, int scheme, double dt, int nsteps, double* disc_sum,
                             int* rank_log, const int* forced_log) {
  if (!ctx || !f) return ctx ? fail(ctx, HOPF_EINVAL, "hopf_step: null argument") : HOPF_EINVAL;
  if (nsteps < 0 || !std::isfinite(dt)) return fail(ctx, HOPF_EINVAL, "hopf_step: bad dt or nsteps");
  if (scheme != HOPF_RK4 && scheme != HOPF_EULER && scheme != HOPF_MIDPOINT)
    return fail(ctx, HOPF_EINVAL, "hopf_step: unknown scheme %d", scheme);
  if (!(ctx->L > 0.0)) return fail(ctx, HOPF_EINVAL, "L is not set (hopf_set_L or hopf_init_gaussian)");
  const int cap = ctx->p.rank_cap;
  const double tol = ctx->p.tol;
  if (f->cap_rank < cap) return fail(ctx, HOPF_EINVAL, "hopf_step: the state needs capacity >= rank_cap");
  for (int k = 0; k <= f->d; ++k)
    if (f->ranks[k] > cap) return fail(ctx, HOPF_EINVAL, "hopf_step: input rank %d exceeds rank_cap", f->ranks[k]);
  TRY(ensure_step_ws(ctx, cap, scheme));
  hopf_tt* big = ctx->big;
  hopf_tt** K = ctx->kst;
  hopf_tt* Y = ctx->ytmp;
  const int d = f->d;
  double dsum = 0.0;
  bool capped = false;
  int round_idx = 0;
  auto T = [&](hopf_tt* x, hopf_tt* dst) -> hopf_status {
    const int* forced = forced_log ? forced_log + (size_t)round_idx * (d + 1) : nullptr;
    double disc = 0.0;
    bool c = false;
    TRY(round_impl(ctx, x, tol, cap, forced, &disc, &c));
    capped |= c;
    dsum += disc;
    if (rank_log) std::copy(x->ranks.begin(), x->ranks.end(), rank_log + (size_t)round_idx * (d + 1));
    ++round_idx;
    return copy_impl(ctx, x, dst);
  };
  // K = T[G y] with the apply fused into the orthogonalisation sweep
  auto TG = [&](const hopf_tt* y, hopf_tt* dst) -> hopf_status {
    const int* forced = forced_log ? forced_log + (size_t)round_idx * (d + 1) : nullptr;
    double disc = 0.0;
    bool c = false;
    TRY(round_apply_impl(ctx, y, big, tol, cap, forced, &disc, &c));
    capped |= c;
    dsum += disc;
    if (rank_log) std::copy(big->ranks.begin(), big->ranks.end(), rank_log + (size_t)round_idx * (d + 1));
    ++round_idx;
    return copy_impl(ctx, big, dst);
  };
  for (int s = 0; s < nsteps; ++s) {
    const hopf_tt* tm[5];
    double cf[10] = {0};
    if (scheme == HOPF_EULER) {
      // f <- T_r[f + dt T_s[G f]]  (Eq. adaptive-euler-method)
      TRY(TG(f, K[0]));
      tm[0] = f; tm[1] = K[0]; cf[0] = 1.0; cf[2] = dt;
      TRY(sum_impl(ctx, 2, tm, cf, big));
      TRY(T(big, f));
      continue;
    }
    if (scheme == HOPF_MIDPOINT) {
      // f <- T_a[f + dt T_b[G(f + dt/2 T_c[G f])]]  (Eq. adaptive-midpoint-method;
      // the inner sum is not truncated)
      TRY(TG(f, K[0]));
      tm[0] = f; tm[1] = K[0]; cf[0] = 1.0; cf[2] = 0.5 * dt;
      TRY(sum_impl(ctx, 2, tm, cf, Y));
      TRY(TG(Y, K[1]));
      tm[1] = K[1]; cf[2] = dt;
      TRY(sum_impl(ctx, 2, tm, cf, big));
      TRY(T(big, f));
      continue;
    }
    // K1 = T[G f]
    TRY(TG(f, K[0]));
    // Y2 = T[f + dt/2 K1]; K2 = T[G Y2]
    tm[0] = f; tm[1] = K[0]; cf[0] = 1.0; cf[2] = 0.5 * dt;
    TRY(sum_impl(ctx, 2, tm, cf, big));
    TRY(T(big, Y));
    TRY(TG(Y, K[1]));
    // Y3 = T[f + dt/2 K2]; K3 = T[G Y3]
    tm[1] = K[1];
    TRY(sum_impl(ctx, 2, tm, cf, big));
    TRY(T(big, Y));
    TRY(TG(Y, K[2]));
    // Y4 = T[f + dt K3]; K4 = T[G Y4]
    tm[1] = K[2]; cf[2] = dt;
    TRY(sum_impl(ctx, 2, tm, cf, big));
    TRY(T(big, Y));
    TRY(TG(Y, K[3]));
    // f <- T[f + dt/6 (K1 + 2 K2 + 2 K3 + K4)]
    tm[0] = f; tm[1] = K[0]; tm[2] = K[1]; tm[3] = K[2]; tm[4] = K[3];
    cf[0] = 1.0; cf[2] = dt / 6.0; cf[4] = dt / 3.0; cf[6] = dt / 3.0; cf[8] = dt / 6.0;
    TRY(sum_impl(ctx, 5, tm, cf, big));
    TRY(T(big, f));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (disc_sum) *disc_sum = dsum;
  return capped ? HOPF_ERANKCAP : HOPF_OK;
}

hopf_status hopf_step(hopf_ctx* ctx, hopf_tt* f, double dt, int nsteps, double* disc_sum, int* rank_log,
                      const int* forced_log) {
  return hopf_step_scheme(ctx, f, HOPF_RK4, dt, nsteps, disc_sum, rank_log, forced_log);
}

hopf_status hopf_set_equation(hopf_ctx* ctx, int equation, double box) {
  if (!ctx) return HOPF_EINVAL;
  if (equation != HOPF_EQ_PHI && equation != HOPF_EQ_CDF) return fail(ctx, HOPF_EINVAL, "unknown equation %d", equation);
  if (!(box >= 0.0) || !std::isfinite(box)) return fail(ctx, HOPF_EINVAL, "box half-width must be >= 0");
  if (equation == HOPF_EQ_CDF && !(box > 0.0)) return fail(ctx, HOPF_EINVAL, "the CDF equation needs a box half-width > 0");
  ctx->equation = equation;
  ctx->L = box;
  unsigned char tab[3][36];
  mpo_tables(tab, equation);
  CK(cudaMemcpyAsync(ctx->d_blocks, tab, sizeof tab, cudaMemcpyHostToDevice, ctx->stream));
  if (box > 0.0) TRY(build_ops(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  return HOPF_OK;
}

hopf_status hopf_init_cdf(hopf_ctx* ctx, double sigma, const double* mu, hopf_tt** out) {
  if (!ctx || !out) return ctx ? fail(ctx, HOPF_EINVAL, "hopf_init_cdf: null argument") : HOPF_EINVAL;
  if (ctx->equation != HOPF_EQ_CDF) return fail(ctx, HOPF_EINVAL, "hopf_init_cdf: the context is not set to the CDF equation");
  if (!(sigma > 0.0)) return fail(ctx, HOPF_EINVAL, "hopf_init_cdf: sigma must be > 0");
  const int d = ctx->p.d, n = ctx->p.n;
  std::vector<double> host((size_t)2 * n * d);
  for (int k = 0; k < d; ++k)
    for (int i = 0; i < n; ++i) {
      const double m = mu ? mu[k] : 0.0;
      host[2 * ((size_t)k * n + i)] = 0.5 * (1.0 + std::erf((ctx->agrid[i] - m) / (sigma * std::sqrt(2.0))));
      host[2 * ((size_t)k * n + i) + 1] = 0.0;
    }
  std::vector<int> ranks(d + 1, 1);
  hopf_tt* t = nullptr;
  TRY(tt_alloc(ctx, ctx->p.rank_cap, &t));
  size_t off = 0;
  for (int k = 0; k < d; ++k) {
    cudaError_t e = cudaMemcpyAsync(t->cores[k], host.data() + 2 * off, (size_t)n * sizeof(cplx), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e != cudaSuccess) {
      tt_free(t);
      return fail(ctx, HOPF_ECUDA, "%s", cudaGetErrorString(e));
    }
    off += n;
  }
  t->ranks = ranks;
  hopf_status st = sync_meta(ctx, t);
  if (st == HOPF_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = fail(ctx, HOPF_ECUDA, "upload failed");
  if (st != HOPF_OK) {
    tt_free(t);
    return st;
  }
  *out = t;
  return HOPF_OK;
}

hopf_status hopf_eval_points(hopf_ctx* ctx, const hopf_tt* t, int npts, const int* idx, double* vals) {
  if (!ctx || !t || (npts > 0 && (!idx || !vals)) || npts < 0)
    return ctx ? fail(ctx, HOPF_EINVAL, "hopf_eval_points: bad arguments") : HOPF_EINVAL;
  if (npts == 0) return HOPF_OK;
  const int d = t->d, n = t->n;
  for (size_t e = 0; e < (size_t)npts * d; ++e)
    if (idx[e] < 0 || idx[e] >= n) return fail(ctx, HOPF_EINVAL, "index %d outside [0, %d)", idx[e], n);
  int maxr = 1;
  for (int r : t->ranks) maxr = std::max(maxr, r);
  TRY(ev_reserve(ctx, (size_t)npts * d, (size_t)npts, 0));
  int* didx = ctx->ev_idx;
  cplx* dv = ctx->ev_vals;
  cudaError_t e = cudaMemcpyAsync(didx, idx, (size_t)npts * d * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = hk::eval_points(t->d_ptrs, t->d_ranks, d, n, maxr, npts, didx, dv, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vals, dv, (size_t)npts * sizeof(cplx), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, HOPF_ECUDA, "hopf_eval_points: %s", cudaGetErrorString(e));
  return HOPF_OK;
}

hopf_status hopf_eval_moments(hopf_ctx* ctx, const hopf_tt* t, double* mean, double* cov, double* imag_resid) {
  if (!ctx || !t || !mean || !cov) return ctx ? fail(ctx, HOPF_EINVAL, "hopf_eval_moments: null argument") : HOPF_EINVAL;
  if (!(ctx->L > 0.0)) return fail(ctx, HOPF_EINVAL, "L is not set");
  if (ctx->equation != HOPF_EQ_PHI) return fail(ctx, HOPF_EINVAL, "hopf_eval_moments: moments come from Phi, not a CDF");
  const int d = t->d, n = t->n, c = n / 2;
  const int npts = 1 + 2 * d + 2 * d * (d - 1);
  std::vector<int> idx((size_t)npts * d, c);
  auto at = [&](int pt, int ax, int off) { idx[(size_t)pt * d + ax] = c + off; };
  int pt = 1;
  for (int k = 0; k < d; ++k) {
    at(pt, k, 1); ++pt;
    at(pt, k, -1); ++pt;
  }
  for (int j = 0; j < d; ++j)
    for (int k = j + 1; k < d; ++k) {
      at(pt, j, 1); at(pt, k, 1); ++pt;
      at(pt, j, 1); at(pt, k, -1); ++pt;
      at(pt, j, -1); at(pt, k, 1); ++pt;
      at(pt, j, -1); at(pt, k, -1); ++pt;
    }
  int maxr = 1;
  for (int r : t->ranks) maxr = std::max(maxr, r);
  TRY(ev_reserve(ctx, idx.size(), (size_t)npts, (size_t)d + (size_t)d * d + 1));
  int* didx = ctx->ev_idx;
  cplx* dv = ctx->ev_vals;
  double* dout = ctx->ev_out;
  cudaError_t e = cudaMemcpyAsync(didx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = hk::eval_points(t->d_ptrs, t->d_ranks, d, n, maxr, npts, didx, dv, ctx->stream);
  const double da = 2.0 * ctx->L / n;
  if (e == cudaSuccess) e = hk::moments_combine(dv, d, da, dout, dout + d, dout + d + (size_t)d * d, ctx->stream);
  double ir = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(mean, dout, d * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cov, dout + d, (size_t)d * d * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ir, dout + d + (size_t)d * d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, HOPF_ECUDA, "hopf_eval_moments: %s", cudaGetErrorString(e));
  if (imag_resid) *imag_resid = ir;
  return HOPF_OK;
}

hopf_status hopf_init_gaussian(hopf_ctx* ctx, const double* m0, const double* C0, hopf_tt** out) {
  if (!ctx || !m0 || !C0 || !out) return ctx ? fail(ctx, HOPF_EINVAL, "hopf_init_gaussian: null argument") : HOPF_EINVAL;
  if (ctx->equation != HOPF_EQ_PHI) return fail(ctx, HOPF_EINVAL, "hopf_init_gaussian: the context is set to the CDF equation");
  const int d = ctx->p.d, n = ctx->p.n;
  bool diag = true;
  double minc = 1e300;
  for (int j = 0; j < d; ++j) {
    minc = std::min(minc, C0[j + d * j]);
    for (int k = 0; k < d; ++k)
      if (j != k && C0[j + d * k] != 0.0) diag = false;
  }
  if (!(minc > 0.0)) return fail(ctx, HOPF_EINVAL, "C0 needs a positive diagonal");
  if (!(ctx->L > 0.0)) {
    ctx->L = std::sqrt(36.8 / minc);
    TRY(build_ops(ctx));
  }
  const int cap = ctx->p.rank_cap;
  if (diag) {
    hopf_tt* t = nullptr;
    TRY(tt_create(ctx, cap, &t));
    for (int k = 0; k < d; ++k) {
      cudaError_t e = hk::gauss_rank1_core(ctx->d_agrid, n, m0[k], C0[k + d * k], t->cores[k], ctx->stream);
      if (e != cudaSuccess) {
        tt_free(t);
        return fail(ctx, HOPF_ECUDA, "%s", cudaGetErrorString(e));
      }
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
      tt_free(t);
      return fail(ctx, HOPF_ECUDA, "init failed");
    }
    *out = t;
    return HOPF_OK;
  }
  // small grids: exact TT of the full grid (identity cores around one data
  // core), then round; larger grids: TT-cross interpolation, then round
  const int c = (d - 1) / 2;
  double total = 1.0;
  for (int k = 0; k < d; ++k) total *= n;
  if (total > (double)(1 << 20)) {
    bool capped = false;
    TRY(init_cross(ctx, m0, C0, out, &capped));
    return capped ? HOPF_ERANKCAP : HOPF_OK;
  }
  size_t A = 1, B = 1;
  for (int k = 0; k < c; ++k) A *= n;
  for (int k = c + 1; k < d; ++k) B *= n;
  const int capr = (int)std::max(A, B);
  hopf_tt* full = nullptr;
  TRY(tt_alloc(ctx, capr, &full));
  std::vector<int> r(d + 1, 1);
  {
    size_t a = 1;
    for (int k = 0; k < c; ++k) {
      r[k] = (int)a;
      a *= n;
    }
    r[c] = (int)A;
    r[c + 1] = (int)B;
    size_t b = B;
    for (int k = c + 1; k < d; ++k) {
      r[k] = (int)b;
      b /= n;
    }
    r[d] = 1;
  }
  double* dmc = nullptr;
  hopf_status st = HOPF_OK;
  cudaError_t e = dalloc(&dmc, (size_t)d + (size_t)d * d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dmc, m0, d * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dmc + d, C0, (size_t)d * d * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  for (int k = 0; k < d && e == cudaSuccess; ++k) {
    if (k < c) e = hk::identity_core(n, r[k], r[k + 1], 1, full->cores[k], ctx->stream);
    else if (k == c) e = hk::gauss_full_core(ctx->d_agrid, n, d, c, dmc, dmc + d, full->cores[k], ctx->stream);
    else e = hk::identity_core(n, r[k], r[k + 1], 0, full->cores[k], ctx->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  dfree(dmc);
  if (e != cudaSuccess) st = fail(ctx, HOPF_ECUDA, "init: %s", cudaGetErrorString(e));
  if (st == HOPF_OK) {
    full->ranks = r;
    st = sync_meta(ctx, full);
  }
  bool capped = false;
  if (st == HOPF_OK) st = round_impl(ctx, full, ctx->p.tol, cap, nullptr, nullptr, &capped);
  hopf_tt* t = nullptr;
  if (st == HOPF_OK) st = tt_alloc(ctx, cap, &t);
  if (st == HOPF_OK) st = copy_impl(ctx, full, t);
  if (st == HOPF_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = fail(ctx, HOPF_ECUDA, "init sync failed");
  tt_free(full);
  if (st != HOPF_OK) {
    tt_free(t);
    return st;
  }
  *out = t;
  return capped ? HOPF_ERANKCAP : HOPF_OK;
}

hopf_status hopf_tc_zgemm(hopf_ctx* ctx, int M, int N, int K, const double* A, int lda, int opA, const double* B,
                          int ldb, int opB, int digits, double* C, int ldc) {
  if (!ctx) return HOPF_EINVAL;
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || (opA != 0 && opA != 1) || (opB != 0 && opB != 1) ||
      digits < 1 || digits > hk::tc_max_digits() || ldc < M || lda < (opA ? K : M) || ldb < (opB ? N : K))
    return fail(ctx, HOPF_EINVAL, "hopf_tc_zgemm: bad arguments");
  const size_t na = (size_t)lda * (opA ? M : K), nb = (size_t)ldb * (opB ? K : N), nc = (size_t)ldc * N;
  const int Kc = hk::tc_chunk();
  const size_t oa = hk::tc_operand_bytes(M, K, digits, Kc), ob = hk::tc_operand_bytes(N, K, digits, Kc);
  const size_t np = hk::tc_part_elems(M, N, K);
  cplx *dA = nullptr, *dB = nullptr, *dC = nullptr, *dP = nullptr;
  unsigned char *bufA = nullptr, *bufB = nullptr;
  auto release = [&]() {
    dfree(dA); dfree(dB); dfree(dC); dfree(dP); dfree(bufA); dfree(bufB);
  };
  if (dalloc(&dA, na) != cudaSuccess || dalloc(&dB, nb) != cudaSuccess || dalloc(&dC, nc) != cudaSuccess ||
      dalloc(&dP, np) != cudaSuccess || dalloc(&bufA, oa) != cudaSuccess || dalloc(&bufB, ob) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(ctx, HOPF_ENOMEM, "hopf_tc_zgemm: allocation failed");
  }
  // op(A)(m, k): A[m + lda k] or conj(A[k + lda m]); B operand rows are the
  // columns n of op(B): op(B)(k, n) = B[k + ldb n] or conj(B[n + ldb k])
  hk::TcOperandView va{dA, opA ? (long long)lda : 1, opA ? 1 : (long long)lda, M, K, opA, 0, 0};
  hk::TcOperandView vb{dB, opB ? 1 : (long long)ldb, opB ? (long long)ldb : 1, N, K, opB, 0, 0};
  hk::TcOperand oA, oB;
  cudaError_t e = cudaMemcpyAsync(dA, A, na * sizeof(cplx), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dB, B, nb * sizeof(cplx), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = hk::tc_split(va, digits, &oA, bufA, ctx->stream);
  if (e == cudaSuccess) e = hk::tc_split(vb, digits, &oB, bufB, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dC, 0, nc * sizeof(cplx), ctx->stream);
  if (e == cudaSuccess) e = hk::tc_zgemm(oA, oB, dC, ldc, 1.0, 0, dP, np, &ctx->coop.bar->err, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(C, dC, nc * sizeof(cplx), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  release();
  if (e != cudaSuccess) return fail(ctx, HOPF_ECUDA, "hopf_tc_zgemm: %s", cudaGetErrorString(e));
  return check_barrier(ctx);
}

hopf_status hopf_step_ensemble(int count, hopf_ctx* const* ctxs, hopf_tt* const* tts, const double* dt,
                               int nsteps, hopf_status* statuses) {
  if (count < 0 || (count > 0 && (!ctxs || !tts || !dt || !statuses))) return HOPF_EINVAL;
  for (int a = 0; a < count; ++a) {
    if (!ctxs[a] || !tts[a]) return HOPF_EINVAL;
    for (int b = 0; b < a; ++b)
      if (ctxs[a] == ctxs[b]) return fail(ctxs[a], HOPF_EINVAL, "hopf_step_ensemble: a context appears twice");
  }
  std::vector<std::thread> pool;
  pool.reserve(count);
  for (int a = 0; a < count; ++a) {
    pool.emplace_back([=]() {
      if (cudaSetDevice(ctxs[a]->device) != cudaSuccess) {
        statuses[a] = fail(ctxs[a], HOPF_ECUDA, "hopf_step_ensemble: cudaSetDevice failed");
        return;
      }
      statuses[a] = hopf_step(ctxs[a], tts[a], dt[a], nsteps, nullptr, nullptr, nullptr);
    });
  }
  for (auto& th : pool) th.join();
  hopf_status worst = HOPF_OK;
  for (int a = 0; a < count; ++a)
    if (statuses[a] != HOPF_OK && statuses[a] != HOPF_ERANKCAP) return statuses[a];
    else if (statuses[a] == HOPF_ERANKCAP) worst = HOPF_ERANKCAP;
  return worst;
}

}  // extern "C"
