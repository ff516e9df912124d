// Learned surrogate: an ensemble of small multilayer perceptrons with BF16
// weights, FP32 activations and FP32 accumulation, trained by Adam on the
// solver's outputs, every step a kernel of this file.
//
// The products run on the tensor cores (tcgen05.mma, BF16 x BF16 -> FP32 in
// tensor memory, operands staged by TMA): weights are BF16, and every FP32
// operand (activations, gradients) is carried as three BF16 parts
// x = p0 + p1 + p2 (each the BF16 rounding of what the previous parts
// leave: 24 significant bits, all of FP32's), so the sum of the part
// products in one FP32 accumulator is the FP32-activation product up to
// FP32 accumulation rounding.  Parts products below 2^-24 of the leading one
// are skipped (pairs i + j > 2).  128 x 128 output tiles, the ensemble
// members on gridDim.z, fused bias / GELU / GELU' epilogues.  A training
// step is about thirty launches; it is captured once as a CUDA graph and
// replayed, with the step number read from device memory so that the same
// graph walks through the batch-index and learning-rate tables.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <utility>
#include <vector>

#include "../../include/hopf.h"
#include "tcgen05.cuh"

// The library's device allocator (hopf.cu: cudaMalloc or the caller's
// functions, hopf_set_allocator) and its count of live objects.
namespace hk {
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);
void live_add(int delta);
}  // namespace hk

typedef __nv_bfloat16 bf16;

// Internal accessors defined in hopf.cu.
cudaStream_t hopf_internal_stream(const hopf_ctx* ctx);
void hopf_internal_set_error(hopf_ctx* ctx, const char* msg);
// The device record a kernel's expired bounded wait is written to, and the
// host check of it (HOPF_ETIMEOUT once a wait expired; resets the record).
int* hopf_internal_wait_record(hopf_ctx* ctx);
hopf_status hopf_internal_check_waits(hopf_ctx* ctx);

namespace {

constexpr int kMaxDim = 4096, kMaxMembers = 64;
constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kAdamEps = 1e-8f;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ float ld(const float* p) { return *p; }
__device__ __forceinline__ float ld(const bf16* p) { return __bfloat162float(*p); }

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_GRAD = 3 };

// C(m, n) = sum_k A(m, k) B(k, n) for member e = blockIdx.z, with
// A(m, k) = A[e ame + m sam + k sak] and B(k, n) = B[e bme + k sbk + n sbn]
// (A in FP32, B in FP32 or BF16: b_bf16).
struct GemmArgs {
  const void* A;
  long long sam, sak, ame;
  const void* B;
  long long sbk, sbn, bme;
  int b_bf16;
  int M, N, K;
  int epi;
  const float* bias;  // EPI_BIAS*: bias[e biasme + n]
  long long biasme;
  float* C;  // C[e cme + m ldc + n]
  long long ldc, cme;
  float* H;  // EPI_BIAS_GELU: GELU(C) at H[e hme + m ldh + n]
  long long ldh, hme;
  const float* Zp;  // EPI_GELU_GRAD: C *= GELU'(Zp[e zpme + m ldzp + n])
  long long ldzp, zpme;
};

// ---- tensor-core products ----------------------------------------------------
constexpr int kMmM = 128, kMmN = 128;   // output tile
constexpr int kMmParts = 3;             // BF16 parts of an FP32 operand
constexpr int kMmThreads = 192;         // warps 0-3 epilogue, 4 TMA producer, 5 MMA issuer
constexpr int kMmStages = 2;
constexpr int kMmTmemCols = kMmN;       // one FP32 accumulator column per output column
constexpr uint32_t kMmIdesc = hk::umma_idesc_bf16(kMmM, kMmN);
static_assert(hk::kTmaSlab == 64, "one K slab is one 128-byte TMA box row");

__host__ __device__ constexpr int mm_a_plane() { return kMmM * 64 * 2; }  // 16 KB
__host__ __device__ constexpr int mm_b_plane() { return kMmN * 64 * 2; }  // 16 KB
__host__ __device__ constexpr int mm_stage(int sa, int sb) { return sa * mm_a_plane() + sb * mm_b_plane(); }
size_t mm_smem_bytes() { return (size_t)kMmStages * mm_stage(kMmParts, kMmParts) + 1024; }

// Parts of an operand view for the tensor cores: X(r, k) = X[e xme + r srow
// + k sk] (FP32 or BF16) for r < R, k < K, written as S BF16 parts in
// K-major planes P[e][j][r][ldk] (zero for k >= K).  Part j is the BF16
// rounding of X minus parts 0..j-1 (exact in FP32).
template <typename T>
__global__ void to_parts_kernel(const T* X, long long srow, long long sk, long long xme, int R, int K, int S,
                                bf16* P, int ldk) {
  const int e = blockIdx.y;
  const long long n = (long long)R * ldk;
  bf16* out = P + (long long)e * S * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ldk), k = (int)(idx % ldk);
    float v = (k < K) ? ld(X + e * xme + r * srow + k * sk) : 0.f;
    for (int j = 0; j < S; ++j) {
      const bf16 q = __float2bfloat16_rn(v);
      out[(long long)j * n + idx] = q;
      v -= __bfloat162float(q);
    }
  }
}

struct MmArgs {
  int M, N, nslab;  // output M x N, K in slabs of 64 (zero-padded)
  int SA, SB;       // parts of A and B
  int a_shared;     // every member reads member 0's A parts
  GemmArgs g;       // epilogue and output layout (A/B fields unused)
  int* err;         // expiry record of a bounded wait
};

// C(m, n) = sum_k A(m, k) B(n, k) for member e = blockIdx.z, over the part
// pairs (i, j), i + j < max(SA, SB), all into one FP32 accumulator; one CTA
// per 128 x 128 output tile.  Warp 4 streams the K slabs of the parts into
// a two-stage ring with TMA, warp 5 issues the MMAs, warps 0-3 read the
// accumulator back (a thread per row) and apply the epilogue.  Waits are
// bounded like those of the complex product kernel.
__global__ void __launch_bounds__(kMmThreads, 1)
    mlp_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, MmArgs a) {
  extern __shared__ unsigned char mm_smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kMmStages], empty_bar[kMmStages], acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(mm_smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kMmM, n0 = blockIdx.x * kMmN, e = blockIdx.z;
  const int SA = a.SA, SB = a.SB, smax = SA > SB ? SA : SB;
  const int sbytes = mm_stage(SA, SB);
  if (threadIdx.x == 0) {
    for (int st = 0; st < kMmStages; ++st) {
      hk::mbar_init(&full_bar[st], 1);
      hk::mbar_init(&empty_bar[st], 1);
    }
    hk::mbar_init(&acc_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(hk::smem_u32(&tmem_slot)),
                 "r"(kMmTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  hk::tc_fence_before();
  __syncthreads();
  hk::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* vabort = &abort_flag;
  const int za = (a.a_shared ? 0 : e) * SA, zb = e * SB;

  if (warp == 4) {
    if (lane == 0) {
      int issued = 0;
      for (int st = 0; st < a.nslab; ++st) {
        const int slot = st % kMmStages;
        if (st >= kMmStages && !hk::mbar_wait(&empty_bar[slot], ((st / kMmStages) - 1) & 1, vabort, a.err)) break;
        unsigned char* base = smem + (size_t)slot * sbytes;
        hk::mbar_expect_tx(&full_bar[slot], (uint32_t)sbytes);
        for (int j = 0; j < SA; ++j)
          hk::tma_load_3d(base + (size_t)j * mm_a_plane(), &mapA, &full_bar[slot], st * 64, m0, za + j);
        for (int j = 0; j < SB; ++j)
          hk::tma_load_3d(base + (size_t)SA * mm_a_plane() + (size_t)j * mm_b_plane(), &mapB, &full_bar[slot], st * 64,
                          n0, zb + j);
        issued = st + 1;
      }
      for (int st = issued > kMmStages ? issued - kMmStages : 0; st < issued; ++st) {
        const uint64_t t0 = global_ns();
        while (!hk::mbar_try_wait(&full_bar[st % kMmStages], (st / kMmStages) & 1))
          if (global_ns() - t0 > hk::kTcWaitNs) break;
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      for (int st = 0; st < a.nslab; ++st) {
        const int slot = st % kMmStages;
        if (!hk::mbar_wait(&full_bar[slot], (st / kMmStages) & 1, vabort, a.err)) break;
        hk::tc_fence_after();
        const uint32_t abase = hk::smem_u32(smem + (size_t)slot * sbytes);
        const uint32_t bbase = abase + (uint32_t)(SA * mm_a_plane());
        bool first = (st == 0);
        for (int i = 0; i < SA; ++i)
          for (int j = 0; j < SB; ++j) {
            if (i + j >= smax) continue;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = hk::sw128_desc(abase + (uint32_t)(i * mm_a_plane() + kk * 32));
              const uint64_t bd = hk::sw128_desc(bbase + (uint32_t)(j * mm_b_plane() + kk * 32));
              hk::umma(tmem, ad, bd, kMmIdesc, first ? 0u : 1u);
              first = false;
            }
          }
        hk::umma_commit(&empty_bar[slot]);
      }
      hk::umma_commit(&acc_bar);
    }
  } else {
    const bool ok = hk::mbar_wait(&acc_bar, 0, vabort, a.err);
    hk::tc_fence_after();
    const int m = m0 + 32 * warp + lane;
    const GemmArgs& g = a.g;
    if (ok && !*vabort) {
#pragma unroll 1
      for (int h = 0; h < kMmN / 16; ++h) {
        float v[16];
        hk::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * h), v);
        if (m >= a.M) continue;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int n = n0 + 16 * h + q;
          if (n >= a.N) continue;
          float x = v[q];
          if (g.epi == EPI_BIAS || g.epi == EPI_BIAS_GELU) x += g.bias[e * g.biasme + n];
          if (g.epi == EPI_GELU_GRAD) x *= gelu_grad(g.Zp[e * g.zpme + (long long)m * g.ldzp + n]);
          g.C[e * g.cme + (long long)m * g.ldc + n] = x;
          if (g.epi == EPI_BIAS_GELU) g.H[e * g.hme + (long long)m * g.ldh + n] = gelu(x);
        }
      }
    }
  }
  hk::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    hk::tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMmTmemCols) : "memory");
  }
}

// db[e][n] = sum_m G[e][m][n] (bias gradient; one thread per column).
__global__ void colsum_kernel(const float* G, long long ldg, long long gme, int M, int N, float* db,
                              long long dbme) {
  const int e = blockIdx.y;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float* g = G + e * gme + n;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += g[m * ldg];
  db[e * dbme + n] = s;
}

// Training batch of each member: normalised inputs and targets gathered
// from the stored data set; the step number comes from counter[0].
__global__ void gather_kernel(const int* idx, const int* counter, int members, int batch, const double* xd,
                              const double* yd, int n_in, int n_out, const double* stats, float* X0, long long xme,
                              float* T, long long tme) {
  const int e = blockIdx.y;
  const int it = counter ? counter[0] : 0;
  const int* id = idx + ((long long)it * members + e) * batch;
  const double *xmu = stats, *xsd = stats + n_in, *ymu = stats + 2 * n_in, *ysd = ymu + n_out;
  const int w = n_in + n_out;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < batch * w; q += gridDim.x * blockDim.x) {
    const int b = q / w, c = q % w;
    const long long s = id[b];
    if (c < n_in)
      X0[e * xme + (long long)b * n_in + c] = (float)((xd[s * n_in + c] - xmu[c]) / xsd[c]);
    else {
      const int o = c - n_in;
      T[e * tme + (long long)b * n_out + o] = (float)((yd[s * n_out + o] - ymu[o]) / ysd[o]);
    }
  }
}

// G = 2 (Y - T) / (batch n_out); loss[it][e] += mean squared error.
__global__ void loss_kernel(const float* Y, long long yme, const float* T, long long tme, int batch, int n_out,
                            float* G, long long gme, const int* counter, int members, float* loss) {
  const int e = blockIdx.y;
  const int total = batch * n_out;
  const float inv = 1.0f / (float)total;
  float part = 0.f;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int b = q / n_out, o = q % n_out;
    const float r = Y[e * yme + q] - T[e * tme + q];
    G[e * gme + (long long)b * n_out + o] = 2.0f * r * inv;
    part += r * r;
  }
  __shared__ float red[32];
  for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) {
      const int it = counter ? counter[0] : 0;
      atomicAdd(loss + (long long)it * members + e, v * inv);
    }
  }
}

// Adam on the FP32 master parameters; refreshes the BF16 copies.  counter:
// [0] step of this call (learning-rate table index), [1] steps taken so far.
__global__ void adam_kernel(float* w, float* m, float* v, const float* g, bf16* wb, long long total,
                            const float* lr_tab, const int* counter) {
  __shared__ float sc[3];
  if (threadIdx.x == 0) {
    const int t = counter[1] + 1;
    sc[0] = lr_tab[counter[0]];
    sc[1] = (float)(1.0 - pow((double)kBeta1, (double)t));
    sc[2] = (float)(1.0 - pow((double)kBeta2, (double)t));
  }
  __syncthreads();
  const float lr = sc[0], bc1 = sc[1], bc2 = sc[2];
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total;
       j += (long long)gridDim.x * blockDim.x) {
    const float gj = g[j];
    const float mj = kBeta1 * m[j] + (1.0f - kBeta1) * gj;
    const float vj = kBeta2 * v[j] + (1.0f - kBeta2) * gj * gj;
    m[j] = mj;
    v[j] = vj;
    const float wj = w[j] - lr * (mj / bc1) / (sqrtf(vj / bc2) + kAdamEps);
    w[j] = wj;
    wb[j] = __float2bfloat16_rn(wj);
  }
}

__global__ void step_counter_kernel(int* counter) {
  counter[0] += 1;
  counter[1] += 1;
}

__global__ void to_bf16_kernel(const float* w, bf16* wb, long long total) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total;
       j += (long long)gridDim.x * blockDim.x)
    wb[j] = __float2bfloat16_rn(w[j]);
}

// Column mean and population standard deviation (two passes, FP64) of the
// data set; one block per column of [x | y].  Constant columns get sd = 1.
__global__ void column_stats_kernel(const double* xd, const double* yd, int ns, int n_in, int n_out,
                                    double* stats) {
  const int c = blockIdx.x;
  const double* col = c < n_in ? xd + c : yd + (c - n_in);
  const int ld = c < n_in ? n_in : n_out;
  __shared__ double red[32];
  __shared__ double mean_sh;
  auto block_sum = [&](double v) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
  };
  double s = 0.0;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) s += col[(long long)i * ld];
  s = block_sum(s);
  if (threadIdx.x == 0) mean_sh = s / ns;
  __syncthreads();
  const double mu = mean_sh;
  double q = 0.0;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const double r = col[(long long)i * ld] - mu;
    q += r * r;
  }
  q = block_sum(q);
  if (threadIdx.x == 0) {
    const double sd = sqrt(q / ns);
    const int o = c < n_in ? c : c - n_in;
    double* base = c < n_in ? stats : stats + 2 * n_in;
    const int w = c < n_in ? n_in : n_out;
    base[o] = mu;
    base[w + o] = sd > 0.0 ? sd : 1.0;
  }
}

// Queries to normalised network inputs (shared by every member).
__global__ void normalize_kernel(const double* x, int nq, int n_in, const double* stats, float* X0) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq * n_in; q += gridDim.x * blockDim.x) {
    const int c = q % n_in;
    X0[q] = (float)((x[q] - stats[c]) / stats[n_in + c]);
  }
}

// Per query b: each member's answer in physical units,
// y_m = base + scale (mu + sd net_m) (base 0 and scale 1 when absent), the
// member mean ybar and the error bound kappa ||s||_2 / ||ybar||_2, s the
// per-output standard deviation of y_m over the members.
__global__ void ensemble_kernel(const float* Y, long long yme, int members, int nq, int n_out,
                                const double* ystats, const double* base, const double* scale, double kappa,
                                double* yout, double* bound, double* ymem) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nq) return;
  const double *mu = ystats, *sd = ystats + n_out;
  const double sc = scale ? scale[b] : 1.0;
  double yy = 0.0, ss = 0.0;
  for (int o = 0; o < n_out; ++o) {
    const double b0 = base ? base[(long long)b * n_out + o] : 0.0;
    double s1 = 0.0;
    for (int e = 0; e < members; ++e) {
      const double v = b0 + sc * (mu[o] + sd[o] * (double)Y[e * yme + (long long)b * n_out + o]);
      s1 += v;
      if (ymem) ymem[((long long)e * nq + b) * n_out + o] = v;
    }
    const double ybar = s1 / members;
    double s2 = 0.0;
    for (int e = 0; e < members; ++e) {
      const double r = b0 + sc * (mu[o] + sd[o] * (double)Y[e * yme + (long long)b * n_out + o]) - ybar;
      s2 += r * r;
    }
    yout[(long long)b * n_out + o] = ybar;
    yy += ybar * ybar;
    ss += s2 / members;
  }
  bound[b] = yy > 0.0 ? kappa * sqrt(ss / yy) : (ss > 0.0 ? INFINITY : 0.0);
}

int blocks_for(long long n, int threads, int cap = 1024) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

struct hopf_mlp {
  hopf_ctx* ctx = nullptr;
  hopf_mlp_params p{};
  int L = 0;                   // linear layers
  std::vector<int> dims;       // L + 1 widths
  std::vector<long long> woff, boff;
  long long P = 0;             // parameters per member
  int gmax = 0;                // widest layer
  cudaStream_t s = nullptr;    // own stream (graph capture)
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  bf16* wb = nullptr;
  std::vector<float*> X, Z;    // per layer [members][max_batch][width]
  float *G0 = nullptr, *G1 = nullptr, *T = nullptr;
  int* counter = nullptr;      // [2]
  double* stats = nullptr;     // [2 (n_in + n_out)]
  bool have_stats = false;
  double *xd = nullptr, *yd = nullptr;
  int ns = 0;
  int* idx = nullptr;
  long long idx_cap = 0;
  float *lr = nullptr, *loss = nullptr;
  long long it_cap = 0;
  double *qx = nullptr, *qy = nullptr, *qb = nullptr, *qm = nullptr, *qbase = nullptr, *qscale = nullptr;
  bf16 *pa = nullptr, *pb = nullptr;  // BF16 parts of the tensor-core products' operands
  size_t pa_elems = 0, pb_elems = 0;
  std::vector<void*> allocs;
};

namespace {

hopf_status mfail(hopf_mlp* m, hopf_status st, const char* fmt, ...) {
  if (m && m->ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    hopf_internal_set_error(m->ctx, buf);
  }
  return st;
}

#define MCK(expr)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      cudaGetLastError();                                                                  \
      return mfail(mm, e_ == cudaErrorMemoryAllocation ? HOPF_ENOMEM : HOPF_ECUDA, "%s: %s", #expr, \
                   cudaGetErrorString(e_));                                                \
    }                                                                                      \
  } while (0)

template <class T>
cudaError_t malloc_track(hopf_mlp* mm, T** p, size_t count) {
  *p = nullptr;
  cudaError_t e = hk::dev_alloc((void**)p, (count ? count : 1) * sizeof(T));
  if (e == cudaSuccess) mm->allocs.push_back(*p);
  return e;
}

bool valid_params(const hopf_mlp_params* p) {
  return p && p->n_in >= 1 && p->n_in <= kMaxDim && p->n_out >= 1 && p->n_out <= kMaxDim && p->depth >= 0 &&
         p->depth <= 64 && (p->depth == 0 || (p->width >= 1 && p->width <= kMaxDim)) && p->members >= 1 &&
         p->members <= kMaxMembers && p->max_batch >= 1 && p->max_batch <= (1 << 20);
}

void layer_dims(const hopf_mlp_params& p, std::vector<int>& dims) {
  dims.clear();
  dims.push_back(p.n_in);
  for (int l = 0; l < p.depth; ++l) dims.push_back(p.width);
  dims.push_back(p.n_out);
}

int rup64(long long x) { return (int)((x + 63) / 64 * 64); }

// The product kernel's shared-memory limit, raised once per process (before
// any stream capture: hopf_mlp_create).
cudaError_t mm_prepare() {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, []() {
    attr = cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mm_smem_bytes());
  });
  return attr;
}

// Parts scratch for a model (elements of each buffer): A operands are the
// activations (batch x width, forward and dX) or the output gradients
// transposed (width x batch, dW); B operands the weights (one part) or the
// activations transposed (dW).
void parts_sizes(const hopf_mlp_params& p, const std::vector<int>& dims, size_t* pa, size_t* pb) {
  const long long mb = p.max_batch;
  int dmax = 0;
  for (int d : dims) dmax = std::max(dmax, d);
  const size_t a1 = (size_t)mb * rup64(dmax), a2 = (size_t)dmax * rup64(mb);
  *pa = (size_t)p.members * kMmParts * std::max(a1, a2);
  *pb = (size_t)p.members * kMmParts * (size_t)dmax * rup64(std::max<long long>(mb, dmax));
}

// C = A B (GemmArgs layout) on the tensor cores: the operands are cut into
// BF16 parts (three for FP32, one for BF16) in K-major planes, then one
// tensor-core launch over all members.  a_shared: every member reads member
// 0's A (ame = 0).
cudaError_t launch_gemm(hopf_mlp* mm, const GemmArgs& g, int members) {
  const int M = g.M, N = g.N, K = g.K;
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int ldk = rup64(K);
  const int SA = kMmParts, SB = g.b_bf16 ? 1 : kMmParts;
  const int a_shared = g.ame == 0 && members > 1;
  const int ma = a_shared ? 1 : members;
  if ((size_t)ma * SA * M * ldk > mm->pa_elems || (size_t)members * SB * N * ldk > mm->pb_elems)
    return cudaErrorInvalidValue;
  cudaStream_t s = mm->s;
  // A(m, k) = A[e ame + m sam + k sak]; B as rows n, K-values k: B[e bme + n sbn + k sbk]
  to_parts_kernel<float><<<dim3(blocks_for((long long)M * ldk, 256, 1024), ma), 256, 0, s>>>(
      static_cast<const float*>(g.A), g.sam, g.sak, g.ame, M, K, SA, mm->pa, ldk);
  if (g.b_bf16)
    to_parts_kernel<bf16><<<dim3(blocks_for((long long)N * ldk, 256, 1024), members), 256, 0, s>>>(
        static_cast<const bf16*>(g.B), g.sbn, g.sbk, g.bme, N, K, SB, mm->pb, ldk);
  else
    to_parts_kernel<float><<<dim3(blocks_for((long long)N * ldk, 256, 1024), members), 256, 0, s>>>(
        static_cast<const float*>(g.B), g.sbn, g.sbk, g.bme, N, K, SB, mm->pb, ldk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap mapA, mapB;
  e = hk::plane_map(&mapA, mm->pa, ldk, ldk, M, ma * SA, kMmM);
  if (e == cudaSuccess) e = hk::plane_map(&mapB, mm->pb, ldk, ldk, N, members * SB, kMmN);
  if (e != cudaSuccess) return e;
  MmArgs args{};
  args.M = M;
  args.N = N;
  args.nslab = ldk / 64;
  args.SA = SA;
  args.SB = SB;
  args.a_shared = a_shared;
  args.g = g;
  args.err = hopf_internal_wait_record(mm->ctx);
  const dim3 grid((N + kMmN - 1) / kMmN, (M + kMmM - 1) / kMmM, members);
  mlp_tc_kernel<<<grid, kMmThreads, mm_smem_bytes(), s>>>(mapA, mapB, args);
  return cudaGetLastError();
}

// Forward pass over `batch` rows; x0_shared: every member reads member 0's
// input rows (inference), else each member has its own (training).
cudaError_t forward(hopf_mlp* mm, int batch, bool x0_shared) {
  const long long mb = mm->p.max_batch, P = mm->P;
  for (int l = 0; l < mm->L; ++l) {
    const int fi = mm->dims[l], fo = mm->dims[l + 1];
    GemmArgs a{};
    a.A = mm->X[l];
    a.sam = fi;
    a.sak = 1;
    a.ame = (l == 0 && x0_shared) ? 0 : mb * fi;
    a.B = mm->wb + mm->woff[l];
    a.sbk = 1;
    a.sbn = fi;
    a.bme = P;
    a.b_bf16 = 1;
    a.M = batch;
    a.N = fo;
    a.K = fi;
    a.bias = mm->w + mm->boff[l];
    a.biasme = P;
    a.C = mm->Z[l];
    a.ldc = fo;
    a.cme = mb * fo;
    if (l < mm->L - 1) {
      a.epi = EPI_BIAS_GELU;
      a.H = mm->X[l + 1];
      a.ldh = fo;
      a.hme = mb * fo;
    } else {
      a.epi = EPI_BIAS;
    }
    cudaError_t e = launch_gemm(mm, a, mm->p.members);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Gradient of the loss with respect to every parameter; G0 holds dL/dY.
cudaError_t backward(hopf_mlp* mm, int batch) {
  const long long mb = mm->p.max_batch, P = mm->P, gme = mb * mm->gmax;
  float* Gc = mm->G0;
  float* Gn = mm->G1;
  for (int l = mm->L - 1; l >= 0; --l) {
    const int fi = mm->dims[l], fo = mm->dims[l + 1];
    GemmArgs a{};  // dW[o][i] = sum_b G[b][o] X[b][i]
    a.A = Gc;
    a.sam = 1;
    a.sak = fo;
    a.ame = gme;
    a.B = mm->X[l];
    a.sbk = fi;
    a.sbn = 1;
    a.bme = mb * fi;
    a.M = fo;
    a.N = fi;
    a.K = batch;
    a.epi = EPI_STORE;
    a.C = mm->g + mm->woff[l];
    a.ldc = fi;
    a.cme = P;
    cudaError_t e = launch_gemm(mm, a, mm->p.members);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<dim3((fo + 255) / 256, mm->p.members), 256, 0, mm->s>>>(Gc, fo, gme, batch, fo,
                                                                            mm->g + mm->boff[l], P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (l == 0) break;
    GemmArgs b{};  // Gn[b][i] = (sum_o G[b][o] W[o][i]) GELU'(Z_{l-1}[b][i])
    b.A = Gc;
    b.sam = fo;
    b.sak = 1;
    b.ame = gme;
    b.B = mm->wb + mm->woff[l];
    b.sbk = fi;
    b.sbn = 1;
    b.bme = P;
    b.b_bf16 = 1;
    b.M = batch;
    b.N = fi;
    b.K = fo;
    b.epi = EPI_GELU_GRAD;
    b.C = Gn;
    b.ldc = fi;
    b.cme = gme;
    b.Zp = mm->Z[l - 1];
    b.ldzp = fi;
    b.zpme = mb * fi;
    if ((e = launch_gemm(mm, b, mm->p.members)) != cudaSuccess) return e;
    std::swap(Gc, Gn);
  }
  return cudaSuccess;
}

// One training step (or, with lr_tab == nullptr, one gradient evaluation):
// gather, forward, loss, backward, Adam, counter.
cudaError_t train_step(hopf_mlp* mm, int batch, const int* idx, float* loss, bool update) {
  const int M = mm->p.members;
  const long long mb = mm->p.max_batch;
  cudaError_t e;
  gather_kernel<<<dim3(blocks_for((long long)batch * (mm->p.n_in + mm->p.n_out), 256, 64), M), 256, 0, mm->s>>>(
      idx, mm->counter, M, batch, mm->xd, mm->yd, mm->p.n_in, mm->p.n_out, mm->stats, mm->X[0], mb * mm->p.n_in,
      mm->T, mb * mm->p.n_out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = forward(mm, batch, false)) != cudaSuccess) return e;
  loss_kernel<<<dim3(blocks_for((long long)batch * mm->p.n_out, 256, 64), M), 256, 0, mm->s>>>(
      mm->Z[mm->L - 1], mb * mm->p.n_out, mm->T, mb * mm->p.n_out, batch, mm->p.n_out, mm->G0,
      mb * mm->gmax, mm->counter, M, loss);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = backward(mm, batch)) != cudaSuccess) return e;
  if (!update) return cudaSuccess;
  const long long total = (long long)M * mm->P;
  adam_kernel<<<blocks_for(total, 256, 2048), 256, 0, mm->s>>>(mm->w, mm->m, mm->v, mm->g, mm->wb, total, mm->lr,
                                                                mm->counter);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  step_counter_kernel<<<1, 1, 0, mm->s>>>(mm->counter);
  return cudaGetLastError();
}

// Orders the library stream after the context's stream.
cudaError_t join_ctx(hopf_mlp* mm) {
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(ev, hopf_internal_stream(mm->ctx));
  if (e == cudaSuccess) e = cudaStreamWaitEvent(mm->s, ev, 0);
  cudaEventDestroy(ev);
  return e;
}

bool finite_all(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

}  // namespace

extern "C" {

hopf_status hopf_mlp_param_count(const hopf_mlp_params* p, long long* P) {
  if (!valid_params(p) || !P) return HOPF_EINVAL;
  std::vector<int> dims;
  layer_dims(*p, dims);
  long long n = 0;
  for (size_t l = 0; l + 1 < dims.size(); ++l) n += (long long)dims[l] * dims[l + 1] + dims[l + 1];
  *P = n;
  return HOPF_OK;
}

void hopf_mlp_free(hopf_mlp* mm) {
  if (!mm) return;
  hk::live_add(-1);
  if (mm->s) cudaStreamSynchronize(mm->s);
  for (void* p : mm->allocs) hk::dev_free(p);
  if (mm->s) cudaStreamDestroy(mm->s);
  delete mm;
}

hopf_status hopf_mlp_create(hopf_ctx* ctx, const hopf_mlp_params* p, const float* init, hopf_mlp** out) {
  if (!ctx || !out) return HOPF_EINVAL;
  *out = nullptr;
  if (!valid_params(p) || !init) {
    hopf_internal_set_error(ctx, "hopf_mlp_create: bad arguments");
    return HOPF_EINVAL;
  }
  hopf_mlp* mm = new hopf_mlp;
  hk::live_add(1);  // hopf_mlp_free takes it back
  mm->ctx = ctx;
  mm->p = *p;
  layer_dims(*p, mm->dims);
  mm->L = (int)mm->dims.size() - 1;
  long long off = 0;
  for (int l = 0; l < mm->L; ++l) {
    mm->woff.push_back(off);
    off += (long long)mm->dims[l] * mm->dims[l + 1];
    mm->boff.push_back(off);
    off += mm->dims[l + 1];
    mm->gmax = std::max(mm->gmax, mm->dims[l + 1]);
  }
  mm->P = off;
  const int M = p->members;
  const long long mb = p->max_batch, tot = (long long)M * mm->P;
  for (size_t i = 0; i < (size_t)tot; ++i)
    if (!std::isfinite(init[i])) {
      hk::live_add(-1);
      delete mm;
      hopf_internal_set_error(ctx, "hopf_mlp_create: non-finite initial parameter");
      return HOPF_EINVAL;
    }
  auto fail_free = [&](hopf_status st) {
    hopf_mlp_free(mm);
    return st;
  };
  hopf_status st = HOPF_OK;
  do {
    cudaError_t e = mm_prepare();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&mm->s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->w, tot);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->m, tot);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->v, tot);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->g, tot);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->wb, tot);
    mm->X.assign(mm->L, nullptr);
    mm->Z.assign(mm->L, nullptr);
    for (int l = 0; l < mm->L && e == cudaSuccess; ++l) {
      e = malloc_track(mm, &mm->X[l], (size_t)M * mb * mm->dims[l]);
      if (e == cudaSuccess) e = malloc_track(mm, &mm->Z[l], (size_t)M * mb * mm->dims[l + 1]);
    }
    if (e == cudaSuccess) e = malloc_track(mm, &mm->G0, (size_t)M * mb * mm->gmax);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->G1, (size_t)M * mb * mm->gmax);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->T, (size_t)M * mb * p->n_out);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->counter, 2);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->stats, (size_t)2 * (p->n_in + p->n_out));
    if (e == cudaSuccess) e = malloc_track(mm, &mm->qx, (size_t)mb * p->n_in);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->qy, (size_t)mb * p->n_out);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->qb, (size_t)mb);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->qm, (size_t)M * mb * p->n_out);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->qbase, (size_t)mb * p->n_out);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->qscale, (size_t)mb);
    parts_sizes(*p, mm->dims, &mm->pa_elems, &mm->pb_elems);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->pa, mm->pa_elems);
    if (e == cudaSuccess) e = malloc_track(mm, &mm->pb, mm->pb_elems);
    if (e == cudaSuccess) e = join_ctx(mm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mm->w, init, tot * sizeof(float), cudaMemcpyHostToDevice, mm->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mm->m, 0, tot * sizeof(float), mm->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mm->v, 0, tot * sizeof(float), mm->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mm->counter, 0, 2 * sizeof(int), mm->s);
    if (e == cudaSuccess) {
      to_bf16_kernel<<<blocks_for(tot, 256, 2048), 256, 0, mm->s>>>(mm->w, mm->wb, tot);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(mm->s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      hopf_internal_set_error(ctx, cudaGetErrorString(e));
      st = e == cudaErrorMemoryAllocation ? HOPF_ENOMEM : HOPF_ECUDA;
    }
  } while (0);
  if (st != HOPF_OK) return fail_free(st);
  *out = mm;
  return HOPF_OK;
}

hopf_status hopf_mlp_get_params(hopf_mlp* mm, float* out) {
  if (!mm || !out) return HOPF_EINVAL;
  MCK(cudaMemcpyAsync(out, mm->w, (size_t)mm->p.members * mm->P * sizeof(float), cudaMemcpyDeviceToHost, mm->s));
  MCK(cudaStreamSynchronize(mm->s));
  return HOPF_OK;
}

hopf_status hopf_mlp_set_data(hopf_mlp* mm, int nsamples, const double* x, const double* y, double* stats) {
  if (!mm) return HOPF_EINVAL;
  const int n_in = mm->p.n_in, n_out = mm->p.n_out;
  if (nsamples < 1 || !x || !y) return mfail(mm, HOPF_EINVAL, "hopf_mlp_set_data: bad arguments");
  if (!finite_all(x, (size_t)nsamples * n_in) || !finite_all(y, (size_t)nsamples * n_out))
    return mfail(mm, HOPF_EINVAL, "hopf_mlp_set_data: non-finite data");
  MCK(cudaStreamSynchronize(mm->s));
  if (nsamples > mm->ns) {
    for (double* p : {mm->xd, mm->yd}) {
      for (size_t i = 0; i < mm->allocs.size(); ++i)
        if (mm->allocs[i] == p) {
          hk::dev_free(p);
          mm->allocs.erase(mm->allocs.begin() + i);
          break;
        }
    }
    mm->xd = mm->yd = nullptr;
    mm->ns = 0;
    MCK(malloc_track(mm, &mm->xd, (size_t)nsamples * n_in));
    MCK(malloc_track(mm, &mm->yd, (size_t)nsamples * n_out));
  }
  mm->ns = nsamples;
  MCK(join_ctx(mm));
  MCK(cudaMemcpyAsync(mm->xd, x, (size_t)nsamples * n_in * sizeof(double), cudaMemcpyHostToDevice, mm->s));
  MCK(cudaMemcpyAsync(mm->yd, y, (size_t)nsamples * n_out * sizeof(double), cudaMemcpyHostToDevice, mm->s));
  column_stats_kernel<<<n_in + n_out, 256, 0, mm->s>>>(mm->xd, mm->yd, nsamples, n_in, n_out, mm->stats);
  MCK(cudaGetLastError());
  if (stats)
    MCK(cudaMemcpyAsync(stats, mm->stats, (size_t)2 * (n_in + n_out) * sizeof(double), cudaMemcpyDeviceToHost,
                        mm->s));
  MCK(cudaStreamSynchronize(mm->s));
  mm->have_stats = true;
  return HOPF_OK;
}

namespace {

hopf_status check_idx(hopf_mlp* mm, long long count, const int* idx) {
  for (long long i = 0; i < count; ++i)
    if (idx[i] < 0 || idx[i] >= mm->ns) return mfail(mm, HOPF_EINVAL, "sample index %d outside [0, %d)", idx[i], mm->ns);
  return HOPF_OK;
}

hopf_status ensure_tables(hopf_mlp* mm, long long idx_count, long long iters) {
  if (idx_count > mm->idx_cap) {
    for (size_t i = 0; i < mm->allocs.size(); ++i)
      if (mm->allocs[i] == mm->idx) {
        hk::dev_free(mm->idx);
        mm->allocs.erase(mm->allocs.begin() + i);
        break;
      }
    mm->idx = nullptr;
    mm->idx_cap = 0;
    MCK(malloc_track(mm, &mm->idx, (size_t)idx_count));
    mm->idx_cap = idx_count;
  }
  if (iters > mm->it_cap) {
    for (float* p : {mm->lr, mm->loss})
      for (size_t i = 0; i < mm->allocs.size(); ++i)
        if (mm->allocs[i] == p) {
          hk::dev_free(p);
          mm->allocs.erase(mm->allocs.begin() + i);
          break;
        }
    mm->lr = mm->loss = nullptr;
    mm->it_cap = 0;
    MCK(malloc_track(mm, &mm->lr, (size_t)iters));
    MCK(malloc_track(mm, &mm->loss, (size_t)iters * mm->p.members));
    mm->it_cap = iters;
  }
  return HOPF_OK;
}

}  // namespace

hopf_status hopf_mlp_train(hopf_mlp* mm, int iters, int batch, const int* idx, const float* lr, float* loss) {
  if (!mm) return HOPF_EINVAL;
  if (!mm->have_stats || mm->ns < 1) return mfail(mm, HOPF_EINVAL, "hopf_mlp_train: no data set");
  if (iters < 0 || batch < 1 || batch > mm->p.max_batch || (iters > 0 && (!idx || !lr)))
    return mfail(mm, HOPF_EINVAL, "hopf_mlp_train: bad arguments");
  if (iters == 0) return HOPF_OK;
  const int M = mm->p.members;
  const long long nidx = (long long)iters * M * batch;
  if (hopf_status st = check_idx(mm, nidx, idx)) return st;
  for (int i = 0; i < iters; ++i)
    if (!std::isfinite(lr[i]) || lr[i] < 0.f) return mfail(mm, HOPF_EINVAL, "hopf_mlp_train: bad learning rate");
  MCK(cudaStreamSynchronize(mm->s));
  if (hopf_status st = ensure_tables(mm, nidx, iters)) return st;
  MCK(join_ctx(mm));
  MCK(cudaMemcpyAsync(mm->idx, idx, nidx * sizeof(int), cudaMemcpyHostToDevice, mm->s));
  MCK(cudaMemcpyAsync(mm->lr, lr, (size_t)iters * sizeof(float), cudaMemcpyHostToDevice, mm->s));
  MCK(cudaMemsetAsync(mm->loss, 0, (size_t)iters * M * sizeof(float), mm->s));
  MCK(cudaMemsetAsync(mm->counter, 0, sizeof(int), mm->s));  // step of this call; [1] keeps counting
  // Capture one step and replay it.
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  MCK(cudaStreamBeginCapture(mm->s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = train_step(mm, batch, mm->idx, mm->loss, true);
  cudaError_t e2 = cudaStreamEndCapture(mm->s, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  for (int i = 0; i < iters && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, mm->s);
  if (e == cudaSuccess && loss)
    e = cudaMemcpyAsync(loss, mm->loss, (size_t)iters * M * sizeof(float), cudaMemcpyDeviceToHost, mm->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mm->s);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  MCK(e);
  return hopf_internal_check_waits(mm->ctx);
}

hopf_status hopf_mlp_loss_grad(hopf_mlp* mm, int batch, const int* idx, float* loss, float* grad) {
  if (!mm) return HOPF_EINVAL;
  if (!mm->have_stats || mm->ns < 1) return mfail(mm, HOPF_EINVAL, "hopf_mlp_loss_grad: no data set");
  if (batch < 1 || batch > mm->p.max_batch || !idx || !loss || !grad)
    return mfail(mm, HOPF_EINVAL, "hopf_mlp_loss_grad: bad arguments");
  const int M = mm->p.members;
  if (hopf_status st = check_idx(mm, (long long)M * batch, idx)) return st;
  MCK(cudaStreamSynchronize(mm->s));
  if (hopf_status st = ensure_tables(mm, (long long)M * batch, 1)) return st;
  MCK(join_ctx(mm));
  MCK(cudaMemcpyAsync(mm->idx, idx, (size_t)M * batch * sizeof(int), cudaMemcpyHostToDevice, mm->s));
  MCK(cudaMemsetAsync(mm->loss, 0, (size_t)M * sizeof(float), mm->s));
  // counter == nullptr in the kernels means step 0 of the tables.
  const int M_ = M;
  const long long mb = mm->p.max_batch;
  gather_kernel<<<dim3(blocks_for((long long)batch * (mm->p.n_in + mm->p.n_out), 256, 64), M_), 256, 0, mm->s>>>(
      mm->idx, nullptr, M_, batch, mm->xd, mm->yd, mm->p.n_in, mm->p.n_out, mm->stats, mm->X[0], mb * mm->p.n_in,
      mm->T, mb * mm->p.n_out);
  MCK(cudaGetLastError());
  MCK(forward(mm, batch, false));
  loss_kernel<<<dim3(blocks_for((long long)batch * mm->p.n_out, 256, 64), M_), 256, 0, mm->s>>>(
      mm->Z[mm->L - 1], mb * mm->p.n_out, mm->T, mb * mm->p.n_out, batch, mm->p.n_out, mm->G0, mb * mm->gmax,
      nullptr, M_, mm->loss);
  MCK(cudaGetLastError());
  MCK(backward(mm, batch));
  MCK(cudaMemcpyAsync(loss, mm->loss, (size_t)M * sizeof(float), cudaMemcpyDeviceToHost, mm->s));
  MCK(cudaMemcpyAsync(grad, mm->g, (size_t)M * mm->P * sizeof(float), cudaMemcpyDeviceToHost, mm->s));
  MCK(cudaStreamSynchronize(mm->s));
  return hopf_internal_check_waits(mm->ctx);
}

hopf_status hopf_mlp_predict(hopf_mlp* mm, int nq, const double* x, const double* base, const double* scale,
                             double kappa, double* y, double* bound, double* members_y) {
  if (!mm) return HOPF_EINVAL;
  if (!mm->have_stats) return mfail(mm, HOPF_EINVAL, "hopf_mlp_predict: no normalisation statistics");
  if (nq < 0 || (nq > 0 && (!x || !y || !bound)) || !(kappa >= 0.0))
    return mfail(mm, HOPF_EINVAL, "hopf_mlp_predict: bad arguments");
  if (nq == 0) return HOPF_OK;
  const int n_in = mm->p.n_in, n_out = mm->p.n_out, M = mm->p.members;
  const int mb = mm->p.max_batch;
  MCK(join_ctx(mm));
  for (int q0 = 0; q0 < nq; q0 += mb) {
    const int c = std::min(mb, nq - q0);
    MCK(cudaMemcpyAsync(mm->qx, x + (size_t)q0 * n_in, (size_t)c * n_in * sizeof(double), cudaMemcpyHostToDevice,
                        mm->s));
    if (base)
      MCK(cudaMemcpyAsync(mm->qbase, base + (size_t)q0 * n_out, (size_t)c * n_out * sizeof(double),
                          cudaMemcpyHostToDevice, mm->s));
    if (scale)
      MCK(cudaMemcpyAsync(mm->qscale, scale + q0, (size_t)c * sizeof(double), cudaMemcpyHostToDevice, mm->s));
    normalize_kernel<<<blocks_for((long long)c * n_in, 256), 256, 0, mm->s>>>(mm->qx, c, n_in, mm->stats,
                                                                               mm->X[0]);
    MCK(cudaGetLastError());
    MCK(forward(mm, c, true));
    ensemble_kernel<<<blocks_for(c, 128, 1 << 20), 128, 0, mm->s>>>(
        mm->Z[mm->L - 1], (long long)mb * n_out, M, c, n_out, mm->stats + 2 * n_in, base ? mm->qbase : nullptr,
        scale ? mm->qscale : nullptr, kappa, mm->qy, mm->qb, members_y ? mm->qm : nullptr);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(y + (size_t)q0 * n_out, mm->qy, (size_t)c * n_out * sizeof(double), cudaMemcpyDeviceToHost,
                        mm->s));
    MCK(cudaMemcpyAsync(bound + q0, mm->qb, (size_t)c * sizeof(double), cudaMemcpyDeviceToHost, mm->s));
    if (members_y)
      for (int e = 0; e < M; ++e)
        MCK(cudaMemcpyAsync(members_y + ((size_t)e * nq + q0) * n_out, mm->qm + (size_t)e * c * n_out,
                            (size_t)c * n_out * sizeof(double), cudaMemcpyDeviceToHost, mm->s));
    MCK(cudaStreamSynchronize(mm->s));
  }
  return hopf_internal_check_waits(mm->ctx);
}

}  // extern "C"
