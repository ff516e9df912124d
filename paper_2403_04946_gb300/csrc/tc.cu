// Complex products on the tensor cores (tcgen05) with FP64-class accuracy.
//
// The mixed-precision rounding (App. A, Alg. 2 / Alg. 4: the QR trailing
// updates, the Q applications and the merges of the orthogonalisation sweep)
// needs products accurate to about 1e-12 of |A||B|, far beyond one BF16 or
// TF32 product.  Each operand is therefore cut into S digit planes
// (Ozaki-style splitting): per row r and per K-chunk, a power-of-two scale
// 2^e[r] brings the row below 1 in magnitude, and
//     x 2^-e = sum_j q_j 2^(-7-8j),   q_j integers with |q_j| <= 128,
// each q_j exactly representable in BF16.  A product of two digits is an
// integer below 2^14 in magnitude, so a K-chunk of at most 192 products per
// digit pair, summed over the pairs (i, j) of one level L = i + j (L + 1 <= 5
// pairs), stays below 2^24: the FP32 accumulation in tensor memory is exact.
// Levels L < S are kept (S (S + 1) / 2 digit products per real product); the
// dropped pairs weigh about S 2^(-8S) of |A||B| (5 digits: ~5e-12).
//
// Complex products use three real products (3M):
//     T1 = Ar Br,  T2 = Ai Bi,  T3 = (Ar + Ai)(Br + Bi),
//     C = (T1 - T2) + i (T3 - T1 - T2),
// each of Ar, Ai, Ar + Ai (and the same for B) split with its own scales.
//
// The product kernel: one CTA per 128 x 32 output tile and K-chunk.  Warp 8
// streams digit slabs (64 K-values, 128 B per row, 128-byte swizzle) into a
// two-stage shared-memory ring with TMA (cp.async.bulk.tensor); warp 9 issues
// tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) into 15 accumulators
// (3 products x 5 levels x 32 columns) in tensor memory, one MMA per A digit
// plane covering all its levels; warps 0-7 (two per tensor-memory lane
// quadrant, 16 columns each) read the accumulators back (tcgen05.ld),
// combine levels, scales and the 3M terms in double-float, and write the
// complex result (overwritten, added, or as a per-chunk partial that a
// reduction kernel sums in a fixed order).
//
// Every wait is bounded (2 s of wall time): on expiry the kernel records
// the error in the grid-barrier record the host checks (HOPF_ETIMEOUT),
// stops issuing work, waits (bounded) for what it issued, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "kernels.h"
#include "tcgen05.cuh"

namespace hk {

namespace {

constexpr int kTcM = 128;        // rows of an output tile (one TMEM lane each)
constexpr int kTcN = 32;         // columns of an output tile
constexpr int kSlab = 64;        // K-values per digit slab (128 bytes of BF16)
constexpr int kMaxDigits = 5;    // 3 products x 5 levels x 32 columns = 480 TMEM columns
constexpr int kTmemCols = 512;
constexpr int kStages = 2;
constexpr int kTcThreads = 320;  // warps 0-7 epilogue, 8 producer, 9 MMA
constexpr uint64_t kWaitNs = kTcWaitNs;
static_assert(kTmaSlab == 64, "digit slabs are one 128-byte TMA box row");

__host__ __device__ constexpr int a_plane_bytes() { return kTcM * kSlab * 2; }  // 16 KB
__host__ __device__ constexpr int b_plane_bytes() { return kTcN * kSlab * 2; }  // 4 KB
__host__ __device__ int stage_bytes(int S) { return S * (a_plane_bytes() + b_plane_bytes()); }
size_t tc_smem_bytes(int S) { return (size_t)kStages * stage_bytes(S) + 1024; }



struct TcArgs {
  int M, N, K, S, Kc, nchunks;
  const int* eA;  // [3][nchunks][M] scale exponents of the A digits
  const int* eB;  // [3][nchunks][N]
  cplx* out;      // out[z * zstride + m + ldo * n]
  long long ldo, zstride;
  int alpha_exp, alpha_neg;  // alpha = (-1)^alpha_neg 2^alpha_exp: out = alpha * result (+ out if accumulate)
  int accumulate;
  int* err;       // expiry record (the context's grid-barrier err field)
};

__global__ void __launch_bounds__(kTcThreads, 1)
    tc_zgemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int eb_sh[3][kTcN];
  // 1024-byte aligned stage ring (the swizzle atoms need it)
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int S = a.S;
  const int sbytes = stage_bytes(S);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // N-tiles fastest: the CTAs that share an A-tile (the large digit planes)
  // run together and find it in L2
  const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * kTcN, z = blockIdx.z;
  const int k_begin = z * a.Kc;
  const int k_len = min(a.Kc, a.K - k_begin);
  const int nslab = (k_len + kSlab - 1) / kSlab;
  const int nstage = 3 * nslab;  // (slab, product) pairs

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* vabort = &abort_flag;

  if (warp == 8) {
    // ---- producer: one (slab, product) stage at a time ------------------
    if (lane == 0) {
      int issued = 0;
      for (int st = 0; st < nstage; ++st) {
        const int slot = st % kStages;
        if (st >= kStages && !mbar_wait(&empty_bar[slot], ((st / kStages) - 1) & 1, vabort, a.err)) break;
        const int c = st % 3, slab = st / 3;
        const int k0 = k_begin + slab * kSlab;
        unsigned char* base = smem + (size_t)slot * sbytes;
        mbar_expect_tx(&full_bar[slot], (uint32_t)sbytes);
        for (int j = 0; j < S; ++j) {
          tma_load_3d(base + (size_t)j * a_plane_bytes(), &mapA, &full_bar[slot], k0, m0, c * S + j);
          tma_load_3d(base + (size_t)S * a_plane_bytes() + (size_t)j * b_plane_bytes(), &mapB, &full_bar[slot], k0, n0,
                      c * S + j);
        }
        issued = st + 1;
      }
      // before leaving, every issued copy has landed (bounded): the stage
      // ring must not be written after the CTA exits
      for (int st = max(0, issued - kStages); st < issued; ++st) {
        uint64_t t0 = global_ns();
        while (!mbar_try_wait(&full_bar[st % kStages], (st / kStages) & 1))
          if (global_ns() - t0 > kWaitNs) break;
      }
    }
  } else if (warp == 9) {
    // ---- MMA issuer -------------------------------------------------------
    if (lane == 0) {
      for (int st = 0; st < nstage; ++st) {
        const int slot = st % kStages;
        if (!mbar_wait(&full_bar[slot], (st / kStages) & 1, vabort, a.err)) break;
        tc_fence_after();
        const int c = st % 3, slab = st / 3;
        const uint32_t abase = smem_u32(smem + (size_t)slot * sbytes);
        const uint64_t a0 = sw128_desc(abase), b0 = sw128_desc(abase + (uint32_t)(S * a_plane_bytes()));
        // A digit plane i against B planes 0 .. S-1-i in one product: the B
        // planes lie one after another (32 rows each), so together they are
        // one (S - i) x 32-row operand whose output columns are the level
        // accumulators L = i .. S-1, contiguous in tensor memory.  The
        // descriptors advance by adding the offset / 16 to their address
        // field (shared-memory addresses stay below 2^18).
        for (int i = 0; i < S; ++i) {
          const uint32_t acc = tmem + (uint32_t)((c * S + i) * kTcN);
          const uint32_t idesc = umma_idesc_bf16(kTcM, kTcN * (S - i));
#pragma unroll
          for (int kk = 0; kk < kSlab / 16; ++kk)
            umma(acc, a0 + (uint64_t)((i * a_plane_bytes() + kk * 32) >> 4), b0 + (uint64_t)(kk * 2), idesc,
                 (slab > 0 || i > 0 || kk > 0) ? 1u : 0u);
        }
        umma_commit(&empty_bar[slot]);  // the stage is free once these MMAs have read it
      }
      umma_commit(&acc_bar);  // all accumulators final (also after an abort)
    }
  } else {
    // ---- epilogue: warps 0-7, thread = output row of its lane quadrant ----
    // Every level accumulator is an exact FP32 integer; the levels, the
    // per-component scales and the 3M combination are summed in
    // double-float arithmetic on the FP32 pipe (error-free TwoSum steps),
    // and only the final value is converted to FP64 and scaled (on this GPU
    // the FP64 pipe is 1/64 of the FP32 one).
    // warp w reads tensor-memory lanes 32 (w % 4) .. +31 (its quadrant) and
    // columns 16 (w / 4) .. +15: two warps per quadrant share the rows
    const int quad = warp & 3, half = warp >> 2;
    const int m = m0 + 32 * quad + lane;
    cplx* out = a.out + (size_t)z * a.zstride;
    // the tile's column exponents of B, staged while the MMAs run (named
    // barrier 1: the eight epilogue warps only)
    {
      const int t = threadIdx.x;
      if (t < 3 * kTcN) {
        const int c = t / kTcN, n = n0 + t % kTcN;
        eb_sh[c][t % kTcN] = (n < a.N) ? a.eB[(size_t)c * a.nchunks * a.N + (size_t)z * a.N + n] : 0;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
    }
    // the values an accumulating product adds to, 8 columns at a time,
    // loaded ahead (independent loads in flight together): the first
    // quarter while the MMAs run, each next one before its accumulators are
    // read
    cplx pre[8];
    auto prefetch = [&](int h) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int n = n0 + 8 * h + q;
        pre[q] = (a.accumulate && m < a.M && n < a.N) ? out[m + (size_t)a.ldo * n] : mk(0, 0);
      }
    };
    prefetch(2 * half);
    const bool ok = mbar_wait(&acc_bar, 0, vabort, a.err);
    tc_fence_after();
    if (ok && !*vabort) {
      const size_t eAs = (size_t)a.nchunks * a.M;
      int ea[3] = {0, 0, 0};
      if (m < a.M)
        for (int c = 0; c < 3; ++c) ea[c] = a.eA[c * eAs + (size_t)z * a.M + m];
      const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16);
#pragma unroll 1
      for (int h = 2 * half; h < 2 * half + 2; ++h) {
        if (h > 2 * half) prefetch(h);
        float th[3][8], tl[3][8];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          // all five level accumulators of product c (levels >= S are not
          // written by the MMAs and are skipped)
          float v[kMaxDigits][8];
          tmem_ld_levels8(lane_base + (uint32_t)(c * S * kTcN + 8 * h), v);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            th[c][q] = v[0][q] * pow2f(-14);  // exact: an integer below 2^24 times a power of two
            tl[c][q] = 0.f;
          }
#pragma unroll
          for (int L = 1; L < kMaxDigits; ++L) {
            if (L >= S) break;
            const float w = pow2f(-14 - 8 * L);
#pragma unroll
            for (int q = 0; q < 8; ++q) df_add_part(th[c][q], tl[c][q], v[L][q] * w, 0.f);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int n = n0 + 8 * h + q;
          if (m >= a.M || n >= a.N) continue;
          int ex[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) ex[c] = ea[c] + eb_sh[c][8 * h + q];
          const int E0 = max(ex[0], max(ex[1], ex[2]));
          // component values relative to 2^E0 (factors <= 1: exact scaling,
          // or below the double-float precision of the largest one)
          const float w0 = pow2f(ex[0] - E0), w1 = pow2f(ex[1] - E0), w2 = pow2f(ex[2] - E0);
          float h0 = th[0][q] * w0, l0 = tl[0][q] * w0;
          float h1 = th[1][q] * w1, l1 = tl[1][q] * w1;
          float h2 = th[2][q] * w2, l2 = tl[2][q] * w2;
          // re = T1 - T2, im = T3 - T1 - T2
          float rh = h0, rl = l0;
          df_add_part(rh, rl, -h1, -l1);
          float ih = h2, il = l2;
          df_add_part(ih, il, -h0, -l0);
          df_add_part(ih, il, -h1, -l1);
          // hi 2^E0 + lo 2^E0 as doubles built from the FP32 bit patterns
          // (exponent rebias plus E0 by integer arithmetic): one FP64
          // addition per part
          const int Es = E0 + a.alpha_exp;
          cplx r = mk(f2d_scaled(rh, Es, a.alpha_neg) + f2d_scaled(rl, Es, a.alpha_neg),
                      f2d_scaled(ih, Es, a.alpha_neg) + f2d_scaled(il, Es, a.alpha_neg));
          if (a.accumulate) r = cadd(pre[q], r);
          out[m + (size_t)a.ldo * n] = r;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---- digit splitting ----------------------------------------------------------
// The operand view of TcOperandView (kernels.h), passed by value.
struct SplitView {
  const cplx* X;
  long long rs, ks;
  int R, K, conj;
  int tri_mode, tri;
};

// What the view holds at an in-range (r, k): 0 the stored value, 1 zero
// (outside the triangle), 2 one (the unit diagonal of a reflector block).
DV int view_kind(const SplitView& v, int r, int k) {
  if (v.tri_mode == 1) return r > k + v.tri ? 1 : 0;
  // reflector s = r (rows of the view are reflector indices), entry i = k:
  // zero above the unit diagonal k < r + tri, one on it
  if (v.tri_mode == 2) return k < r + v.tri ? 1 : (k == r + v.tri ? 2 : 0);
  // same reflector block, view with rows = entry index i, columns = s
  if (v.tri_mode == 3) return r < k + v.tri ? 1 : (r == k + v.tri ? 2 : 0);
  return 0;
}

// Splitting, one CTA per (16 rows, K-chunk): the chunk (16 x at most 192
// values, 48 KB) is staged once into shared memory by cp.async along
// whichever index is contiguous in memory (entries outside the view's
// triangle are written as their constants instead of read); pass 1 finds
// each row's per-component exponent e (max |x| 2^-e < 1) over the chunk,
// pass 2 cuts the digits, written as consecutive BF16 digits per row and
// plane.  Four CTAs per SM keep about 190 KB of loads in flight.  No FP64
// arithmetic beyond one addition (re + im): the magnitudes are compared as
// integers and the digits cut from the IEEE bit pattern (on this GPU the
// FP64 pipe retires two multiply-adds per clock per SM).
constexpr int kSplitRows = 16;
constexpr int kSplitThreads = 256;
constexpr int kSplitLd = 3 * kSlab + 1;  // one K-chunk and a zero pad per shared-memory row
size_t split_smem_bytes() { return (size_t)kSplitRows * kSplitLd * sizeof(cplx); }

DV void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
DV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// |x| as an ordered integer key (the IEEE bits without the sign).
DV long long mag_key(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll; }
// e with |x| 2^-e < 1 for the value whose key is given (ilogb + 1; 0 for 0).
DV int key_exponent(long long key) {
  if (key == 0) return 0;
  const int ex = (int)(key >> 52);
  return ex == 0 ? -1021 : ex - 1022;  // subnormal: below 2^-1022
}
// round(v 2^(nbits - e)) as an integer, |v| < 2^e: from v = M 2^E (M the
// 53-bit significand) by a rounding right shift.
DV long long fixed_point(double v, int e, int nbits) {
  const long long b = __double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  long long M = b & 0xFFFFFFFFFFFFFll;
  int E;
  if (ex == 0) {
    E = -1074;
  } else {
    M |= 1ll << 52;
    E = ex - 1075;
  }
  const int sh = E - e + nbits;
  long long X;
  if (M == 0 || sh < -62) X = 0;
  else if (sh >= 0) X = M << sh;  // not reached for |v| < 2^e, nbits <= 46
  else X = (M + (1ll << (-sh - 1))) >> (-sh);
  return b < 0 ? -X : X;
}

// BF16 bits of a small integer (|d| <= 128: exact in BF16, so the upper
// half of its FP32 bits).
DV unsigned int bf16_bits(int d) { return __float_as_uint((float)d) >> 16; }

// The S balanced base-256 digits of two fixed-point values, digit j of both
// as one 32-bit word (first value in the low half) at dst[j * pstride].
// |X| <= 2^39 (S = 5): after the lowest digit the rest can reach 2^31 (a
// value within 2^-32 of its power-of-two scale), after the second it is
// below 2^24, so the first two steps run in 64 bits and the rest in 32.
DV void digit_pair(long long X0, long long X1, int S, unsigned int* dst, size_t pstride) {
  if (S == 1) {  // one digit: the value itself (|X| <= 128)
    dst[0] = bf16_bits((int)X0) | (bf16_bits((int)X1) << 16);
    return;
  }
  int d0 = (int)((X0 + 128) & 255) - 128, d1 = (int)((X1 + 128) & 255) - 128;
  X0 = (X0 - d0) >> 8;
  X1 = (X1 - d1) >> 8;
  dst[(size_t)(S - 1) * pstride] = bf16_bits(d0) | (bf16_bits(d1) << 16);
  if (S == 2) {
    dst[0] = bf16_bits((int)X0) | (bf16_bits((int)X1) << 16);
    return;
  }
  d0 = (int)((X0 + 128) & 255) - 128;
  d1 = (int)((X1 + 128) & 255) - 128;
  int y0 = (int)((X0 - d0) >> 8), y1 = (int)((X1 - d1) >> 8);
  dst[(size_t)(S - 2) * pstride] = bf16_bits(d0) | (bf16_bits(d1) << 16);
  for (int j = S - 3; j >= 1; --j) {
    d0 = ((y0 + 128) & 255) - 128;
    d1 = ((y1 + 128) & 255) - 128;
    y0 = (y0 - d0) >> 8;
    y1 = (y1 - d1) >> 8;
    dst[(size_t)j * pstride] = bf16_bits(d0) | (bf16_bits(d1) << 16);
  }
  dst[0] = bf16_bits(y0) | (bf16_bits(y1) << 16);
}

__global__ void __launch_bounds__(kSplitThreads)
    split_kernel(SplitView v, int Kc, int nchunks, int S, int* e, __nv_bfloat16* planes, long long ldk) {
  extern __shared__ cplx tile[];  // [kSplitRows][kSplitLd]
  __shared__ int esh[3][kSplitRows];
  const int r0 = blockIdx.x * kSplitRows, z = blockIdx.y;
  const int kb = z * Kc, klen = min(v.K - kb, Kc);
  const int tid = threadIdx.x;
  const int nval = kSplitRows * klen;
  const bool rows_contiguous = v.rs == 1 && v.ks != 1;
  for (int idx = tid; idx < nval; idx += kSplitThreads) {
    int r, k;
    if (rows_contiguous) {
      r = idx % kSplitRows;
      k = idx / kSplitRows;
    } else {
      k = idx % klen;
      r = idx / klen;
    }
    cplx* dst = tile + r * kSplitLd + k;
    const int kind = (r0 + r < v.R) ? view_kind(v, r0 + r, kb + k) : 1;
    if (kind == 0) cp_async16(dst, v.X + (long long)(r0 + r) * v.rs + (long long)(kb + k) * v.ks);
    else *dst = mk(kind == 2 ? 1.0 : 0.0, 0.0);
  }
  if ((klen & 1) && tid < kSplitRows) tile[tid * kSplitLd + klen] = mk(0, 0);  // second value of the last pair
  cp_async_wait_all();
  __syncthreads();
  const double sgn = v.conj ? -1.0 : 1.0;
  // pass 1: largest magnitude per row and component, a half-warp per row
  {
    const int r = tid >> 4, j = tid & 15;
    long long k0m = 0, k1m = 0, k2m = 0;
    for (int k = j; k < klen; k += 16) {
      const cplx x = tile[r * kSplitLd + k];
      const double im = sgn * x.y;
      k0m = max(k0m, mag_key(x.x));
      k1m = max(k1m, mag_key(im));
      k2m = max(k2m, mag_key(x.x + im));
    }
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
      k0m = max(k0m, __shfl_xor_sync(0xffffffffu, k0m, o));
      k1m = max(k1m, __shfl_xor_sync(0xffffffffu, k1m, o));
      k2m = max(k2m, __shfl_xor_sync(0xffffffffu, k2m, o));
    }
    if (j < 3) {
      const int ex = key_exponent(j == 0 ? k0m : (j == 1 ? k1m : k2m));
      esh[j][r] = ex;
      if (r0 + r < v.R) e[((size_t)j * nchunks + z) * v.R + r0 + r] = ex;
    }
  }
  __syncthreads();
  // pass 2: balanced base-256 digits of round(x 2^(8S-1)), |x| = |v| 2^-e < 1:
  // x ~ sum_j q_j 2^(-7-8j) with |q_j| <= 128.  Each thread cuts two
  // consecutive K-values of a row and stores each digit pair as one 32-bit
  // word (K-chunks start at even K, ldk is even).
  const size_t plane = (size_t)v.R * ldk;
  const int nbits = 8 * S - 1;
  const int nph = (klen + 1) >> 1;
  for (int pi = tid; pi < kSplitRows * nph; pi += kSplitThreads) {
    const int r = pi / nph, kk = 2 * (pi - r * nph);
    if (r0 + r >= v.R) break;
    const cplx x0 = tile[r * kSplitLd + kk], x1 = tile[r * kSplitLd + kk + 1];
    const double i0 = sgn * x0.y, i1 = sgn * x1.y;
    const double c0[3] = {x0.x, i0, x0.x + i0};
    const double c1[3] = {x1.x, i1, x1.x + i1};
    unsigned int* dst = reinterpret_cast<unsigned int*>(planes + (size_t)(r0 + r) * ldk + kb + kk);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int ex = esh[q][r];
      digit_pair(fixed_point(c0[q], ex, nbits), fixed_point(c1[q], ex, nbits), S, dst + (size_t)(q * S) * (plane / 2),
                 plane / 2);
    }
  }
}

// out[m + ldo n] = alpha * sum_z part[z * zstride + m + M n] (+ out)
__global__ void reduce_parts_kernel(const cplx* part, int M, int N, int nz, long long zstride, double alpha, int accumulate,
                                    cplx* out, long long ldo) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int m = (int)(idx % M), n = (int)(idx / M);
  cplx s = mk(0, 0);
  for (int z = 0; z < nz; ++z) s = cadd(s, part[(size_t)z * zstride + idx]);
  cplx* p = out + m + (size_t)ldo * n;
  cplx r = mk(alpha * s.x, alpha * s.y);
  if (accumulate) r = cadd(*p, r);
  *p = r;
}

}  // namespace

// ---- host entry points ------------------------------------------------------------

size_t tc_operand_bytes(int R, int K, int S, int Kc) {
  const long long ldk = ((long long)K + kSlab - 1) / kSlab * kSlab;
  const int nchunks = (K + Kc - 1) / Kc;
  const size_t planes = (size_t)3 * S * R * ldk * sizeof(__nv_bfloat16);
  const size_t exps = (size_t)3 * nchunks * R * sizeof(int);
  return ((planes + 255) & ~(size_t)255) + exps + 256;
}

int tc_chunk() { return 3 * kSlab; }
int tc_max_digits() { return kMaxDigits; }

cudaError_t tc_split(const TcOperandView& ov, int S, TcOperand* out, void* buf, cudaStream_t s) {
  if (S < 1 || S > kMaxDigits || ov.R <= 0 || ov.K <= 0) return cudaErrorInvalidValue;
  const int Kc = tc_chunk();
  const long long ldk = ((long long)ov.K + kSlab - 1) / kSlab * kSlab;
  const int nchunks = (ov.K + Kc - 1) / Kc;
  const size_t planes = (size_t)3 * S * ov.R * ldk * sizeof(__nv_bfloat16);
  out->planes = buf;
  out->e = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(buf) + ((planes + 255) & ~(size_t)255));
  out->R = ov.R;
  out->K = ov.K;
  out->S = S;
  out->ldk = ldk;
  out->nchunks = nchunks;
  SplitView v{ov.X, ov.rs, ov.ks, ov.R, ov.K, ov.conj, ov.tri_mode, ov.tri};
  const dim3 grid((ov.R + kSplitRows - 1) / kSplitRows, nchunks);
  cudaError_t e = allow_smem((const void*)split_kernel, split_smem_bytes());
  if (e != cudaSuccess) return e;
  split_kernel<<<grid, kSplitThreads, split_smem_bytes(), s>>>(v, Kc, nchunks, S, out->e, reinterpret_cast<__nv_bfloat16*>(buf), ldk);
  return cudaGetLastError();
}

cudaError_t tc_zgemm(const TcOperand& A, const TcOperand& B, cplx* out, long long ldo, double alpha, int accumulate,
                     cplx* part, size_t part_elems, int* err, cudaStream_t s) {
  if (A.K != B.K || A.S != B.S || A.nchunks != B.nchunks) return cudaErrorInvalidValue;
  const int M = A.R, N = B.R, K = A.K, S = A.S, nz = A.nchunks;
  CUtensorMap ma, mb;
  cudaError_t e = plane_map(&ma, static_cast<const __nv_bfloat16*>(A.planes), K, A.ldk, M, 3 * S, kTcM);
  if (e == cudaSuccess) e = plane_map(&mb, static_cast<const __nv_bfloat16*>(B.planes), K, B.ldk, N, 3 * S, kTcN);
  if (e != cudaSuccess) return e;
  const size_t smem = tc_smem_bytes(S);
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, []() {
    attr = cudaFuncSetAttribute(tc_zgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem_bytes(kMaxDigits));
  });
  if (attr != cudaSuccess) return attr;
  TcArgs a{};
  a.M = M;
  a.N = N;
  a.K = K;
  a.S = S;
  a.Kc = tc_chunk();
  a.nchunks = nz;
  a.eA = A.e;
  a.eB = B.e;
  a.err = err;
  const dim3 grid((N + kTcN - 1) / kTcN, (M + kTcM - 1) / kTcM, nz);
  // alpha must be a signed power of two (the callers use +-1)
  int aexp = 0;
  const double am = std::frexp(std::fabs(alpha), &aexp);
  if (am != 0.5) return cudaErrorInvalidValue;
  if (nz == 1) {
    a.out = out;
    a.ldo = ldo;
    a.zstride = 0;
    a.alpha_exp = aexp - 1;
    a.alpha_neg = alpha < 0.0;
    a.accumulate = accumulate;
    tc_zgemm_kernel<<<grid, kTcThreads, smem, s>>>(ma, mb, a);
    return cudaGetLastError();
  }
  if (!part || part_elems < (size_t)nz * M * N) return cudaErrorInvalidValue;
  a.out = part;
  a.ldo = M;
  a.zstride = (long long)M * N;
  a.alpha_exp = 0;
  a.alpha_neg = 0;
  a.accumulate = 0;
  tc_zgemm_kernel<<<grid, kTcThreads, smem, s>>>(ma, mb, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)M * N;
  reduce_parts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, M, N, nz, (long long)M * N, alpha, accumulate,
                                                                   out, ldo);
  return cudaGetLastError();
}

size_t tc_part_elems(int M, int N, int K) {
  const int nz = (K + tc_chunk() - 1) / tc_chunk();
  return nz > 1 ? (size_t)nz * M * N : 0;
}

}  // namespace hk
