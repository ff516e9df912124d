// Blocked Householder QR and Q application whose dense products run on the
// tensor cores (tc.cu), for the mixed-precision rounding.
//
// The right-to-left sweep and the truncation sweep (App. A, Alg. 1/2
// mirrored, with Alg. 4's factor-then-SVD structure) spend their time in
// QR factorisations of tall flattenings, m x K with m = n p up to 49152 and
// K = 6 r = 384.  Here the columns are taken in outer panels of width
// kOuter = 128:
//   1. the panel is factored by the cooperative Householder kernel (qr.cu,
//      double-float arithmetic, FP64 scalars), leaving reflectors V (unit
//      lower trapezoidal) and tau;
//   2. the panel's Gram G = V^H V is formed on the tensor cores; with
//      D = diag(1/tau), T^{-1} = D + striu(G) is the triangular factor of the
//      compact WY form H_0 ... H_{b-1} = I - V T V^H;
//   3. the trailing columns A_t receive Q^H: W = V^H A_t (tensor cores,
//      split over the m rows in exact chunks), W2 = T^H W (forward
//      substitution on D-bar + striu(G)^H, FP64), A_t -= V W2 (tensor cores).
// Applying Q = H_0 ... H_{p-1} (ormqr_tc) walks the panels backwards with
// W2 = T W (back substitution on D + striu(G)).  G of every panel is kept
// by the caller between the two.
#include <algorithm>

#include "kernels.h"

namespace hk {

namespace {

constexpr int kOuter = 128;

// W2 = T^H W (forward) or T W (backward) for the compact WY factor given by
// G (v_s^H v_u in G[s + ldg u]; Hermitian) and tau: one warp per column l
// of W (nbk x nt, ldw), each lane holding rows s = lane + 32 q.  The
// recurrence runs in double-float arithmetic on the FP32 pipe (a chain of
// FP64 multiply-adds waits on this GPU's narrow FP64 pipe at every step);
// its ~2^-48 relative rounding is far below the tensor-core products'
// error.  The triangle of G it reads and tau are packed once per panel
// (wy_pack_kernel: negated, in double-float form, column u of the triangle
// holding -G[s, u] for s > u (forward) or s < u (backward)) and copied into
// shared memory by every CTA (the solve is a chain of nbk dependent steps;
// each step then reads shared memory, not L2).
constexpr int kWyWarps = 4;

DV int wy_off(int u, int nbk, int forward) {  // packed offset of column u
  return forward ? u * (2 * nbk - u - 1) / 2 : u * (u - 1) / 2;
}
HD size_t wy_packed_elems(int nbk) { return (size_t)nbk * (nbk - 1) / 2 + nbk; }

__global__ void wy_pack_kernel(const cplx* G, int ldg, const cplx* tau, int nbk, int forward, df2* packed) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nbk * nbk) return;
  const int s = idx % nbk, u = idx / nbk;
  if (forward ? s > u : s < u) {
    const cplx gv = G[s + (size_t)ldg * u];
    packed[wy_off(u, nbk, forward) + (forward ? s - u - 1 : s)] = df_from(mk(-gv.x, -gv.y));
  }
  // forward: w2_u = conj(tau_u) (...); backward: w2_u = tau_u (...)
  if (s == u) packed[(size_t)nbk * (nbk - 1) / 2 + u] = df_from(forward ? cconj(tau[u]) : tau[u]);
}

__global__ void __launch_bounds__(32 * kWyWarps)
    wy_solve_kernel(const df2* packed, int nbk, const cplx* W, int ldw, int nt, cplx* W2, int ldw2, int forward) {
  extern __shared__ __align__(16) unsigned char wy_raw[];
  df2* tri = reinterpret_cast<df2*>(wy_raw);  // nbk (nbk - 1) / 2 packed
  df2* tsh = tri + (size_t)nbk * (nbk - 1) / 2;
  auto off = [&](int u) -> int { return wy_off(u, nbk, forward); };
  {
    // coalesced 16-byte loads, eight in flight per thread
    const float4* src = reinterpret_cast<const float4*>(packed);
    float4* dst = reinterpret_cast<float4*>(wy_raw);
    const int n16 = (int)wy_packed_elems(nbk);
    constexpr int U = 8;
    for (int e0 = threadIdx.x; e0 < n16; e0 += U * blockDim.x) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < n16) v[u] = __ldg(src + e);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < n16) dst[e] = v[u];
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.x * kWyWarps + (threadIdx.x >> 5);
  if (l >= nt) return;
  constexpr int Q = kOuter / 32;
  // the column scaled by a power of two to a maximum below one (the FP32
  // exponent range of the double-float parts is then never left; W2 = T^H W
  // is linear in W, so the scale comes back exactly at the end)
  cplx wv[Q];
  double mx = 0.0;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int s = lane + 32 * q;
    wv[q] = (s < nbk) ? W[s + (size_t)ldw * l] : mk(0, 0);
    mx = fmax(mx, fmax(fabs(wv[q].x), fabs(wv[q].y)));
  }
  for (int o = 16; o >= 1; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int E = (mx > 0.0) ? ilogb(mx) + 1 : 0;
  df2 acc[Q], mine[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    acc[q] = df_from(mk(scalbn(wv[q].x, -E), scalbn(wv[q].y, -E)));
    mine[q] = df_zero();
  }
  for (int step = 0; step < nbk; ++step) {
    const int u = forward ? step : nbk - 1 - step;
    const int qu = u >> 5, lu = u & 31;
    df2 own = df_zero();
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (q == qu) own = acc[q];
    df2 w2 = df_zero();
    df_cmac(w2, tsh[u], own);  // valid on lane lu
    w2 = df2{__shfl_sync(0xffffffffu, w2.rh, lu), __shfl_sync(0xffffffffu, w2.ih, lu),
             __shfl_sync(0xffffffffu, w2.rl, lu), __shfl_sync(0xffffffffu, w2.il, lu)};
    if (lane == lu) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (q == qu) mine[q] = w2;
    }
    const df2* col = tri + off(u);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = lane + 32 * q;
      if (s >= nbk) continue;
      // forward: (T^-H)[s, u] = conj(G[u, s]) = G[s, u] for s > u
      if (forward && s > u) df_cmac(acc[q], col[s - u - 1], w2);
      else if (!forward && s < u) df_cmac(acc[q], col[s], w2);
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int s = lane + 32 * q;
    if (s < nbk) {
      const cplx v = df_to(mine[q]);
      W2[s + (size_t)ldw2 * l] = mk(scalbn(v.x, E), scalbn(v.y, E));
    }
  }
}

// `packed` holds wy_packed_elems(nbk) double-float values of scratch.
cudaError_t wy_solve(const cplx* G, int ldg, const cplx* tau, int nbk, const cplx* W, int ldw, int nt, cplx* W2,
                     int ldw2, int forward, df2* packed, cudaStream_t s) {
  if (nt <= 0) return cudaSuccess;
  const size_t smem = sizeof(df2) * wy_packed_elems(nbk);
  static cudaError_t attr = cudaFuncSetAttribute(wy_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(sizeof(df2) * wy_packed_elems(kOuter)));
  if (attr != cudaSuccess) return attr;
  wy_pack_kernel<<<(nbk * nbk + 255) / 256, 256, 0, s>>>(G, ldg, tau, nbk, forward, packed);
  wy_solve_kernel<<<(nt + kWyWarps - 1) / kWyWarps, 32 * kWyWarps, smem, s>>>(packed, nbk, W, ldw, nt, W2, ldw2,
                                                                             forward);
  return cudaGetLastError();
}

// G[s, u] <- conj(G[u, s]) for s > u: the Gram exactly Hermitian, so that
// the forward solve (which reads the lower triangle, contiguous across the
// lanes) and the backward solve (the upper one) use the same numbers.
__global__ void hermitize_kernel(cplx* G, int ldg, int nb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * nb) return;
  const int s = idx % nb, u = idx / nb;
  if (s > u) G[s + (size_t)ldg * u] = cconj(G[u + (size_t)ldg * s]);
}

// Carves the scratch for one panel step out of ws.
struct Carve {
  unsigned char* p;
  size_t left;
  bool ok = true;
  void* take(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes > left) {
      ok = false;
      return nullptr;
    }
    void* r = p;
    p += bytes;
    left -= bytes;
    return r;
  }
};

}  // namespace

int tc_outer_panel() { return kOuter; }

bool qr_tc_applies(int m, int p) { return m >= 4096 && p > 32; }

size_t qr_tc_scratch_bytes(int m, int k, int S) {
  const int Kc = tc_chunk();
  const int nt = std::max(k, 1);
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
  add(tc_operand_bytes(kOuter, m, S, Kc));  // V^H
  add(tc_operand_bytes(kOuter, m, S, Kc));  // V (as the Gram's second operand)
  add(tc_operand_bytes(nt, m, S, Kc));      // trailing columns / C
  add(tc_operand_bytes(m, kOuter, S, Kc));  // V
  add(tc_operand_bytes(nt, kOuter, S, Kc)); // W2
  add(std::max(tc_part_elems(kOuter, nt, m), tc_part_elems(kOuter, kOuter, m)) * sizeof(cplx));
  add((size_t)kOuter * nt * sizeof(cplx) * 2);  // W, W2
  add(wy_packed_elems(kOuter) * sizeof(df2));   // packed WY triangle
  return b + 1024;
}

size_t qr_tc_gram_elems(int k) { return (size_t)((k + kOuter - 1) / kOuter) * kOuter * kOuter; }

// Complex GEMM FLOPs (8 per complex multiply-add) of an M x N x K product.
static double zflops(double M, double N, double K) { return 8.0 * M * N * K; }

cudaError_t geqrf_tc(cplx* A, int lda, int m, int k, cplx* tau, cplx* T, cplx* Gout, void* scratch,
                     size_t scratch_bytes, const CoopWs& cws, int S, cudaStream_t s, const PhaseTimer& pt) {
  const int p = std::min(m, k);
  const int Kc = tc_chunk();
  cudaError_t e = cudaSuccess;
  for (int j0 = 0; j0 < p && e == cudaSuccess; j0 += kOuter) {
    const int nbk = std::min(kOuter, p - j0);
    const int mv = m - j0;
    cplx* Ap = A + j0 + (size_t)lda * j0;
    int nb = 32;
    int slot = pt.b();
    e = geqrf(Ap, lda, mv, nbk, tau + j0, T + (size_t)(j0 / 32) * 32 * 32, &nb, cws, s, 1);
    pt.e(slot, pt.cls_panel, 8.0 * mv * (double)nbk * nbk - 8.0 * (double)nbk * nbk * nbk / 3.0, 1);
    if (e != cudaSuccess) break;
    Carve c{static_cast<unsigned char*>(scratch), scratch_bytes};
    void* bVH = c.take(tc_operand_bytes(nbk, mv, S, Kc));
    void* bVB = c.take(tc_operand_bytes(nbk, mv, S, Kc));
    const int nt = k - j0 - nbk;
    void* bX = c.take(tc_operand_bytes(std::max(nt, 1), mv, S, Kc));
    void* bV = c.take(tc_operand_bytes(mv, nbk, S, Kc));
    void* bW2 = c.take(tc_operand_bytes(std::max(nt, 1), nbk, S, Kc));
    const size_t npart = std::max(tc_part_elems(nbk, std::max(nt, 1), mv), tc_part_elems(nbk, nbk, mv));
    cplx* part = static_cast<cplx*>(c.take(npart * sizeof(cplx)));
    cplx* W = static_cast<cplx*>(c.take((size_t)nbk * std::max(nt, 1) * sizeof(cplx)));
    cplx* W2 = static_cast<cplx*>(c.take((size_t)nbk * std::max(nt, 1) * sizeof(cplx)));
    df2* packed = static_cast<df2*>(c.take(wy_packed_elems(nbk) * sizeof(df2)));
    if (!c.ok) return cudaErrorInvalidValue;
    // G = V^H V (reflector s along rows, entries i along K)
    TcOperand oVH, oVB, oX, oV, oW2;
    slot = pt.b();
    e = tc_split(TcOperandView{Ap, lda, 1, nbk, mv, 1, 2, 0}, S, &oVH, bVH, s);
    if (e == cudaSuccess) e = tc_split(TcOperandView{Ap, lda, 1, nbk, mv, 0, 2, 0}, S, &oVB, bVB, s);
    cplx* G = Gout + (size_t)(j0 / kOuter) * kOuter * kOuter;
    if (e == cudaSuccess) e = tc_zgemm(oVH, oVB, G, kOuter, 1.0, 0, part, npart, &cws.bar->err, s);
    if (e == cudaSuccess) {
      hermitize_kernel<<<(nbk * nbk + 255) / 256, 256, 0, s>>>(G, kOuter, nbk);
      e = cudaGetLastError();
    }
    // launches: two splits, the product, its chunk reduction (K > one chunk), hermitize
    pt.e(slot, pt.cls_tc, zflops(nbk, nbk, mv), 4 + (mv > Kc));
    if (e != cudaSuccess || nt <= 0) continue;
    // trailing columns: W = V^H A_t, W2 = T^H W, A_t -= V W2
    cplx* At = A + j0 + (size_t)lda * (j0 + nbk);
    slot = pt.b();
    e = tc_split(TcOperandView{At, lda, 1, nt, mv, 0, 0, 0}, S, &oX, bX, s);
    if (e == cudaSuccess) e = tc_zgemm(oVH, oX, W, nbk, 1.0, 0, part, npart, &cws.bar->err, s);
    pt.e(slot, pt.cls_tc, zflops(nbk, nt, mv), 2 + (mv > Kc));
    slot = pt.b();
    if (e == cudaSuccess) e = wy_solve(G, kOuter, tau + j0, nbk, W, nbk, nt, W2, nbk, 1, packed, s);
    pt.e(slot, pt.cls_small, 0.0, 2);  // pack + solve
    slot = pt.b();
    if (e == cudaSuccess) e = tc_split(TcOperandView{W2, nbk, 1, nt, nbk, 0, 0, 0}, S, &oW2, bW2, s);
    if (e == cudaSuccess) e = tc_split(TcOperandView{Ap, 1, lda, mv, nbk, 0, 3, 0}, S, &oV, bV, s);
    if (e == cudaSuccess) e = tc_zgemm(oV, oW2, At, lda, -1.0, 1, nullptr, 0, &cws.bar->err, s);
    pt.e(slot, pt.cls_tc, zflops(mv, nt, nbk), 3);  // two splits, one chunk
  }
  return e;
}

cudaError_t ormqr_tc(const cplx* A, int lda, int m, int p, const cplx* tau, const cplx* Gin, cplx* C, int ldc, int q,
                     void* scratch, size_t scratch_bytes, int* err, int S, cudaStream_t s, const PhaseTimer& pt) {
  if (m <= 0 || p <= 0 || q <= 0) return cudaSuccess;
  const int Kc = tc_chunk();
  const int npanel = (p + kOuter - 1) / kOuter;
  cudaError_t e = cudaSuccess;
  for (int j = npanel - 1; j >= 0 && e == cudaSuccess; --j) {
    const int j0 = j * kOuter, nbk = std::min(kOuter, p - j0), mv = m - j0;
    const cplx* Ap = A + j0 + (size_t)lda * j0;
    cplx* Cj = C + j0;
    Carve c{static_cast<unsigned char*>(scratch), scratch_bytes};
    void* bVH = c.take(tc_operand_bytes(nbk, mv, S, Kc));
    void* bX = c.take(tc_operand_bytes(q, mv, S, Kc));
    void* bV = c.take(tc_operand_bytes(mv, nbk, S, Kc));
    void* bW2 = c.take(tc_operand_bytes(q, nbk, S, Kc));
    const size_t npart = tc_part_elems(nbk, q, mv);
    cplx* part = static_cast<cplx*>(c.take(std::max<size_t>(npart, 1) * sizeof(cplx)));
    cplx* W = static_cast<cplx*>(c.take((size_t)nbk * q * sizeof(cplx)));
    cplx* W2 = static_cast<cplx*>(c.take((size_t)nbk * q * sizeof(cplx)));
    df2* packed = static_cast<df2*>(c.take(wy_packed_elems(nbk) * sizeof(df2)));
    if (!c.ok) return cudaErrorInvalidValue;
    TcOperand oVH, oX, oV, oW2;
    int slot = pt.b();
    e = tc_split(TcOperandView{Ap, lda, 1, nbk, mv, 1, 2, 0}, S, &oVH, bVH, s);
    if (e == cudaSuccess) e = tc_split(TcOperandView{Cj, ldc, 1, q, mv, 0, 0, 0}, S, &oX, bX, s);
    if (e == cudaSuccess) e = tc_zgemm(oVH, oX, W, nbk, 1.0, 0, part, npart, err, s);
    pt.e(slot, pt.cls_tc, zflops(nbk, q, mv), 3 + (mv > Kc));
    slot = pt.b();
    if (e == cudaSuccess)
      e = wy_solve(Gin + (size_t)j * kOuter * kOuter, kOuter, tau + j0, nbk, W, nbk, q, W2, nbk, 0, packed, s);
    pt.e(slot, pt.cls_small, 0.0, 2);
    slot = pt.b();
    if (e == cudaSuccess) e = tc_split(TcOperandView{W2, nbk, 1, q, nbk, 0, 0, 0}, S, &oW2, bW2, s);
    if (e == cudaSuccess) e = tc_split(TcOperandView{Ap, 1, lda, mv, nbk, 0, 3, 0}, S, &oV, bV, s);
    if (e == cudaSuccess) e = tc_zgemm(oV, oW2, Cj, ldc, -1.0, 1, nullptr, 0, err, s);
    pt.e(slot, pt.cls_tc, zflops(mv, q, nbk), 3);
  }
  return e;
}

}  // namespace hk
