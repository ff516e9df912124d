// hopf_eval_points_noalloc: point evaluation of a TT without any device
// allocation.
//
// hopf_eval_points stages its index list and its results in buffers it
// allocates with cudaMalloc and releases with cudaFree on every call.  Some
// callers cannot afford that: cudaFree waits for all work on the device, so
// a monitor that probes Phi at a few points between solver steps (on its own
// stream, while the solver keeps the GPU busy) would stall the solver; and a
// process whose device memory is fully reserved by another allocator (a deep
// learning framework's caching allocator, say) may see cudaMalloc fail.
// This entry point stages the same data in two fixed-size arrays that live
// in this library's device image instead.
#include <mutex>

#include "../../include/hopf.h"
#include "kernels.h"

namespace {

// Fixed staging capacity (bytes: 512 KiB of indices + 32 KiB of results per
// GPU that loads the library, held until the process exits).
constexpr int kMaxPoints = HOPF_NOALLOC_MAX_POINTS;
constexpr int kMaxIdx = HOPF_NOALLOC_MAX_POINTS * HOPF_NOALLOC_MAX_D;

static __device__ __align__(256) int g_noalloc_idx[kMaxIdx];
static __device__ __align__(256) double2 g_noalloc_vals[kMaxPoints];

// Device addresses of the two arrays, looked up once per device.  In host
// code the array names are host-side stand-ins, not device addresses, so
// the kernels only ever receive these looked-up pointers.
struct Addrs {
  int* idx = nullptr;
  double2* vals = nullptr;
  bool ready = false;
};
constexpr int kMaxDevices = 64;
Addrs g_addrs[kMaxDevices];
std::mutex g_addrs_mu;

// Looks up (once) the arrays' addresses on device `dev`, which must be the
// current device.
cudaError_t device_addrs(int dev, Addrs* out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addrs_mu);
  Addrs& a = g_addrs[dev];
  if (!a.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_idx);
    if (e != cudaSuccess) return e;
    a.idx = static_cast<int*>(p);
    e = cudaGetSymbolAddress(&p, g_noalloc_vals);
    if (e != cudaSuccess) return e;
    a.vals = static_cast<double2*>(p);
    a.ready = true;
  }
  *out = a;
  return cudaSuccess;
}

// Makes `dev` current for the lifetime of the guard and restores the
// caller's device afterwards (on every return path).
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    else if (err == cudaSuccess) prev = -1;  // nothing to restore
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

// Internal accessors defined in hopf.cu (the tensor layout is private there).
hopf_ctx* hopf_internal_tt_ctx(const hopf_tt* t);
cudaStream_t hopf_internal_stream(const hopf_ctx* ctx);
int hopf_internal_device(const hopf_ctx* ctx);
hopf_status hopf_internal_tt_view(const hopf_tt* t, const double2* const** d_ptrs, const int** d_ranks,
                                  int* d, int* n, int* maxr);
void hopf_internal_set_error(hopf_ctx* ctx, const char* msg);

extern "C" hopf_status hopf_eval_points_noalloc(const hopf_tt* t, int npts, const int* idx, double* vals) {
  if (!t) return HOPF_EINVAL;
  hopf_ctx* ctx = hopf_internal_tt_ctx(t);
  const double2* const* d_ptrs = nullptr;
  const int* d_ranks = nullptr;
  int d = 0, n = 0, maxr = 1;
  hopf_status st = hopf_internal_tt_view(t, &d_ptrs, &d_ranks, &d, &n, &maxr);
  if (st != HOPF_OK) return st;
  if (npts < 0 || (npts > 0 && (!idx || !vals))) {
    hopf_internal_set_error(ctx, "hopf_eval_points_noalloc: bad arguments");
    return HOPF_EINVAL;
  }
  if (npts > kMaxPoints || d > HOPF_NOALLOC_MAX_D) {
    hopf_internal_set_error(ctx, "hopf_eval_points_noalloc: more than HOPF_NOALLOC_MAX_POINTS points "
                                 "or more than HOPF_NOALLOC_MAX_D modes");
    return HOPF_EINVAL;
  }
  for (size_t e = 0; e < (size_t)npts * d; ++e)
    if (idx[e] < 0 || idx[e] >= n) {
      hopf_internal_set_error(ctx, "hopf_eval_points_noalloc: index outside [0, n)");
      return HOPF_EINVAL;
    }
  if (npts == 0) return HOPF_OK;
  // The tensor's data, its context's stream and the arrays used here all
  // belong to the context's device, whatever device the caller has current.
  const int dev = hopf_internal_device(ctx);
  DeviceGuard guard(dev);
  cudaError_t e = guard.err;
  Addrs a;
  if (e == cudaSuccess) e = device_addrs(dev, &a);
  const cudaStream_t s = hopf_internal_stream(ctx);
  // Every value read below is written first in this call: the index list is
  // copied in, and the kernel writes one result per point.
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(a.idx, idx, (size_t)npts * d * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = hk::eval_points(d_ptrs, d_ranks, d, n, maxr, npts, a.idx, a.vals, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(vals, a.vals, (size_t)npts * sizeof(double2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    hopf_internal_set_error(ctx, cudaGetErrorString(e));
    return HOPF_ECUDA;
  }
  return HOPF_OK;
}
