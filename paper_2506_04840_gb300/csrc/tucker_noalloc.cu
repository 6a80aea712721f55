// tucker_sketch_noalloc: the sketch Y = A_(k) Omega_k without any device
// allocation.  Its per-block partial products live in a fixed array in the
// library's own device memory instead of memory obtained from cudaMalloc.
//
// Who needs it: programs that reserve all device memory up front and forbid
// later allocation (inference servers with a fixed memory budget, plugins
// whose host application owns the allocator, latency-critical loops that
// cannot risk an allocation failing or stalling mid-request).  Such callers
// cannot let the library call cudaMalloc or cudaMallocAsync on their behalf.
#include <mutex>
#include <vector>

#include "tk_common.cuh"
#include "tk_internal.h"
#include "tk_plan.h"

namespace tk {

// Scratch for the partial products: TK_NOALLOC_SCRATCH_BYTES (8 MiB) in every
// GPU that loads the library, held until the process exits.  Shared by all
// calls; each call overwrites the part it uses before reading it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TK_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device.  In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, called once per device with that device current.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

}  // namespace tk

using namespace tk;

extern "C" tk_status tucker_sketch_noalloc(const tk_tensor* A, int k, int l, uint64_t seed,
                                           uint32_t tag, double* Y, void* stream) {
  // the same argument checks and mode-k view as tucker_sketch
  if (!valid_tensor(A, true) || k < 0 || k >= A->d || l < 1 || l > TK_MAX_L || !Y ||
      tag >= (1u << 24))
    return TK_EINVAL;
  std::vector<int64_t> dims(A->n, A->n + A->d);
  const View v = view_of(dims, k);
  const XType xt = xtype(A->dtype);
  const int lc = xb_lc(l);
  const size_t per_split = (size_t)v.n * lc * asize(xt);
  if (per_split > (size_t)TK_NOALLOC_SCRATCH_BYTES) return TK_EWORKSPACE;
  int splits = xb_splits(xt, v, l);
  const int fit = (int)((size_t)TK_NOALLOC_SCRATCH_BYTES / per_split);
  if (splits > fit) splits = fit;
  void* part = nullptr;
  cudaError_t e = scratch_address(&part);
  if (e != cudaSuccess) return from_cuda(e);
  cudaStream_t st = (cudaStream_t)stream;
  // k_xb writes every entry of the partial blocks it uses, so the scratch
  // needs no clearing between calls.
  e = launch_xb(xt, A->data, v, nullptr, l, seed, tag, k, part, splits, st);
  if (e == cudaSuccess) e = launch_reduce(xt, part, splits, v.n, l, lc, nullptr, nullptr, Y, st);
  return from_cuda(e);
}
