// sxe_mlp_train_l2_static: the fused network forward + L2 loss + backward of
// sxe_mlp_train_l2, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's allocator (which owns all device memory and forbids foreign
// allocations), code driven from a real-time or embedded loop where an allocation
// may block or fail, and code that must not touch the allocator while a stream is
// being captured into a CUDA graph.  They can still pass their inputs and outputs,
// but not the per-CTA scratch the backward kernel needs for its weight-gradient
// partials.  This entry point takes that scratch from a fixed array in the
// library's own device memory instead.
//
// The array is a file-scope __device__ object of SXE_MLP_STATIC_SCRATCH_FLOATS
// floats (8 MiB); every GPU that loads the library holds it until the process exits.
// Host code must not use the array's name as a device address: on the first call on
// each device (with that device current) the entry point asks the runtime for the
// array's device address with cudaGetSymbolAddress, checks the result and caches it.
// That first call should therefore happen before any stream capture begins.
//
// Every call shares the one array and leaves its contents behind.  Nothing in it has
// to start at zero: each CTA overwrites all of its partials before the reduction
// reads them.  Two calls whose kernels overlap on the GPU (different streams without
// ordering) race on the array and give wrong gradients; serialise them.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "sxe_internal.cuh"

#define SXE_MLP_STATIC_SCRATCH_FLOATS (1 << 21)

namespace sxe {
namespace {

__device__ __align__(256) float g_mlp_scratch[SXE_MLP_STATIC_SCRATCH_FLOATS];

constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

sxe_status scratch_for_current_device(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(SXE_ECUDA, "mlp_train_l2_static: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(SXE_EUNSUPPORTED, "mlp_train_l2_static: device %d", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mlp_scratch);
    if (e != cudaSuccess || !p)
      return set_error(SXE_ECUDA, "mlp_train_l2_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SXE_OK;
}

}  // namespace
}  // namespace sxe

using namespace sxe;

extern "C" sxe_status sxe_mlp_train_l2_static(const sxe_mlp_desc* d, const void* W, const void* in,
                                              const float* target, float loss_scale, int64_t P, float* din,
                                              float* dW, float* sq_sum, void* stream) {
  sxe_status st = check_mlp("mlp_train_l2_static", d);
  if (st != SXE_OK) return st;
  if (P < 0) return set_error(SXE_EINVAL, "mlp_train_l2_static: n_points < 0");
  if (!(loss_scale > 0.f) || !isfinite(loss_scale)) return set_error(SXE_EINVAL, "mlp_train_l2_static: loss_scale must be > 0");
  if (P > 0 && (!target || !sq_sum || !W || !in || !dW))
    return set_error(SXE_EINVAL, "mlp_train_l2_static: NULL weights, in, target, dweights or sq_sum");
  if ((uintptr_t)in % 16 || (uintptr_t)W % 4 || (din && (uintptr_t)din % 8))
    return set_error(SXE_EINVAL, "mlp_train_l2_static: in must be 16-byte aligned, weights 4, din 8");
  const int64_t per_cta = sxe_mlp_n_params(d) + 1;   // weight partials + one loss partial
  if (per_cta > SXE_MLP_STATIC_SCRATCH_FLOATS)
    return set_error(SXE_ENOMEM, "mlp_train_l2_static: %lld floats of scratch per CTA exceed the static %d",
                     (long long)per_cta, SXE_MLP_STATIC_SCRATCH_FLOATS);
  if (P == 0) return empty_batch_sq_sum("mlp_train_l2_static", sq_sum, stream);
  float* ws = nullptr;
  st = scratch_for_current_device(&ws);
  if (st != SXE_OK) return st;
  // the persistent grid is cut down to what the static scratch holds (results do not
  // depend on the grid beyond the summation order of the weight-gradient partials)
  const int64_t fit = SXE_MLP_STATIC_SCRATCH_FLOATS / per_cta;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(mlp_grid_blocks(d, P), fit));
  return launch_mlp_bwd(d, W, in, nullptr, target, loss_scale, P, din, dW, sq_sum, ws, grid, (cudaStream_t)stream);
}
