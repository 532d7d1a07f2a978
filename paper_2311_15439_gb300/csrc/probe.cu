// Measurement aids: the scattered access patterns that bound the encoding kernels, timed
// alone so that a kernel's rate can be compared with what the memory system gives for the
// same pattern (the paper has no counterpart).  Slot indexes come from a counter-based
// 64-bit mixer and are masked into [0, n_slots), n_slots a power of two.
#include "sxe_internal.cuh"

namespace sxe {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// kind 0: float2 reduction into the last two floats of a random slot of `slot_floats` floats
// kind 1: 4-byte load from the start of a random slot, summed per thread
// kind 2: read-modify-write of a random 32-byte slot (slot_floats = 8): four slots per thread
//         and iteration, all four loaded before any is stored (the optimiser's pattern)
__global__ void __launch_bounds__(256)
probe_kernel(int kind, float* __restrict__ buf, uint64_t mask, int slot_floats, int64_t n, uint64_t seed,
             float* __restrict__ sink) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float acc = 0.f;
  if (kind == 2) {
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i < n; i += stride * 4) {
      float4* r[4];
      float4 a[4], b[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        r[j] = reinterpret_cast<float4*>(buf + (mix64(seed ^ (uint64_t)(i + j)) & mask) * 8u);
        if (i + j < n) { a[j] = __ldcg(r[j]); b[j] = __ldcg(r[j] + 1); }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (i + j < n) {
          a[j].x += 1.f;
          b[j].w = 0.f;
          r[j][0] = a[j];
          r[j][1] = b[j];
        }
    }
    return;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t s = mix64(seed ^ (uint64_t)i) & mask;
    float* p = buf + s * (uint64_t)slot_floats;
    if (kind == 0) atomicAdd(reinterpret_cast<float2*>(p + slot_floats - 2), make_float2(1.f, 1.f));
    else acc += __ldg(p);
  }
  if (kind == 1 && acc == -1.f) sink[0] = acc;     // keeps the loads; never true for a zeroed buffer
}

}  // namespace

sxe_status launch_probe(int kind, float* buf, int64_t n_slots, int slot_floats, int64_t n_ops, uint64_t seed,
                        float* sink, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  probe_kernel<<<8 * (sms > 0 ? sms : 148), 256, 0, s>>>(kind, buf, (uint64_t)n_slots - 1, slot_floats, n_ops, seed,
                                                          sink);
  return check_launch("probe");
}

}  // namespace sxe
