// Bench-only measurement library (libsxeprobe.so, built by bench.py; not part of libsimplexenc):
// the scattered access patterns that bound the encoding's table kernels, timed alone so that a
// kernel's rate can be set against what the memory system gives for the same pattern on the same
// footprint.  The paper has no counterpart.
//
//   int sxe_probe_random_access(int kind, float* buf, int64_t n_slots, int slot_floats,
//                               int64_t n_ops, uint64_t seed, float* sink, void* stream);
//
// n_ops accesses to random slots of the device buffer buf [n_slots][slot_floats] binary32
// (n_slots a power of two, slot_floats even, 2..64); slot = mix64(seed ^ i) mod n_slots with a
// counter-based 64-bit mixer (the splitmix64 finaliser):
//   kind 0: a float2 atomic add of (1, 1) into the slot's last two floats (the shape of the table
//           backward's reductions into optimiser records);
//   kind 1: a 4-byte load of the slot's first float (the shape of the forward gathers); sink[0]
//           is written only if the loaded sum is -1, which a zeroed or bounded buffer never gives;
//   kind 2: a read and write back of the whole 32-byte slot (slot_floats = 8, buf 16-byte
//           aligned; the shape of the table optimiser), four slots in flight per thread.
// buf is 8-byte aligned (16 for kind 2) and n_slots <= 2^34.  Returns 0, -1 for an argument
// outside these ranges (nothing launched) or -3 if the launch failed.  Asynchronous on `stream` (a cudaStream_t).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

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
  if (kind == 1 && acc == -1.f) sink[0] = acc;
}

}  // namespace

extern "C" int sxe_probe_random_access(int kind, float* buf, int64_t n_slots, int slot_floats, int64_t n_ops,
                                       uint64_t seed, float* sink, void* stream) {
  if (kind < 0 || kind > 2 || !buf || !sink || n_slots < 1 || (n_slots & (n_slots - 1)) ||
      n_slots > ((int64_t)1 << 34) || slot_floats < 2 || slot_floats > 64 || slot_floats % 2 || n_ops < 0 ||
      (uintptr_t)buf % (kind == 2 ? 16 : 8) || (kind == 2 && slot_floats != 8))
    return -1;
  if (n_ops == 0) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  probe_kernel<<<8 * (sms > 0 ? sms : 148), 256, 0, (cudaStream_t)stream>>>(kind, buf, (uint64_t)n_slots - 1,
                                                                             slot_floats, n_ops, seed, sink);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
