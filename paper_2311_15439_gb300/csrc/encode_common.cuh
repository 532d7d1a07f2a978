// Work-item helpers shared by the encoding kernels (forward, backward, input gradient, table
// step): one thread per (point, level) pair, the level fastest (or, for the forward, level-major).
#pragma once

#include "sxe_internal.cuh"

namespace sxe {
namespace encode_detail {

constexpr int kThreads = 256;

template <bool SIMPLEX, int D> struct Verts { static constexpr int V = SIMPLEX ? D + 1 : (1 << D); };

template <bool SIMPLEX, int D>
__device__ __forceinline__ void lattice(const float (&x)[D], float s, float skewF, uint32_t mask, uint32_t width,
                                        uint32_t (&slot)[Verts<SIMPLEX, D>::V], float (&w)[Verts<SIMPLEX, D>::V]) {
  if constexpr (SIMPLEX) simplex_lattice<D>(x, s, skewF, mask, width, slot, w);
  else grid_lattice<D>(x, s, mask, width, slot, w);
}

// Decode work item i = blockIdx.x * kThreads + threadIdx.x into (point, level) = (i / L, i % L)
// with 32-bit divisions only: blockIdx.x = qb L + rb gives i = qb kThreads L + j with
// j = rb kThreads + threadIdx.x < L kThreads, so i / L = qb kThreads + j / L.
struct Item { int64_t p; int l; };
// Level-major decode: blocks [l bpl, (l + 1) bpl) take level l of the points (blockIdx.x - l bpl)
// kThreads + threadIdx.x, so that the blocks in flight at any time read one or two levels' tables.
__device__ __forceinline__ Item item_level_major(int bpl) {
  const uint32_t l = blockIdx.x / (uint32_t)bpl;
  return Item{(int64_t)(blockIdx.x - l * (uint32_t)bpl) * kThreads + threadIdx.x, (int)l};
}

__device__ __forceinline__ Item item_of(int L) {
  if ((L & (L - 1)) == 0) {                          // L a power of two: shifts
    const int sh = __ffs(L) - 1;
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    return Item{i >> sh, (int)(i & (L - 1))};
  }
  const uint32_t uL = (uint32_t)L;
  const uint32_t qb = blockIdx.x / uL;
  const uint32_t j = (blockIdx.x - qb * uL) * kThreads + threadIdx.x;
  const uint32_t q = j / uL;
  return Item{(int64_t)qb * kThreads + q, (int)(j - q * uL)};
}

template <int D>
__device__ __forceinline__ void load_point(const float* __restrict__ x, int64_t p, float (&v)[D]) {
  if constexpr (D == 2) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(x) + p);
    v[0] = a.x; v[1] = a.y;
  } else if constexpr (D == 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(x) + p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = __ldg(x + p * D + i);
  }
}

inline unsigned grid_for(int64_t P, int L) { return (unsigned)((P * L + kThreads - 1) / kThreads); }

}  // namespace encode_detail
}  // namespace sxe
