// Lattice arithmetic of the simplex-grid hash encoding (Wen & Yang, arXiv 2311.15439), device
// side: scale + skew (Eq. 2, Sec. 5.1), simplicial subdivision by ranking the fractional parts
// (Sec. 4.2, Remark 2), barycentric weights (Sec. 4.3) and the vertex hash (Sec. 5 a), the 2^d grid
// corners of the comparator (Algorithm 1), and the table entry loads and gradient reductions of
// the encoding kernels.  Included by sxe_internal.cuh; the encoding kernels depend only on this
// header, encode_common.cuh and encode.cu.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "simplexenc.h"

namespace sxe {

// ---------------------------------------------------------------------------
// host-side handle
// ---------------------------------------------------------------------------
struct EncParams {
  int32_t n_levels;
  int32_t log2_T;
  int32_t out_dtype;
  float skew_F;                    // F_n of Eq. 2 rounded to binary32 (simplex only)
  float scale[SXE_MAX_LEVELS];     // per-level input multiplier (binary32)
  uint32_t width[SXE_MAX_LEVELS];  // box width B of a directly indexed level, 0 = hashed
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Hash multipliers per axis: 1, 2654435761, 805459861 (the Instant-NGP spatial hash
// the paper's backbone uses) and, for axes 4 and 5, the smallest primes not below
// frac(sqrt(5)) * 2^32 and frac(sqrt(7)) * 2^32.
__host__ __device__ constexpr uint32_t hash_prime(int axis) {
  return axis == 0 ? 1u : axis == 1 ? 2654435761u : axis == 2 ? 805459861u
       : axis == 3 ? 1013904263u : 2773480771u;
}

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Store `n` binary32 values as dtype `dt` at element offset `off` of `base`.
__device__ __forceinline__ void store_as(void* base, int64_t off, int32_t dt, float v) {
  if (dt == SXE_F32) reinterpret_cast<float*>(base)[off] = v;
  else if (dt == SXE_F16) reinterpret_cast<__half*>(base)[off] = __float2half_rn(v);
  else reinterpret_cast<__nv_bfloat16*>(base)[off] = __float2bfloat16_rn(v);
}

// Raw aligned vector of B bytes.
template <int B> struct RawVec;
template <> struct RawVec<2> { using type = unsigned short; };
template <> struct RawVec<4> { using type = unsigned int; };
template <> struct RawVec<8> { using type = uint2; };
template <> struct RawVec<16> { using type = uint4; };

// Gather the F features of one table entry through the read-only path.
template <typename T, int F>
__device__ __forceinline__ void load_entry(const T* __restrict__ p, float (&o)[F]) {
  constexpr int B = F * (int)sizeof(T);
  if constexpr (B <= 16) {
    using V = typename RawVec<B>::type;
    union { V v; T t[F]; } u;
    u.v = __ldg(reinterpret_cast<const V*>(p));
#pragma unroll
    for (int f = 0; f < F; ++f) o[f] = to_f32(u.t[f]);
  } else {
    union { uint4 v[B / 16]; T t[F]; } u;
#pragma unroll
    for (int j = 0; j < B / 16; ++j) u.v[j] = __ldg(reinterpret_cast<const uint4*>(p) + j);
#pragma unroll
    for (int f = 0; f < F; ++f) o[f] = to_f32(u.t[f]);
  }
}

// Vector atomic add of F binary32 values (8/16-byte vector atomics on sm_90+).
template <int F>
__device__ __forceinline__ void atomic_add_entry(float* p, const float (&v)[F]) {
  if constexpr (F == 1) {
    atomicAdd(p, v[0]);
  } else if constexpr (F == 2) {
    atomicAdd(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
  } else {
#pragma unroll
    for (int j = 0; j < F / 4; ++j)
      atomicAdd(reinterpret_cast<float4*>(p) + j, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
  }
}

// Compare-exchange of a descending sort of (f, axis) with ties broken by the lower axis first,
// carrying each axis's hash step along.
__device__ __forceinline__ void sort_cx(float& fa, int& ia, uint32_t& da, float& fb, int& ib, uint32_t& db) {
  const bool sw = (fb > fa) || (fb == fa && ib < ia);
  const float f = sw ? fb : fa;
  const int i = sw ? ib : ia;
  const uint32_t d = sw ? db : da;
  fb = sw ? fa : fb; ib = sw ? ia : ib; db = sw ? da : db;
  fa = f; ia = i; da = d;
}

// Sorting networks (1, 3, 5 and 9 comparators for 2, 3, 4 and 5 keys).
template <int D>
__device__ __forceinline__ void sort_desc(float (&f)[D], int (&ix)[D], uint32_t (&dl)[D]) {
#define SXE_CX(a, b) sort_cx(f[a], ix[a], dl[a], f[b], ix[b], dl[b])
  if constexpr (D == 2) {
    SXE_CX(0, 1);
  } else if constexpr (D == 3) {
    SXE_CX(0, 1); SXE_CX(1, 2); SXE_CX(0, 1);
  } else if constexpr (D == 4) {
    SXE_CX(0, 1); SXE_CX(2, 3); SXE_CX(0, 2); SXE_CX(1, 3); SXE_CX(1, 2);
  } else {
    static_assert(D == 5, "d = 2..5");
    SXE_CX(0, 1); SXE_CX(3, 4); SXE_CX(2, 4); SXE_CX(2, 3); SXE_CX(0, 3);
    SXE_CX(0, 2); SXE_CX(1, 4); SXE_CX(1, 3); SXE_CX(1, 2);
  }
#undef SXE_CX
}

// ---------------------------------------------------------------------------
// Simplex lattice of one point at one level.
//   Sec. 5.1 + Eq. 2: p_i = x_i * s, sigma = sum_i p_i (left to right), t = F * sigma,
//   q_i = p_i + t; each operation rounded once (no contraction).
//   Sec. 4.2: c = floor(q), f = q - c (exact); the fractional parts are sorted in decreasing
//   order, ties lower axis first (a sorting network carrying the axis and its hash step).
//   Remark 2: vertex k = c + the unit vectors of the first k sorted axes; its slot is the base
//   vertex's hash updated by the hash steps of those axes.
//   Sec. 4.3: w_0 = 1 - s_0, w_k = s_{k-1} - s_k, w_d = s_{d-1} on the sorted s.
//   Sec. 5 (a): slot = XOR_i (uint32(v_i) * prime_i) mod T; on a directly indexed level
//   (width B > 0) slot = (sum_i uint32(v_i) * B^i) mod T instead.  rank_i is the position of
//   axis i in the sorted order.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void simplex_lattice(const float (&x)[D], float s, float skewF, uint32_t mask,
                                                uint32_t width, uint32_t (&slot)[D + 1], float (&w)[D + 1],
                                                int (&rank)[D], int (&cell)[D]) {
  float p[D];
#pragma unroll
  for (int i = 0; i < D; ++i) p[i] = __fmul_rn(x[i], s);
  float sigma = p[0];
#pragma unroll
  for (int i = 1; i < D; ++i) sigma = __fadd_rn(sigma, p[i]);
  const float t = __fmul_rn(skewF, sigma);
  float f[D];
  int ix[D];
  uint32_t dl[D];
  uint32_t h = 0, pw = 1u;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const float q = __fadd_rn(p[i], t);
    const float fl = floorf(q);
    f[i] = __fsub_rn(q, fl);
    cell[i] = __float2int_rz(fl);
    const uint32_t c = (uint32_t)cell[i];
    const uint32_t mult = width ? pw : hash_prime(i);
    pw *= width;
    const uint32_t h0 = c * mult;
    h = width ? h + h0 : h ^ h0;
    dl[i] = width ? mult : (h0 ^ (h0 + mult));          // hash step of moving +1 along axis i
    ix[i] = i;
  }
  sort_desc<D>(f, ix, dl);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    int r = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) r = ix[k] == i ? k : r;
    rank[i] = r;
  }
  w[0] = __fsub_rn(1.f, f[0]);
#pragma unroll
  for (int k = 1; k < D; ++k) w[k] = __fsub_rn(f[k - 1], f[k]);
  w[D] = f[D - 1];
  slot[0] = h & mask;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    h = width ? h + dl[k] : h ^ dl[k];
    slot[k + 1] = h & mask;
  }
}

template <int D>
__device__ __forceinline__ void simplex_lattice(const float (&x)[D], float s, float skewF, uint32_t mask,
                                                uint32_t width, uint32_t (&slot)[D + 1], float (&w)[D + 1],
                                                int (&rank)[D]) {
  int cell[D];
  simplex_lattice<D>(x, s, skewF, mask, width, slot, w, rank, cell);
}

template <int D>
__device__ __forceinline__ void simplex_lattice(const float (&x)[D], float s, float skewF, uint32_t mask,
                                                uint32_t width, uint32_t (&slot)[D + 1], float (&w)[D + 1]) {
  int rank[D];
  simplex_lattice<D>(x, s, skewF, mask, width, slot, w, rank);
}

// 2^D grid corners of one point at one level (Algorithm 1's multilinear weights):
// p_i = x_i * N (binary32), c = floor(p), f = p - c; corner b (axis 0 = most
// significant bit) has weight prod_i (b_i ? f_i : 1 - f_i), multiplied in axis order.
template <int D>
__device__ __forceinline__ void grid_lattice(const float (&x)[D], float N, uint32_t mask, uint32_t width,
                                             uint32_t (&slot)[1 << D], float (&w)[1 << D], float (&f)[D],
                                             int (&cell)[D]) {
  uint32_t h0[D], h1[D];
  uint32_t pw = 1u;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const float p = __fmul_rn(x[i], N);
    const float fl = floorf(p);
    f[i] = __fsub_rn(p, fl);
    cell[i] = __float2int_rz(fl);
    const uint32_t c = (uint32_t)cell[i];
    const uint32_t mult = width ? pw : hash_prime(i);
    pw *= width;
    h0[i] = c * mult;
    h1[i] = (c + 1u) * mult;
  }
#pragma unroll
  for (int b = 0; b < (1 << D); ++b) {
    float wt = 1.f;
    uint32_t h = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const bool bi = (b >> (D - 1 - i)) & 1;
      wt = __fmul_rn(wt, bi ? f[i] : __fsub_rn(1.f, f[i]));
      const uint32_t v = bi ? h1[i] : h0[i];
      h = width ? h + v : h ^ v;
    }
    w[b] = wt;
    slot[b] = h & mask;
  }
}

template <int D>
__device__ __forceinline__ void grid_lattice(const float (&x)[D], float N, uint32_t mask, uint32_t width,
                                             uint32_t (&slot)[1 << D], float (&w)[1 << D], float (&f)[D]) {
  int cell[D];
  grid_lattice<D>(x, N, mask, width, slot, w, f, cell);
}

template <int D>
__device__ __forceinline__ void grid_lattice(const float (&x)[D], float N, uint32_t mask, uint32_t width,
                                             uint32_t (&slot)[1 << D], float (&w)[1 << D]) {
  float f[D];
  grid_lattice<D>(x, N, mask, width, slot, w, f);
}

// Table slot of lattice vertex v under a level's rule (hash, or direct index for width > 0).
template <int D>
__device__ __forceinline__ uint32_t vertex_slot(const uint32_t (&v)[D], uint32_t width, uint32_t mask) {
  uint32_t h = 0, pw = 1u;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    h = width ? h + v[i] * pw : h ^ (v[i] * hash_prime(i));
    pw *= width;
  }
  return h & mask;
}

}  // namespace sxe
