// Device helpers shared by the tcgen05 network kernels (mlp_tc.cu, mlp_tc3.cu): 16-bit packing,
// warp-level mma.sync and ldmatrix/stmatrix, core-matrix tile stores and loads, the tcgen05 product
// over K of two core-matrix tiles, and the named barriers of a 128-thread tile group.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "sxe_internal.cuh"
#include "tc_ptx.cuh"

namespace sxe {
namespace mlpc {

constexpr int kW = 64;                      // hidden width
constexpr int kM = 128;                     // points per tile (tcgen05 M, one TMEM lane each)
constexpr uint32_t kWaitPolls = 1u << 26;   // bound of every mbarrier wait

template <typename T> __device__ __forceinline__ uint32_t pack2(float lo, float hi);
template <> __device__ __forceinline__ uint32_t pack2<__half>(float lo, float hi) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}
template <typename T> __device__ __forceinline__ float2 unpack2(uint32_t u);
template <> __device__ __forceinline__ float2 unpack2<__half>(uint32_t u) {
  return __half22float2(*reinterpret_cast<__half2*>(&u));
}
template <> __device__ __forceinline__ float2 unpack2<__nv_bfloat16>(uint32_t u) {
  return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&u));
}

template <typename T>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if constexpr (std::is_same<T, __half>::value) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], uint32_t saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(saddr));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t& r0, uint32_t& r1, uint32_t saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(saddr));
}

// element (n, k) of a [N][K] core-matrix tile at `base`
template <typename T>
__device__ __forceinline__ T* cm(unsigned char* base, int n, int k, int K) {
  return reinterpret_cast<T*>(base + tc::cm_offset(n, k, K));
}

// row r, columns c0..c0+15 of a K-column core-matrix tile from 16 fp32 values
template <typename T>
__device__ __forceinline__ void store16(unsigned char* tile, int r, int c0, int K, const float (&v)[16]) {
  uint4 lo, hi;
  lo.x = pack2<T>(v[0], v[1]);   lo.y = pack2<T>(v[2], v[3]);   lo.z = pack2<T>(v[4], v[5]);   lo.w = pack2<T>(v[6], v[7]);
  hi.x = pack2<T>(v[8], v[9]);   hi.y = pack2<T>(v[10], v[11]); hi.z = pack2<T>(v[12], v[13]); hi.w = pack2<T>(v[14], v[15]);
  *reinterpret_cast<uint4*>(tile + tc::cm_offset(r, c0, K)) = lo;
  *reinterpret_cast<uint4*>(tile + tc::cm_offset(r, c0 + 8, K)) = hi;
}

template <typename T>
__device__ __forceinline__ void load16(const unsigned char* tile, int r, int c0, int K, float (&v)[16]) {
  const uint4 lo = *reinterpret_cast<const uint4*>(tile + tc::cm_offset(r, c0, K));
  const uint4 hi = *reinterpret_cast<const uint4*>(tile + tc::cm_offset(r, c0 + 8, K));
  const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float2 f = unpack2<T>(w[j]);
    v[2 * j] = f.x;
    v[2 * j + 1] = f.y;
  }
}

// D = A B^T over K (multiple of 16) from two core-matrix tiles (A: [128][K], B: [N][K])
__device__ __forceinline__ void issue_gemm(uint32_t tmem, const unsigned char* A, const unsigned char* B, int K,
                                           uint32_t idesc) {
  const uint32_t sbo = (uint32_t)(K / 8) * 128u;
  const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
  for (int ks = 0; ks < K / 16; ++ks)
    tc::mma_f16(tmem, tc::smem_desc(a0 + ks * 256u, 128u, sbo), tc::smem_desc(b0 + ks * 256u, 128u, sbo), idesc,
                ks > 0);
}

__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// true on every thread of the 128-thread group if `p` holds on any of them (a barrier too)
__device__ __forceinline__ bool group_any(int id, bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, %2, 128, q;\n selp.u32 %0, 1, 0, o;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id)
      : "memory");
  return r != 0;
}

// A fragments of m16n8k16 from a core-matrix tile: matrix i of the four is rows 8 (i % 2) .. + 7,
// columns 8 (i / 2) .. + 7 of the 16 x 16 block; lane l gives the address of row l % 8 of matrix l / 8
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(saddr) : "memory");
}
// the inverse: four 8 x 8 matrices from fragment registers into the rows the lanes address
__device__ __forceinline__ void stsm_x4(uint32_t saddr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};\n"
               :: "r"(saddr), "r"(r0), "r"(r1), "r"(r2), "r"(r3) : "memory");
}

}  // namespace mlpc
}  // namespace sxe
