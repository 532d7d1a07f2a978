// Inline-PTX wrappers for the 5th-generation tensor cores (tcgen05) of sm_100/sm_103:
// shared-memory matrix descriptors, instruction descriptors, TMEM allocation, MMA issue,
// commit to an mbarrier, bounded mbarrier waits and TMEM loads.
//
// Operand layout used throughout: K-major, no swizzle.  A tile of R rows x K elements
// (16-bit) is stored as 8x8 "core matrices" of 128 contiguous bytes (8 rows of 16 bytes);
// element (r, k) sits at byte  (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// with SBO = (K / 8) * 128.  In the descriptor the leading-dimension byte offset is the
// distance between core matrices adjacent in K (128) and the stride-dimension byte offset
// the distance between 8-row groups (SBO).
#pragma once

#include <stdint.h>

namespace sxe {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a core-matrix tile with K columns
__host__ __device__ __forceinline__ int cm_offset(int r, int k, int K) {
  return (r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor (no swizzle, version 1)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: fp32 accumulate, A and B of the same 16-bit type
// (bf16 = 1, fp16 = 0), both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// The same with A and B "MN-major" (transposed): operand element (mn, k) stored with 8 consecutive
// MN elements in 16 contiguous bytes and the 8 k of a core matrix 16 bytes apart.  For these the
// descriptor's leading-dimension offset is the distance between core matrices adjacent in K and
// the stride-dimension offset the distance between core matrices adjacent in MN (measured on
// sm_103a with exactly representable operands).  A tile stored K-major for M = points ([points]
// [features], 8-feature core rows) is thus read, unchanged, as the MN-major operand of a product
// that reduces over the points.
__host__ __device__ constexpr uint32_t idesc_f16_mn(int M, int N, bool bf16) {
  return idesc_f16(M, N, bf16) | (1u << 15) | (1u << 16);
}

// Accumulator rows of an M = 64 product (cta_group::1) sit in TMEM lanes 32 (m / 16) + m % 16:
// warp w % 4 reads rows 16 (w % 4) .. +15 from its lanes 0-15 (measured on sm_103a).

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(dst_smem)),
               "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[desc] * B[desc]^T, issued by one thread
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate) : "memory");
}

// arrive on the mbarrier once every tcgen05 operation issued so far by this thread completes
__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait until the barrier's phase with the given parity has completed; gives up after
// max_iter polls and returns false (the caller records the failure and unwinds).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_iter) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < max_iter; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// The same wait with the polling thread suspended between polls (up to `hint_ns` per poll, woken
// when the phase completes), so that waiting warps take few issue and shared-memory slots; it gives
// up once the global timer shows more than `limit_ns` since the first timed poll (or after
// max_iter polls, whichever comes first) and returns false.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* mbar, uint32_t parity, uint32_t hint_ns, uint64_t limit_ns,
                                                uint32_t max_iter) {
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < max_iter; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity), "r"(hint_ns) : "memory");
    if (done) return true;
    if ((it & 15) == 15) {
      const uint64_t t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
  return false;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make generic-proxy shared-memory writes visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive fp32 columns of this thread's TMEM lane (warp w reads lanes 32*(w%4)..+31)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// N (a multiple of 16) consecutive fp32 columns of this thread's TMEM lane: N / 16 loads in
// flight, then one wait
template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[N]) {
  static_assert(N % 16 == 0, "16-column loads");
  uint32_t r[N];
#pragma unroll
  for (int c = 0; c < N; c += 16)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[c + 0]), "=r"(r[c + 1]), "=r"(r[c + 2]), "=r"(r[c + 3]), "=r"(r[c + 4]), "=r"(r[c + 5]),
                   "=r"(r[c + 6]), "=r"(r[c + 7]), "=r"(r[c + 8]), "=r"(r[c + 9]), "=r"(r[c + 10]), "=r"(r[c + 11]),
                   "=r"(r[c + 12]), "=r"(r[c + 13]), "=r"(r[c + 14]), "=r"(r[c + 15])
                 : "r"(taddr + (uint32_t)c));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < N; ++j) v[j] = __uint_as_float(r[j]);
}

// 64 consecutive fp32 columns of this thread's TMEM lane: two loads in flight, one wait
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
#define SXE_LD32(OFF, B)                                                                                         \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15," \
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                       \
               : "=r"(B[0]), "=r"(B[1]), "=r"(B[2]), "=r"(B[3]), "=r"(B[4]), "=r"(B[5]), "=r"(B[6]), "=r"(B[7]), \
                 "=r"(B[8]), "=r"(B[9]), "=r"(B[10]), "=r"(B[11]), "=r"(B[12]), "=r"(B[13]), "=r"(B[14]),       \
                 "=r"(B[15]), "=r"(B[16]), "=r"(B[17]), "=r"(B[18]), "=r"(B[19]), "=r"(B[20]), "=r"(B[21]),     \
                 "=r"(B[22]), "=r"(B[23]), "=r"(B[24]), "=r"(B[25]), "=r"(B[26]), "=r"(B[27]), "=r"(B[28]),     \
                 "=r"(B[29]), "=r"(B[30]), "=r"(B[31])                                                           \
               : "r"(taddr + (OFF)))
  SXE_LD32(0u, r);
  SXE_LD32(32u, (r + 32));
#undef SXE_LD32
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 64; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 consecutive fp32 columns of this thread's TMEM lane, loaded and waited for in one statement
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace tc
}  // namespace sxe
