// Adam (Kingma & Ba, Algorithm 1) on a binary32 master copy, and the L2 loss of the
// image-fitting task (Sec. 6.1 of arXiv 2311.15439).
//
// Two layouts:
//   * dense SoA arrays (network weights): one thread per parameter;
//   * table entries in an interleaved record {param[F], m[F], v[F], grad[F]} plus a
//     bitmap of entries that received a gradient in this step.  One warp covers the 32
//     entries of one bitmap word: the warp reads the word once, only its marked lanes
//     touch their (consecutive, coalesced) records, and lane 0 clears the word.  An
//     entry that was never marked has gradient zero and is skipped, which is exactly the
//     zero-gradient skip rule applied to every entry.
#include <cmath>

#include "sxe_internal.cuh"

namespace sxe {
namespace {

__global__ void adam_dense_kernel(AdamConst kin, int64_t n, float* __restrict__ p, float* __restrict__ m,
                                  float* __restrict__ v, float* __restrict__ g, void* __restrict__ lowp, int ldt) {
  const AdamConst k = adam_resolve(kin);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    float pi = p[i];
    if (!(k.skip && gi == 0.f)) {
      float mi = m[i], vi = v[i];
      adam_one(k, gi, pi, mi, vi);
      p[i] = pi; m[i] = mi; v[i] = vi;
      g[i] = 0.f;
    }
    if (lowp) store_as(lowp, i, ldt, pi);
  }
}

// The same over 4 consecutive parameters per thread with 16-byte accesses (n a multiple of 4,
// every array 16-byte aligned and the low-precision copy 8-byte aligned).  Every element is
// written back: a skipped element keeps its values and its gradient is already zero, so the
// result equals the scalar kernel's.
__global__ void adam_dense4_kernel(AdamConst kin, int64_t n4, float4* __restrict__ p, float4* __restrict__ m,
                                   float4* __restrict__ v, float4* __restrict__ g, void* __restrict__ lowp,
                                   int ldt) {
  const AdamConst k = adam_resolve(kin);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 gi = g[i];
    float4 pi = p[i], mi = m[i], vi = v[i];
    const float ga[4] = {gi.x, gi.y, gi.z, gi.w};
    float pa[4] = {pi.x, pi.y, pi.z, pi.w}, ma[4] = {mi.x, mi.y, mi.z, mi.w}, va[4] = {vi.x, vi.y, vi.z, vi.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (!(k.skip && ga[j] == 0.f)) adam_one(k, ga[j], pa[j], ma[j], va[j]);
    p[i] = make_float4(pa[0], pa[1], pa[2], pa[3]);
    m[i] = make_float4(ma[0], ma[1], ma[2], ma[3]);
    v[i] = make_float4(va[0], va[1], va[2], va[3]);
    g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lowp) {
      if (ldt == SXE_F32) {
        reinterpret_cast<float4*>(lowp)[i] = make_float4(pa[0], pa[1], pa[2], pa[3]);
      } else if (ldt == SXE_F16) {
        __half2 lo = __floats2half2_rn(pa[0], pa[1]), hi = __floats2half2_rn(pa[2], pa[3]);
        reinterpret_cast<uint2*>(lowp)[i] = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
      } else {
        __nv_bfloat162 lo = __floats2bfloat162_rn(pa[0], pa[1]), hi = __floats2bfloat162_rn(pa[2], pa[3]);
        reinterpret_cast<uint2*>(lowp)[i] = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
      }
    }
  }
}

// A warp takes 32 consecutive bitmap words (1024 entries).  The set bits of the 32 words are
// listed in shared memory in address order (a warp prefix sum of the words' popcounts gives
// each word's place in the list); then the lanes take the listed entries in turn, NB records per
// lane loaded before any is updated, so a warp keeps up to 32 NB record loads in flight however
// sparse the words are.  Each lane clears the word it loaded.
template <int F>
__global__ void __launch_bounds__(256, 4)
adam_touched_kernel(AdamConst kin, int64_t n_entries, float* __restrict__ state, uint32_t* __restrict__ touched,
                    void* __restrict__ lowp, int ldt) {
  const AdamConst k = adam_resolve(kin);
  constexpr int NB = F <= 2 ? 4 : (F == 4 ? 2 : 1);
  __shared__ uint16_t list[8][1024];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t n_words = (n_entries + 31) >> 5;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint16_t* my = list[wib];
  for (int64_t w0 = warp0 << 5; w0 < n_words; w0 += n_warps << 5) {
    const int64_t wi = w0 + lane;
    const uint32_t mine = wi < n_words ? touched[wi] : 0u;
    const int cnt = __popc(mine);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;
    int at = incl - cnt;
    for (uint32_t bits = mine; bits; bits &= bits - 1u) my[at++] = (uint16_t)(lane * 32 + __ffs(bits) - 1);
    __syncwarp();
    const int64_t ebase = w0 << 5;
    for (int i0 = 0; i0 < total; i0 += 32 * NB) {
      int64_t e[NB];
      bool on[NB];
      union Rec { float4 v[F]; float f[4 * F]; } r[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int i = i0 + b * 32 + lane;
        on[b] = i < total;
        e[b] = on[b] ? ebase + my[i] : 0;
        on[b] = on[b] && e[b] < n_entries;
        if (on[b]) {
          const float4* rec = reinterpret_cast<const float4*>(state + e[b] * (4 * F));
#pragma unroll
          for (int j = 0; j < F; ++j) r[b].v[j] = rec[j];
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (on[b]) {
          float p[F];
#pragma unroll
          for (int f = 0; f < F; ++f) {
            float pp = r[b].f[f], mm = r[b].f[F + f], vv = r[b].f[2 * F + f];
            const float g = r[b].f[3 * F + f];
            if (g != 0.f) adam_one(k, g, pp, mm, vv);
            r[b].f[f] = pp; r[b].f[F + f] = mm; r[b].f[2 * F + f] = vv; r[b].f[3 * F + f] = 0.f;
            p[f] = pp;
          }
          float4* rec = reinterpret_cast<float4*>(state + e[b] * (4 * F));
#pragma unroll
          for (int j = 0; j < F; ++j) rec[j] = r[b].v[j];
          store_lowp<F>(lowp, e[b], ldt, p);
        }
    }
    __syncwarp();
    if (mine) touched[wi] = 0u;
  }
}

__global__ void loss_l2_kernel(const float* __restrict__ y, const float* __restrict__ tgt, int64_t n, float scale,
                               float* __restrict__ dy, float* __restrict__ sq_sum) {
  float sq = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = y[i] - tgt[i];
    dy[i] = r * scale;
    sq = fmaf(r, r, sq);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += part[i];
    if (s != 0.f) atomicAdd(sq_sum, s);
  }
}

// Double-word binary32 arithmetic (Dekker 1971; the bounds of Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic", 2017): a value is the
// unevaluated sum hi + lo of two binary32 numbers with |lo| <= ulp(hi) / 2, about 48 significant
// bits.  The product uses the exact error of a binary32 product, fmaf(a, b, -a*b); every other
// operation is an explicitly rounded intrinsic so that no contraction changes the error terms.
struct Dw {
  float hi, lo;
};

__device__ __forceinline__ Dw dw_mul(Dw a, Dw b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);                  // a.hi * b.hi = p + e exactly
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));  // cross terms (a.lo * b.lo is below u^2)
  const float s = __fadd_rn(p, e);                      // Fast2Sum renormalisation, |p| >= |e|
  return {s, __fsub_rn(e, __fsub_rn(s, p))};
}

// 1 / (1 - b) for a double-word b in [0, 1), rounded to binary32: 1 - b by Fast2Sum (|1| >= |b.hi|),
// then one Newton correction of the correctly rounded reciprocal of the leading part, whose
// residual 1 - d.hi * r is exact in one fma.
__device__ __forceinline__ float dw_recip_one_minus(Dw b) {
  const float s = __fadd_rn(1.f, -b.hi);
  const float z = __fsub_rn(s, 1.f);
  const float err = __fsub_rn(-b.hi, z);                // 1 - b.hi = s + err exactly
  const float lo = __fsub_rn(err, b.lo);
  const float dh = __fadd_rn(s, lo), dl = __fsub_rn(lo, __fsub_rn(dh, s));
  const float r = __frcp_rn(dh);
  const float res = __fmaf_rn(-dl, r, __fmaf_rn(-dh, r, 1.f));   // 1 - (dh + dl) r
  return __fmaf_rn(r, res, r);
}

// Two threads: the step count t += 1 and the bias corrections 1 / (1 - beta_i^t) of the new t,
// thread i for beta_i.  beta^t by binary exponentiation in double-word binary32 arithmetic (about
// 2 log2 t products, each with a relative error of a few 2^-48), then 1 / (1 - beta^t) as above:
// the amplification 1 / (1 - beta) <= 100 of the subtraction for beta <= 0.99 keeps the result
// far inside half a binary32 ulp of the exact value before its last rounding.  No FP64 on the
// device.  Near underflow the low parts lose their meaning, but beta^t is then below 2^-100 and
// 1 - beta^t rounds to 1 either way.
__global__ void adam_advance_kernel(int64_t* __restrict__ t, float* __restrict__ c, float b1, float b2) {
  const int64_t tn = *t + 1;
  Dw p = {1.f, 0.f}, x = {threadIdx.x == 0 ? b1 : b2, 0.f};
  for (int64_t e = tn; e > 0; e >>= 1) {
    if (e & 1) p = dw_mul(p, x);
    x = dw_mul(x, x);
  }
  c[threadIdx.x] = dw_recip_one_minus(p);
  __syncthreads();                                      // both threads have read the old t
  if (threadIdx.x == 0) *t = tn;
}

unsigned blocks_for(int64_t n, int threads, unsigned cap) {
  const int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

sxe_status launch_adam_dense(const sxe_adam_desc* a, int64_t t, int64_t n, float* p, float* m, float* v, float* g,
                             void* lowp, int32_t ldt, cudaStream_t s, const float* corrections) {
  AdamConst k = make_adam_const(a, corrections ? 1 : t);
  k.cdev = corrections;
  auto al = [](const void* q, uintptr_t b) { return ((uintptr_t)q % b) == 0; };
  const bool vec = n % 4 == 0 && al(p, 16) && al(m, 16) && al(v, 16) && al(g, 16) &&
                   (!lowp || al(lowp, ldt == SXE_F32 ? 16 : 8));
  if (vec)
    adam_dense4_kernel<<<blocks_for(n / 4, 256, 1u << 16), 256, 0, s>>>(
        k, n / 4, reinterpret_cast<float4*>(p), reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v),
        reinterpret_cast<float4*>(g), lowp, ldt);
  else
    adam_dense_kernel<<<blocks_for(n, 256, 1u << 16), 256, 0, s>>>(k, n, p, m, v, g, lowp, ldt);
  return check_launch("adam_dense");
}

sxe_status launch_adam_touched(const sxe_adam_desc* a, int64_t t, int64_t n_entries, int32_t F, float* state,
                               uint32_t* touched, void* lowp, int32_t ldt, cudaStream_t s, const float* corrections) {
  AdamConst k = make_adam_const(a, corrections ? 1 : t);
  k.cdev = corrections;
  // one warp per 32 bitmap words, at most 16 blocks of 8 warps per SM
  const int sms = device_sm_count();
  const int64_t chunks = (((n_entries + 31) >> 5) + 31) >> 5;
  const unsigned nb = blocks_for(chunks * 32, 256, (unsigned)(16 * sms));
  switch (F) {
    case 1: adam_touched_kernel<1><<<nb, 256, 0, s>>>(k, n_entries, state, touched, lowp, ldt); break;
    case 2: adam_touched_kernel<2><<<nb, 256, 0, s>>>(k, n_entries, state, touched, lowp, ldt); break;
    case 4: adam_touched_kernel<4><<<nb, 256, 0, s>>>(k, n_entries, state, touched, lowp, ldt); break;
    default: adam_touched_kernel<8><<<nb, 256, 0, s>>>(k, n_entries, state, touched, lowp, ldt); break;
  }
  return check_launch("adam_touched");
}

sxe_status launch_loss_l2(const float* y, const float* target, int64_t P, int32_t n_out, float* dy, float* sq_sum,
                          cudaStream_t s) {
  const int64_t n = P * n_out;
  loss_l2_kernel<<<blocks_for(n, 256, 4096), 256, 0, s>>>(y, target, n, (float)(2.0 / (double)n), dy, sq_sum);
  return check_launch("loss_l2");
}

sxe_status launch_adam_advance(const sxe_adam_desc* a, int64_t* t, float* corrections, cudaStream_t s) {
  adam_advance_kernel<<<1, 2, 0, s>>>(t, corrections, a->beta1, a->beta2);
  return check_launch("adam_advance");
}

}  // namespace sxe
