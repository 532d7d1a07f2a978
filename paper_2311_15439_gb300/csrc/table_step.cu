// Training update of the feature tables, one level at a time (Sec. 5 e of arXiv
// 2311.15439: the loss gradient is accumulated in the looked-up entries; then Adam).
//
// For each level l:
//   1. table_bwd_level_kernel: every point's d+1 (or 2^d) vertices at level l add
//      w_k * dL/d(enc)[p][l*F + f] into a dense binary32 scratch [T][F] with vector atomics
//      and mark the entries in the level's slice of the touched bitmap.  The scratch is the
//      same 32 MiB (T = 2^22, F = 2) for every level, so it stays resident in L2 and the
//      atomics hit there instead of pulling random DRAM sectors.
//   2. table_adam_level_kernel: for every marked entry, Adam on its record (zero-gradient
//      skip rule per parameter), refresh the low-precision copy inside the same record, zero
//      the scratch gradient and clear the bit -- leaving scratch and bitmap zero again.
//
// State record of entry e = l*T + slot: 4F binary32 words
//   [0, F) parameter, [F, 2F) first moment, [2F, 3F) second moment,
//   [3F, 4F) the table-dtype copy of the parameter packed from its start (the rest zero).
// Each record is written whole (one 32-byte sector for F = 2), and the forward pass gathers
// the low-precision copy straight from it (entry stride 4F words).
#include <algorithm>

#include "sxe_internal.cuh"

namespace sxe {
namespace {

constexpr int kThreads = 256;

template <bool SIMPLEX, int D> struct NV { static constexpr int V = SIMPLEX ? D + 1 : (1 << D); };

template <bool SIMPLEX, int D, int F>
__global__ void __launch_bounds__(kThreads)
table_bwd_level_kernel(const float* __restrict__ x, int64_t P, const float* __restrict__ dout, int L, int l,
                       float scale, float skewF, uint32_t mask, float* __restrict__ scratch,
                       uint32_t* __restrict__ touched_l) {
  constexpr int V = NV<SIMPLEX, D>::V;
  const int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= P) return;
  float xv[D];
#pragma unroll
  for (int i = 0; i < D; ++i) xv[i] = __ldg(x + p * D + i);
  uint32_t slot[V];
  float w[V];
  if constexpr (SIMPLEX) simplex_lattice<D>(xv, scale, skewF, mask, slot, w);
  else grid_lattice<D>(xv, scale, mask, slot, w);
  float g[F];
#pragma unroll
  for (int f = 0; f < F; ++f) g[f] = __ldg(dout + (p * L + l) * F + f);
#pragma unroll
  for (int k = 0; k < V; ++k) {
    float c[F];
#pragma unroll
    for (int f = 0; f < F; ++f) c[f] = w[k] * g[f];
    atomic_add_entry<F>(scratch + (int64_t)slot[k] * F, c);
    const uint32_t bit = 1u << (slot[k] & 31u);
    uint32_t* word = touched_l + (slot[k] >> 5);
    if (!(__ldcg(word) & bit)) atomicOr(word, bit);
  }
}

template <int F, typename LT>
__device__ __forceinline__ void update_record(const AdamConst& k, float* rec_f, float* grad) {
  union { float4 v[F]; float f[4 * F]; } r;
  float4* rec = reinterpret_cast<float4*>(rec_f);
#pragma unroll
  for (int j = 0; j < F; ++j) r.v[j] = rec[j];
  float g[F];
#pragma unroll
  for (int f = 0; f < F; ++f) { g[f] = grad[f]; grad[f] = 0.f; }
#pragma unroll
  for (int f = 0; f < F; ++f) {
    float pp = r.f[f], mm = r.f[F + f], vv = r.f[2 * F + f];
    if (g[f] != 0.f) adam_one(k, g[f], pp, mm, vv);
    r.f[f] = pp; r.f[F + f] = mm; r.f[2 * F + f] = vv;
  }
  // low-precision copy packed at the start of the last F words, the rest zero
  union { float f[F]; LT t[F * 4 / (int)sizeof(LT)]; } low;
#pragma unroll
  for (int f = 0; f < F; ++f) low.f[f] = 0.f;
#pragma unroll
  for (int f = 0; f < F; ++f) low.t[f] = from_f32<LT>(r.f[f]);
#pragma unroll
  for (int f = 0; f < F; ++f) r.f[3 * F + f] = low.f[f];
#pragma unroll
  for (int j = 0; j < F; ++j) rec[j] = r.v[j];
}

// Same warp-chunked bitmap walk as the whole-table step: a warp loads 32 words at once and
// visits the nonzero ones, its lanes taking the word's 32 entries.
template <int F, typename LT>
__global__ void __launch_bounds__(kThreads)
table_adam_level_kernel(AdamConst k, int64_t T, float* __restrict__ state_l, float* __restrict__ scratch,
                        uint32_t* __restrict__ touched_l) {
  const int lane = threadIdx.x & 31;
  const int64_t n_words = T >> 5;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = warp0 << 5; w0 < n_words; w0 += n_warps << 5) {
    const int64_t wi = w0 + lane;
    const uint32_t mine = wi < n_words ? touched_l[wi] : 0u;
    uint32_t todo = __ballot_sync(0xffffffffu, mine != 0u);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1u;
      const uint32_t bits = __shfl_sync(0xffffffffu, mine, src);
      const int64_t e = ((w0 + src) << 5) + lane;
      if ((bits >> lane) & 1u) update_record<F, LT>(k, state_l + e * (4 * F), scratch + e * F);
    }
    if (mine) touched_l[wi] = 0u;
  }
}

template <bool SIMPLEX, int D, int F>
void launch_bwd_level(const sxe_encoder* e, const float* x, int64_t P, const float* dout, int l, float* scratch,
                      uint32_t* touched_l, cudaStream_t s) {
  const unsigned g = (unsigned)((P + kThreads - 1) / kThreads);
  table_bwd_level_kernel<SIMPLEX, D, F><<<g, kThreads, 0, s>>>(x, P, dout, e->prm.n_levels, l, e->prm.scale[l],
                                                                e->prm.skew_F, (1u << e->prm.log2_T) - 1u,
                                                                scratch, touched_l);
}

template <bool SIMPLEX, int D>
void bwd_level_f(const sxe_encoder* e, const float* x, int64_t P, const float* dout, int l, float* scratch,
                 uint32_t* t, cudaStream_t s) {
  switch (e->desc.n_features) {
    case 1: launch_bwd_level<SIMPLEX, D, 1>(e, x, P, dout, l, scratch, t, s); break;
    case 2: launch_bwd_level<SIMPLEX, D, 2>(e, x, P, dout, l, scratch, t, s); break;
    case 4: launch_bwd_level<SIMPLEX, D, 4>(e, x, P, dout, l, scratch, t, s); break;
    default: launch_bwd_level<SIMPLEX, D, 8>(e, x, P, dout, l, scratch, t, s); break;
  }
}

template <bool SIMPLEX>
void bwd_level_d(const sxe_encoder* e, const float* x, int64_t P, const float* dout, int l, float* scratch,
                 uint32_t* t, cudaStream_t s) {
  switch (e->desc.d) {
    case 2: bwd_level_f<SIMPLEX, 2>(e, x, P, dout, l, scratch, t, s); break;
    case 3: bwd_level_f<SIMPLEX, 3>(e, x, P, dout, l, scratch, t, s); break;
    case 4: bwd_level_f<SIMPLEX, 4>(e, x, P, dout, l, scratch, t, s); break;
    default: bwd_level_f<SIMPLEX, 5>(e, x, P, dout, l, scratch, t, s); break;
  }
}

template <typename LT>
void adam_level_t(int F, const AdamConst& k, int64_t T, float* st, float* scratch, uint32_t* t, unsigned nb,
                  cudaStream_t s) {
  switch (F) {
    case 1: table_adam_level_kernel<1, LT><<<nb, kThreads, 0, s>>>(k, T, st, scratch, t); break;
    case 2: table_adam_level_kernel<2, LT><<<nb, kThreads, 0, s>>>(k, T, st, scratch, t); break;
    case 4: table_adam_level_kernel<4, LT><<<nb, kThreads, 0, s>>>(k, T, st, scratch, t); break;
    default: table_adam_level_kernel<8, LT><<<nb, kThreads, 0, s>>>(k, T, st, scratch, t); break;
  }
}

}  // namespace

sxe_status launch_table_step(const sxe_encoder* e, const sxe_adam_desc* adam, int64_t t, const float* x, int64_t P,
                             const float* dout, float* state, float* scratch, uint32_t* touched, cudaStream_t s) {
  const AdamConst k = make_adam_const(adam, t);
  const int F = e->desc.n_features;
  const int64_t T = (int64_t)1 << e->desc.log2_T;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t chunks = ((T >> 5) + 31) >> 5;                        // 32-word chunks per level
  const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((chunks + 7) / 8, 16 * sms));
  for (int l = 0; l < e->desc.n_levels; ++l) {
    uint32_t* tl = touched + ((l * T) >> 5);
    float* sl = state + (int64_t)l * T * 4 * F;
    if (P > 0) {
      if (e->desc.kind == SXE_SIMPLEX) bwd_level_d<true>(e, x, P, dout, l, scratch, tl, s);
      else bwd_level_d<false>(e, x, P, dout, l, scratch, tl, s);
    }
    switch (e->desc.table_dtype) {
      case SXE_F32: adam_level_t<float>(F, k, T, sl, scratch, tl, nb, s); break;
      case SXE_F16: adam_level_t<__half>(F, k, T, sl, scratch, tl, nb, s); break;
      default: adam_level_t<__nv_bfloat16>(F, k, T, sl, scratch, tl, nb, s); break;
    }
    sxe_status st = check_launch("table_step");
    if (st != SXE_OK) return st;
  }
  return SXE_OK;
}

}  // namespace sxe
