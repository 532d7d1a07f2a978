// Training update of the feature tables (Sec. 5 e of arXiv 2311.15439: the loss gradient is
// accumulated in the looked-up entries; then Adam with the zero-gradient skip rule).
//
// State record of entry e = l*T + slot: 4F binary32 words {param[F], m[F], v[F], grad[F]};
// the forward pass reads a separate dense [L][T][F] low-precision copy of the parameters.
// dL/d(encoding) arrives level-major, [L][P][F], so every level's slice is contiguous.
//
// Coarse levels (lattice box (N_l+2)^d <= T/4: few distinct entries, their records stay in
// L2) are handled together: scatter into the records' grad fields with vector atomics and
// the touched bitmap, then the bitmap-driven Adam over their entries.  Every finer level l
// is handled on its own:
//   1. table_bwd_level_kernel: the level's contributions go into a dense binary32 scratch
//      [T][F] with vector atomics, marking the level's slice of the bitmap.  The scratch is
//      reused by every fine level, so it stays resident in L2 and the atomics hit there
//      instead of pulling a random DRAM sector each;
//   2. table_adam_level_kernel: each marked entry takes Adam from its scratch gradient,
//      writes its record whole (one 32-byte sector for F = 2) and its low-precision copy,
//      and clears scratch and bit again.
#include <algorithm>
#include <cmath>

#include "sxe_internal.cuh"

namespace sxe {
namespace {

constexpr int kThreads = 256;

template <bool SIMPLEX, int D> struct NV { static constexpr int V = SIMPLEX ? D + 1 : (1 << D); };

template <bool SIMPLEX, int D, int F>
__global__ void __launch_bounds__(kThreads)
table_bwd_level_kernel(const float* __restrict__ x, int64_t P, const float* __restrict__ dout_l,
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
  if constexpr (F == 2) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(dout_l) + p);
    g[0] = a.x; g[1] = a.y;
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f) g[f] = __ldg(dout_l + p * F + f);
  }
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

template <int F>
__device__ __forceinline__ void update_record(const AdamConst& k, float* rec_f, float* grad, void* lowp, int64_t e,
                                              int ldt) {
  union { float4 v[F]; float f[4 * F]; } r;
  float4* rec = reinterpret_cast<float4*>(rec_f);
#pragma unroll
  for (int j = 0; j < F; ++j) r.v[j] = rec[j];
  float p[F];
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const float g = grad[f];
    grad[f] = 0.f;
    float pp = r.f[f], mm = r.f[F + f], vv = r.f[2 * F + f];
    if (g != 0.f) adam_one(k, g, pp, mm, vv);
    r.f[f] = pp; r.f[F + f] = mm; r.f[2 * F + f] = vv;
    p[f] = pp;
  }
#pragma unroll
  for (int j = 0; j < F; ++j) rec[j] = r.v[j];
  store_lowp<F>(lowp, e, ldt, p);
}

// Same warp-chunked bitmap walk as the whole-table step: a warp loads 32 words at once and
// visits the nonzero ones, its lanes taking the word's 32 entries.
template <int F>
__global__ void __launch_bounds__(kThreads)
table_adam_level_kernel(AdamConst k, int64_t T, float* __restrict__ state_l, float* __restrict__ scratch,
                        uint32_t* __restrict__ touched_l, void* __restrict__ lowp_l, int ldt) {
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
      if ((bits >> lane) & 1u) update_record<F>(k, state_l + e * (4 * F), scratch + e * F, lowp_l, e, ldt);
    }
    if (mine) touched_l[wi] = 0u;
  }
}

template <bool SIMPLEX, int D, int F>
void launch_bwd_level(const sxe_encoder* e, const float* x, int64_t P, const float* dout_l, int l, float* scratch,
                      uint32_t* touched_l, cudaStream_t s) {
  const unsigned g = (unsigned)((P + kThreads - 1) / kThreads);
  table_bwd_level_kernel<SIMPLEX, D, F><<<g, kThreads, 0, s>>>(x, P, dout_l, e->prm.scale[l], e->prm.skew_F,
                                                                (1u << e->prm.log2_T) - 1u, scratch, touched_l);
}

template <bool SIMPLEX, int D>
void bwd_level_f(const sxe_encoder* e, const float* x, int64_t P, const float* dout_l, int l, float* scratch,
                 uint32_t* t, cudaStream_t s) {
  switch (e->desc.n_features) {
    case 1: launch_bwd_level<SIMPLEX, D, 1>(e, x, P, dout_l, l, scratch, t, s); break;
    case 2: launch_bwd_level<SIMPLEX, D, 2>(e, x, P, dout_l, l, scratch, t, s); break;
    case 4: launch_bwd_level<SIMPLEX, D, 4>(e, x, P, dout_l, l, scratch, t, s); break;
    default: launch_bwd_level<SIMPLEX, D, 8>(e, x, P, dout_l, l, scratch, t, s); break;
  }
}

template <bool SIMPLEX>
void bwd_level_d(const sxe_encoder* e, const float* x, int64_t P, const float* dout_l, int l, float* scratch,
                 uint32_t* t, cudaStream_t s) {
  switch (e->desc.d) {
    case 2: bwd_level_f<SIMPLEX, 2>(e, x, P, dout_l, l, scratch, t, s); break;
    case 3: bwd_level_f<SIMPLEX, 3>(e, x, P, dout_l, l, scratch, t, s); break;
    case 4: bwd_level_f<SIMPLEX, 4>(e, x, P, dout_l, l, scratch, t, s); break;
    default: bwd_level_f<SIMPLEX, 5>(e, x, P, dout_l, l, scratch, t, s); break;
  }
}

void adam_level(int F, const AdamConst& k, int64_t T, float* st, float* scratch, uint32_t* t, void* lowp, int ldt,
                unsigned nb, cudaStream_t s) {
  switch (F) {
    case 1: table_adam_level_kernel<1><<<nb, kThreads, 0, s>>>(k, T, st, scratch, t, lowp, ldt); break;
    case 2: table_adam_level_kernel<2><<<nb, kThreads, 0, s>>>(k, T, st, scratch, t, lowp, ldt); break;
    case 4: table_adam_level_kernel<4><<<nb, kThreads, 0, s>>>(k, T, st, scratch, t, lowp, ldt); break;
    default: table_adam_level_kernel<8><<<nb, kThreads, 0, s>>>(k, T, st, scratch, t, lowp, ldt); break;
  }
}

}  // namespace

// Levels whose lattice box (N_l + 2)^d holds at most T/4 vertices.
int table_step_coarse_levels(const sxe_encoder* e) {
  const double T = (double)((int64_t)1 << e->desc.log2_T);
  int lc = 0;
  while (lc < e->desc.n_levels && std::pow((double)e->level_res[lc] + 2.0, (double)e->desc.d) <= T / 4.0) ++lc;
  return lc;
}

sxe_status launch_table_step(const sxe_encoder* e, const sxe_adam_desc* adam, int64_t t, const float* x, int64_t P,
                             const float* dout, float* state, void* table_lowp, float* scratch, uint32_t* touched,
                             cudaStream_t s) {
  const AdamConst k = make_adam_const(adam, t);
  const int F = e->desc.n_features;
  const int L = e->desc.n_levels;
  const int64_t T = (int64_t)1 << e->desc.log2_T;
  const int ldt = e->desc.table_dtype;
  const size_t esz = ldt == SXE_F32 ? 4 : 2;
  const int lc = table_step_coarse_levels(e);
  if (lc > 0) {
    if (P > 0) {
      sxe_status st = launch_encode_bwd(e, x, P, dout, state + 3 * F, 4 * F, touched, s, 0, lc, true);
      if (st != SXE_OK) return st;
    }
    sxe_adam_desc a = *adam;
    a.skip_zero_grad = 1;
    sxe_status st = launch_adam_touched(&a, t, (int64_t)lc * T, F, state, touched, table_lowp, ldt, s);
    if (st != SXE_OK) return st;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t chunks = ((T >> 5) + 31) >> 5;                        // 32-word chunks per level
  const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((chunks + 7) / 8, 16 * sms));
  for (int l = lc; l < L; ++l) {
    uint32_t* tl = touched + ((l * T) >> 5);
    float* sl = state + (int64_t)l * T * 4 * F;
    void* lowp_l = static_cast<char*>(table_lowp) + (size_t)l * T * F * esz;
    if (P > 0) {
      if (e->desc.kind == SXE_SIMPLEX) bwd_level_d<true>(e, x, P, dout + (int64_t)l * P * F, l, scratch, tl, s);
      else bwd_level_d<false>(e, x, P, dout + (int64_t)l * P * F, l, scratch, tl, s);
    }
    adam_level(F, k, T, sl, scratch, tl, lowp_l, ldt, nb, s);
    sxe_status st = check_launch("table_step");
    if (st != SXE_OK) return st;
  }
  return SXE_OK;
}

}  // namespace sxe
