// Multiresolution simplex / grid hash encoding kernels (Sec. 5 a-e of arXiv 2311.15439,
// and the 2^d grid of Algorithm 1 as comparator).
//
// Work item = one (point, level) pair, flattened as i = p * L + l so that consecutive
// threads write consecutive F-feature groups of the [P][L*F] output (coalesced) and
// read consecutive groups of dout; the forward can also take the items level by level
// (fwd_level_major below).  Every item issues its V = d+1 (simplex) or 2^d (grid)
// independent gathers before it consumes any of them.
#include <algorithm>

#include "encode_common.cuh"

namespace sxe {
namespace {

using namespace encode_detail;

template <bool SIMPLEX, int D, int F, typename TT>
__global__ void __launch_bounds__(kThreads)
encode_fwd_kernel(const float* __restrict__ x, int64_t P, const TT* __restrict__ tables, int64_t tstride,
                  void* __restrict__ out, const EncParams prm, uint32_t* __restrict__ touched, int bpl) {
  constexpr int V = Verts<SIMPLEX, D>::V;
  __shared__ float s_scale[SXE_MAX_LEVELS];
  __shared__ uint32_t s_width[SXE_MAX_LEVELS];
  if (threadIdx.x < SXE_MAX_LEVELS) {
    s_scale[threadIdx.x] = prm.scale[threadIdx.x];
    s_width[threadIdx.x] = prm.width[threadIdx.x];
  }
  __syncthreads();
  const int L = prm.n_levels;
  const Item it = bpl ? item_level_major(bpl) : item_of(L);
  if (it.p >= P) return;
  float xv[D];
  load_point<D>(x, it.p, xv);
  const uint32_t mask = (1u << prm.log2_T) - 1u;
  uint32_t slot[V];
  float w[V];
  lattice<SIMPLEX, D>(xv, s_scale[it.l], prm.skew_F, mask, s_width[it.l], slot, w);
  const TT* tab = tables + ((int64_t)it.l << prm.log2_T) * tstride;
  float val[V][F];
#pragma unroll
  for (int k = 0; k < V; ++k) load_entry<TT, F>(tab + (int64_t)slot[k] * tstride, val[k]);
  if (touched) {
    // mark every entry read (the entries the backward of the same points adds to), while the
    // gathers are in flight: all bitmap words first, then the missing bits
    const int64_t lbase = (int64_t)it.l << prm.log2_T;
    uint32_t words[V];
#pragma unroll
    for (int k = 0; k < V; ++k) words[k] = __ldcg(touched + ((lbase + slot[k]) >> 5));
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int64_t e = lbase + slot[k];
      const uint32_t bit = 1u << (uint32_t)(e & 31);
      if (!(words[k] & bit)) atomicOr(touched + (e >> 5), bit);
    }
  }
  float acc[F];
#pragma unroll
  for (int f = 0; f < F; ++f) acc[f] = 0.f;
#pragma unroll
  for (int k = 0; k < V; ++k)
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = fmaf(w[k], val[k][f], acc[f]);
  const int64_t o = (it.p * L + it.l) * F;
  if (prm.out_dtype == SXE_F32) {
    float* po = reinterpret_cast<float*>(out) + o;
    if constexpr (F == 2) *reinterpret_cast<float2*>(po) = make_float2(acc[0], acc[1]);
    else {
#pragma unroll
      for (int f = 0; f < F; ++f) po[f] = acc[f];
    }
  } else if (prm.out_dtype == SXE_F16) {
    __half* po = reinterpret_cast<__half*>(out) + o;
    if constexpr (F == 2) *reinterpret_cast<__half2*>(po) = __floats2half2_rn(acc[0], acc[1]);
    else {
#pragma unroll
      for (int f = 0; f < F; ++f) po[f] = __float2half_rn(acc[f]);
    }
  } else {
    __nv_bfloat16* po = reinterpret_cast<__nv_bfloat16*>(out) + o;
    if constexpr (F == 2) *reinterpret_cast<__nv_bfloat162*>(po) = __floats2bfloat162_rn(acc[0], acc[1]);
    else {
#pragma unroll
      for (int f = 0; f < F; ++f) po[f] = __float2bfloat16_rn(acc[f]);
    }
  }
}

// Levels [l0, l0 + nl) of every point; work item i = p * nl + (l - l0).
template <bool SIMPLEX, int D, int F>
__global__ void __launch_bounds__(kThreads)
encode_bwd_kernel(const float* __restrict__ x, int64_t P, const float* __restrict__ dout,
                  float* __restrict__ grad, int64_t stride, uint32_t* __restrict__ touched,
                  const EncParams prm, int l0, int nl) {
  constexpr int V = Verts<SIMPLEX, D>::V;
  __shared__ float s_scale[SXE_MAX_LEVELS];
  __shared__ uint32_t s_width[SXE_MAX_LEVELS];
  if (threadIdx.x < SXE_MAX_LEVELS) {
    s_scale[threadIdx.x] = prm.scale[threadIdx.x];
    s_width[threadIdx.x] = prm.width[threadIdx.x];
  }
  __syncthreads();
  const int L = prm.n_levels;
  Item it = item_of(nl);
  if (it.p >= P) return;
  it.l += l0;
  // issue the gradient and point loads first, the lattice arithmetic overlaps them
  float g[F];
  const float* pd = dout + (it.p * L + it.l) * F;
  if constexpr (F == 2) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(pd));
    g[0] = a.x; g[1] = a.y;
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f) g[f] = __ldg(pd + f);
  }
  float xv[D];
  load_point<D>(x, it.p, xv);
  const uint32_t mask = (1u << prm.log2_T) - 1u;
  uint32_t slot[V];
  float w[V];
  lattice<SIMPLEX, D>(xv, s_scale[it.l], prm.skew_F, mask, s_width[it.l], slot, w);
  const int64_t lbase = (int64_t)it.l << prm.log2_T;
  // all bitmap words in flight at once, then the (fire-and-forget) atomics, then the marks
  uint32_t words[V];
  if (touched) {
#pragma unroll
    for (int k = 0; k < V; ++k) words[k] = __ldcg(touched + ((lbase + slot[k]) >> 5));
  }
#pragma unroll
  for (int k = 0; k < V; ++k) {
    float c[F];
#pragma unroll
    for (int f = 0; f < F; ++f) c[f] = w[k] * g[f];
    atomic_add_entry<F>(grad + (lbase + slot[k]) * stride, c);
  }
  if (touched) {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int64_t e = lbase + slot[k];
      const uint32_t bit = 1u << (uint32_t)(e & 31);
      if (!(words[k] & bit)) atomicOr(touched + (e >> 5), bit);
    }
  }
}

// Backward with warp-level sums of colliding terms, for batches whose consecutive points are
// spatially coherent (the samples of a ray).  Block b takes the 32 points [32 b, 32 b + 32) and
// warp w the levels l0 + w, l0 + w + 8, ... of them, lane i point 32 b + i, so the 32 lanes of a
// warp add into the same level's table.  For every vertex k the lanes whose entries coincide are
// found with match.any; a lane alone adds its term directly, a group sums its terms in the warp's
// shared scratch and its lowest lane adds the sum with one reduction.  dout rows are read through
// L1 (the 8 warps of a block read the 16 levels of the same 32 rows).
constexpr int kAggPoints = 32;

template <bool SIMPLEX, int D, int F>
__global__ void __launch_bounds__(kThreads)
encode_bwd_agg_kernel(const float* __restrict__ x, int64_t P, const float* __restrict__ dout,
                      float* __restrict__ grad, int64_t stride, uint32_t* __restrict__ touched,
                      const EncParams prm, int l0, int nl) {
  constexpr int V = Verts<SIMPLEX, D>::V;
  constexpr int kWarps = kThreads / 32;
  __shared__ float s_scr[kWarps][32][F];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int f = 0; f < F; ++f) s_scr[warp][lane][f] = 0.f;
  __syncwarp();
  const int L = prm.n_levels;
  const int64_t p = (int64_t)blockIdx.x * kAggPoints + lane;
  const bool live = p < P;
  float xv[D];
  if (live) load_point<D>(x, p, xv);
  else {
#pragma unroll
    for (int i = 0; i < D; ++i) xv[i] = 0.f;
  }
  const uint32_t mask = (1u << prm.log2_T) - 1u;
  for (int l = l0 + warp; l < l0 + nl; l += kWarps) {
    float g[F];
#pragma unroll
    for (int f = 0; f < F; ++f) g[f] = live ? __ldg(dout + (p * L + l) * F + f) : 0.f;
    uint32_t slot[V];
    float w[V];
    lattice<SIMPLEX, D>(xv, prm.scale[l], prm.skew_F, mask, prm.width[l], slot, w);
    const int64_t lbase = (int64_t)l << prm.log2_T;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const uint32_t key = live ? slot[k] : 0xffffffffu;        // slots are < T <= 2^26
      const uint32_t peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      float c[F];
#pragma unroll
      for (int f = 0; f < F; ++f) c[f] = w[k] * g[f];
      const bool alone = __popc(peers) == 1;
      if (live && !alone) {
#pragma unroll
        for (int f = 0; f < F; ++f) atomicAdd(&s_scr[warp][leader][f], c[f]);
      }
      __syncwarp();
      if (live && (alone || lane == leader)) {
        if (!alone) {
#pragma unroll
          for (int f = 0; f < F; ++f) {
            c[f] = s_scr[warp][lane][f];
            s_scr[warp][lane][f] = 0.f;
          }
        }
        const int64_t e = lbase + slot[k];
        atomic_add_entry<F>(grad + e * stride, c);
        if (touched) {
          const uint32_t bit = 1u << (uint32_t)(e & 31);
          if (!(__ldcg(touched + (e >> 5)) & bit)) atomicOr(touched + (e >> 5), bit);
        }
      }
      __syncwarp();
    }
  }
}

template <bool SIMPLEX, int D>
__global__ void __launch_bounds__(kThreads)
encode_vertices_kernel(const float* __restrict__ x, int64_t P, uint32_t* __restrict__ slots,
                       float* __restrict__ weights, const EncParams prm) {
  constexpr int V = Verts<SIMPLEX, D>::V;
  const int L = prm.n_levels;
  const Item it = item_of(L);
  if (it.p >= P) return;
  float xv[D];
  load_point<D>(x, it.p, xv);
  uint32_t slot[V];
  float w[V];
  lattice<SIMPLEX, D>(xv, prm.scale[it.l], prm.skew_F, (1u << prm.log2_T) - 1u, prm.width[it.l], slot, w);
  const int64_t o = (it.p * L + it.l) * V;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    if (slots) slots[o + k] = slot[k];
    if (weights) weights[o + k] = w[k];
  }
}


// ---- dispatch ---------------------------------------------------------------
// Coarse levels, privately per CTA.  The lattice box of a coarse level has few vertices
// (B^d, B coordinates per axis) that receive many contributions each, and same-address
// reductions serialise in L2.  CTA k of level c sums the contributions of its chunk of the
// points in shared memory, indexed by the vertex's box coordinate sum_i v_i B^i, marks the
// vertices it touched in a shared bitmap, then adds each touched vertex to its table slot
// once.  Vertices outside the box (points outside [0,1]^d) take the global path directly.
constexpr int kMaxCoarse = 4;
constexpr int kCoarseSmem = 48 * 1024;

struct CoarsePlan {
  int first;                                // level of plan entry 0
  int n;                                    // coarse levels first..first+n-1
  int start[kMaxCoarse + 1];                // CTAs of level c: [start[c], start[c+1])
  uint32_t box[kMaxCoarse];                 // box width B of level c
  int smem;                                 // dynamic shared memory bytes
};

template <bool SIMPLEX, int D, int F>
__global__ void __launch_bounds__(kThreads)
encode_bwd_coarse_kernel(const float* __restrict__ x, int64_t P, const float* __restrict__ dout,
                         float* __restrict__ grad, int64_t stride, uint32_t* __restrict__ touched,
                         const EncParams prm, const CoarsePlan plan) {
  constexpr int V = Verts<SIMPLEX, D>::V;
  extern __shared__ float s_acc[];
  int c = 0;                                            // plan entry; its level is plan.first + c
  while (c + 1 < plan.n && (int)blockIdx.x >= plan.start[c + 1]) ++c;
  const uint32_t B = c == 0 ? plan.box[0] : c == 1 ? plan.box[1] : c == 2 ? plan.box[2] : plan.box[3];
  const int lev = plan.first + c;
  uint32_t cells = 1;
#pragma unroll
  for (int i = 0; i < D; ++i) cells *= B;
  uint32_t* s_flag = reinterpret_cast<uint32_t*>(s_acc + cells * F);
  for (uint32_t i = threadIdx.x; i < cells * F; i += kThreads) s_acc[i] = 0.f;
  for (uint32_t i = threadIdx.x; i < (cells + 31) / 32; i += kThreads) s_flag[i] = 0u;
  __syncthreads();
  const int L = prm.n_levels;
  const int K = plan.start[c + 1] - plan.start[c];
  const int k = (int)blockIdx.x - plan.start[c];
  const int64_t p0 = P * k / K, p1 = P * (k + 1) / K;
  const uint32_t mask = (1u << prm.log2_T) - 1u;
  const uint32_t width = prm.width[lev];
  const float s = prm.scale[lev];
  const int64_t lbase = (int64_t)lev << prm.log2_T;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) {
    float g[F];
    const float* pd = dout + (p * L + lev) * F;
#pragma unroll
    for (int f = 0; f < F; ++f) g[f] = __ldg(pd + f);
    float xv[D];
    load_point<D>(x, p, xv);
    uint32_t box[V];
    float w[V];
    int cell[D];
    bool inside = true;
    if constexpr (SIMPLEX) {
      int rank[D];
      simplex_lattice<D>(xv, s, prm.skew_F, 0xffffffffu, B, box, w, rank, cell);
#pragma unroll
      for (int i = 0; i < D; ++i) inside &= cell[i] >= 0 && cell[i] <= (int)B - 2;
      if (!inside) {
#pragma unroll
        for (int kk = 0; kk < V; ++kk) {
          uint32_t v[D];
#pragma unroll
          for (int i = 0; i < D; ++i) v[i] = (uint32_t)cell[i] + (rank[i] < kk ? 1u : 0u);
          box[kk] = vertex_slot<D>(v, width, mask);
        }
      }
    } else {
      float fr[D];
      grid_lattice<D>(xv, s, 0xffffffffu, B, box, w, fr, cell);
#pragma unroll
      for (int i = 0; i < D; ++i) inside &= cell[i] >= 0 && cell[i] <= (int)B - 2;
      if (!inside) {
#pragma unroll
        for (int b = 0; b < V; ++b) {
          uint32_t v[D];
#pragma unroll
          for (int i = 0; i < D; ++i) v[i] = (uint32_t)cell[i] + ((b >> (D - 1 - i)) & 1);
          box[b] = vertex_slot<D>(v, width, mask);
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < V; ++kk) {
      if (inside) {
#pragma unroll
        for (int f = 0; f < F; ++f) atomicAdd(s_acc + box[kk] * F + f, w[kk] * g[f]);
        atomicOr(s_flag + (box[kk] >> 5), 1u << (box[kk] & 31));
      } else {
        float cc[F];
#pragma unroll
        for (int f = 0; f < F; ++f) cc[f] = w[kk] * g[f];
        const int64_t e = lbase + box[kk];
        atomic_add_entry<F>(grad + e * stride, cc);
        if (touched) atomicOr(touched + (e >> 5), 1u << (uint32_t)(e & 31));
      }
    }
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < cells; b += kThreads) {
    if (!((s_flag[b >> 5] >> (b & 31)) & 1u)) continue;
    uint32_t v[D], r = b;
#pragma unroll
    for (int i = 0; i < D; ++i) { v[i] = r % B; r /= B; }
    const int64_t e = lbase + vertex_slot<D>(v, width, mask);
    float cc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) cc[f] = s_acc[b * F + f];
    atomic_add_entry<F>(grad + e * stride, cc);
    if (touched) {
      const uint32_t bit = 1u << (uint32_t)(e & 31);
      if (!(__ldcg(touched + (e >> 5)) & bit)) atomicOr(touched + (e >> 5), bit);
    }
  }
}

// Input gradient: dx[p][i] += sum over levels and features of dout * d out / d x_i.
// Simplex (Sec. 4.3 weights): inside the point's simplex the output is affine in the
// fractional parts, and moving f along the axis of rank k shifts weight from vertex k to
// vertex k+1, so d out / d q_i = H(v_{rank_i + 1}) - H(v_{rank_i}); Eq. 2's skew matrix
// is symmetric (d/dp_j = g_j + F_n sum_i g_i) and p = x s_l.  Grid (Algorithm 1): the
// derivative of the n-linear weights along each axis, times N_l.  The levels of one point
// are consecutive lanes: a segmented shuffle reduction leaves one atomic add per axis per
// point and warp.
template <bool SIMPLEX, int D, int F, typename TT>
__global__ void __launch_bounds__(kThreads)
encode_dx_kernel(const float* __restrict__ x, int64_t P, const TT* __restrict__ tables,
                 const float* __restrict__ dout, float* __restrict__ dx, const EncParams prm) {
  constexpr int V = Verts<SIMPLEX, D>::V;
  __shared__ float s_scale[SXE_MAX_LEVELS];
  __shared__ uint32_t s_width[SXE_MAX_LEVELS];
  if (threadIdx.x < SXE_MAX_LEVELS) {
    s_scale[threadIdx.x] = prm.scale[threadIdx.x];
    s_width[threadIdx.x] = prm.width[threadIdx.x];
  }
  __syncthreads();
  const int L = prm.n_levels;
  const Item it = item_of(L);
  const bool live = it.p < P;
  float g[D];
#pragma unroll
  for (int i = 0; i < D; ++i) g[i] = 0.f;
  if (live) {
    float xv[D];
    load_point<D>(x, it.p, xv);
    float dl[F];
    const float* pd = dout + (it.p * L + it.l) * F;
#pragma unroll
    for (int f = 0; f < F; ++f) dl[f] = __ldg(pd + f);
    const uint32_t mask = (1u << prm.log2_T) - 1u;
    const float s = s_scale[it.l];
    uint32_t slot[V];
    float w[V];
    const TT* tab = tables + ((int64_t)it.l << prm.log2_T) * F;
    if constexpr (SIMPLEX) {
      int rank[D];
      simplex_lattice<D>(xv, s, prm.skew_F, mask, s_width[it.l], slot, w, rank);
      float proj[V];                                  // dout . H(v_k)
#pragma unroll
      for (int k = 0; k < V; ++k) {
        float h[F];
        load_entry<TT, F>(tab + (int64_t)slot[k] * F, h);
        float a = 0.f;
#pragma unroll
        for (int f = 0; f < F; ++f) a = fmaf(dl[f], h[f], a);
        proj[k] = a;
      }
      float gq[D], sum = 0.f;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) v = (rank[i] == k) ? proj[k + 1] - proj[k] : v;
        gq[i] = v;
        sum += v;
      }
      const float t = prm.skew_F * sum;
#pragma unroll
      for (int i = 0; i < D; ++i) g[i] = s * (gq[i] + t);
    } else {
      float fr[D];
      grid_lattice<D>(xv, s, mask, s_width[it.l], slot, w, fr);
      float proj[V];
#pragma unroll
      for (int k = 0; k < V; ++k) {
        float h[F];
        load_entry<TT, F>(tab + (int64_t)slot[k] * F, h);
        float a = 0.f;
#pragma unroll
        for (int f = 0; f < F; ++f) a = fmaf(dl[f], h[f], a);
        proj[k] = a;
      }
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float a = 0.f;
#pragma unroll
        for (int b = 0; b < V; ++b) {
          float wt = 1.f;
#pragma unroll
          for (int i = 0; i < D; ++i) {
            const bool bi = (b >> (D - 1 - i)) & 1;
            if (i == j) wt = bi ? wt : -wt;
            else wt *= bi ? fr[i] : 1.f - fr[i];
          }
          a = fmaf(wt, proj[b], a);
        }
        g[j] = s * a;
      }
    }
  }
  // segmented reduction over the lanes that hold levels of the same point
  const int lane = threadIdx.x & 31;
  const uint32_t key = live ? (uint32_t)it.p : 0xffffffffu;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t ko = __shfl_down_sync(0xffffffffu, key, o);
    const bool take = lane + o < 32 && ko == key;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float v = __shfl_down_sync(0xffffffffu, g[i], o);
      if (take) g[i] += v;
    }
  }
  const uint32_t kprev = __shfl_up_sync(0xffffffffu, key, 1);
  if (live && (lane == 0 || kprev != key)) {
#pragma unroll
    for (int i = 0; i < D; ++i) atomicAdd(dx + it.p * D + i, g[i]);
  }
}

template <bool SIMPLEX, int D, int F>
sxe_status dx_tt(const sxe_encoder* e, const float* x, int64_t P, const void* tab, const float* dout, float* dx,
                 cudaStream_t s) {
  const unsigned g = grid_for(P, e->prm.n_levels);
  switch (e->desc.table_dtype) {
    case SXE_F32: encode_dx_kernel<SIMPLEX, D, F, float><<<g, kThreads, 0, s>>>(x, P, (const float*)tab, dout, dx, e->prm); break;
    case SXE_F16: encode_dx_kernel<SIMPLEX, D, F, __half><<<g, kThreads, 0, s>>>(x, P, (const __half*)tab, dout, dx, e->prm); break;
    default: encode_dx_kernel<SIMPLEX, D, F, __nv_bfloat16><<<g, kThreads, 0, s>>>(x, P, (const __nv_bfloat16*)tab, dout, dx, e->prm); break;
  }
  return check_launch("encode_bwd_input");
}

template <bool SIMPLEX, int D>
sxe_status dx_f(const sxe_encoder* e, const float* x, int64_t P, const void* t, const float* d, float* dx, cudaStream_t s) {
  switch (e->desc.n_features) {
    case 1: return dx_tt<SIMPLEX, D, 1>(e, x, P, t, d, dx, s);
    case 2: return dx_tt<SIMPLEX, D, 2>(e, x, P, t, d, dx, s);
    case 4: return dx_tt<SIMPLEX, D, 4>(e, x, P, t, d, dx, s);
    default: return dx_tt<SIMPLEX, D, 8>(e, x, P, t, d, dx, s);
  }
}

template <bool SIMPLEX>
sxe_status dx_d(const sxe_encoder* e, const float* x, int64_t P, const void* t, const float* d, float* dx, cudaStream_t s) {
  switch (e->desc.d) {
    case 2: return dx_f<SIMPLEX, 2>(e, x, P, t, d, dx, s);
    case 3: return dx_f<SIMPLEX, 3>(e, x, P, t, d, dx, s);
    case 4: return dx_f<SIMPLEX, 4>(e, x, P, t, d, dx, s);
    default: return dx_f<SIMPLEX, 5>(e, x, P, t, d, dx, s);
  }
}

}  // namespace

sxe_status launch_encode_bwd_input(const sxe_encoder* enc, const float* x, int64_t P, const void* tables,
                                   const float* dout, float* dx, cudaStream_t s) {
  return enc->desc.kind == SXE_SIMPLEX ? dx_d<true>(enc, x, P, tables, dout, dx, s)
                                       : dx_d<false>(enc, x, P, tables, dout, dx, s);
}

namespace {

// The forward's work-item order.  Point-major (the level fastest) keeps every level's table in use
// at once, which suits tables that L2 holds.  Level-major (blocks of consecutive points of one
// level, the levels in turn) keeps one or two levels' tables in use at a time, so that where the
// tables together exceed L2 but one level's fits, a sector fetched for one point stays in L2 for
// the later points of its level: image workload (16 levels of 16 MB fp16) 71 -> 60 us per
// forward; the SDF-style workload (32 MB of tables in all) 0.750 -> 0.764 ms per step the other
// way.  The backward keeps the point-major order (level-major re-reads each dout sector once per
// level: image 313 -> 324 us).
bool fwd_level_major(const sxe_encoder* enc, int64_t entry_stride) {
  if (enc->fwd_order != SXE_FWD_ORDER_AUTO) return enc->fwd_order == SXE_FWD_ORDER_LEVEL_MAJOR;
  const int64_t level_bytes = (entry_stride << enc->desc.log2_T) * (enc->desc.table_dtype == SXE_F32 ? 4 : 2);
  const int64_t l2 = device_l2_bytes();
  return level_bytes * enc->desc.n_levels > l2 && 2 * level_bytes <= l2;
}

template <bool SIMPLEX, int D, int F>
sxe_status fwd_tt(const sxe_encoder* enc, const float* x, int64_t P, const void* tab, int64_t ts, void* out,
                  uint32_t* touched, cudaStream_t s) {
  const int bpl = fwd_level_major(enc, ts) ? (int)((P + kThreads - 1) / kThreads) : 0;
  const unsigned g = bpl ? (unsigned)bpl * enc->prm.n_levels : grid_for(P, enc->prm.n_levels);
  switch (enc->desc.table_dtype) {
    case SXE_F32: encode_fwd_kernel<SIMPLEX, D, F, float><<<g, kThreads, 0, s>>>(x, P, (const float*)tab, ts, out, enc->prm, touched, bpl); break;
    case SXE_F16: encode_fwd_kernel<SIMPLEX, D, F, __half><<<g, kThreads, 0, s>>>(x, P, (const __half*)tab, ts, out, enc->prm, touched, bpl); break;
    default: encode_fwd_kernel<SIMPLEX, D, F, __nv_bfloat16><<<g, kThreads, 0, s>>>(x, P, (const __nv_bfloat16*)tab, ts, out, enc->prm, touched, bpl); break;
  }
  return check_launch("encode_fwd");
}

template <bool SIMPLEX, int D>
sxe_status fwd_f(const sxe_encoder* e, const float* x, int64_t P, const void* t, int64_t ts, void* o, uint32_t* tm,
                 cudaStream_t s) {
  switch (e->desc.n_features) {
    case 1: return fwd_tt<SIMPLEX, D, 1>(e, x, P, t, ts, o, tm, s);
    case 2: return fwd_tt<SIMPLEX, D, 2>(e, x, P, t, ts, o, tm, s);
    case 4: return fwd_tt<SIMPLEX, D, 4>(e, x, P, t, ts, o, tm, s);
    default: return fwd_tt<SIMPLEX, D, 8>(e, x, P, t, ts, o, tm, s);
  }
}

template <bool SIMPLEX>
sxe_status fwd_d(const sxe_encoder* e, const float* x, int64_t P, const void* t, int64_t ts, void* o, uint32_t* tm,
                 cudaStream_t s) {
  switch (e->desc.d) {
    case 2: return fwd_f<SIMPLEX, 2>(e, x, P, t, ts, o, tm, s);
    case 3: return fwd_f<SIMPLEX, 3>(e, x, P, t, ts, o, tm, s);
    case 4: return fwd_f<SIMPLEX, 4>(e, x, P, t, ts, o, tm, s);
    default: return fwd_f<SIMPLEX, 5>(e, x, P, t, ts, o, tm, s);
  }
}

// Coarse levels for the privatised backward: a prefix of levels whose box fits the shared
// memory budget and receives at least 8 contributions per vertex.  A level gets one CTA per
// 4096 contributions, fewer if a CTA would then see under 1 contribution per vertex, and at
// most 2 per SM: short per-thread loops (the kernel is latency-bound), a flush of at most
// one global reduction per contribution into L2-resident entries, and each table entry
// receives at most K flushed sums instead of thousands of single terms (measured: 324.7 ->
// 315.0 us for the image backward against 8192 and 4 per vertex; 2048 and 1/2 was slower).
CoarsePlan coarse_plan(const sxe_encoder* e, int64_t P) {
  CoarsePlan plan{};
  const int d = e->desc.d, F = e->desc.n_features;
  const int64_t V = e->desc.kind == SXE_SIMPLEX ? d + 1 : (1 << d);
  const int sms = device_sm_count();
  plan.start[0] = 0;
  for (int c = 0; c < kMaxCoarse && c < e->prm.n_levels; ++c) {
    const uint32_t B = e->box_width[c];
    if (B == 0) break;
    int64_t cells = 1;
    for (int i = 0; i < d; ++i) cells *= B;
    const int64_t bytes = cells * F * 4 + (cells + 31) / 32 * 4;
    if (bytes > kCoarseSmem || P * V < 8 * cells) break;
    const int64_t K = std::max<int64_t>(1, std::min<int64_t>(std::min(P * V / 4096, P * V / cells), 2 * sms));
    plan.box[c] = B;
    plan.start[c + 1] = plan.start[c] + (int)K;
    plan.smem = std::max(plan.smem, (int)bytes);
    plan.n = c + 1;
  }
  return plan;
}

// The part of the plan inside levels [lb, le): its coarse levels, renumbered from lb.
CoarsePlan slice_plan(const CoarsePlan& full, int lb, int le) {
  CoarsePlan plan{};
  plan.first = lb;
  const int c1 = std::min(full.n, le);
  for (int c = lb; c < c1; ++c) {
    plan.box[c - lb] = full.box[c];
    plan.start[c - lb + 1] = full.start[c + 1] - full.start[lb];
    plan.n = c - lb + 1;
  }
  plan.smem = plan.n > 0 ? full.smem : 0;
  return plan;
}

template <bool SIMPLEX, int D, int F>
sxe_status bwd_f(const sxe_encoder* e, const float* x, int64_t P, const float* dout, float* g, int64_t stride,
                 uint32_t* touched, cudaStream_t s, int lb, int le) {
  const CoarsePlan full = coarse_plan(e, P);
  const CoarsePlan plan = slice_plan(full, lb, le);
  if (plan.n > 0) {
    encode_bwd_coarse_kernel<SIMPLEX, D, F><<<plan.start[plan.n], kThreads, plan.smem, s>>>(
        x, P, dout, g, stride, touched, e->prm, plan);
    sxe_status st = check_launch("encode_bwd_coarse");
    if (st != SXE_OK) return st;
  }
  const int l0 = std::max(lb, full.n);
  const int nl = le - l0;
  if (nl <= 0) return SXE_OK;
  if (e->bwd_aggregate) {
    const unsigned nb = (unsigned)((P + kAggPoints - 1) / kAggPoints);
    encode_bwd_agg_kernel<SIMPLEX, D, F><<<nb, kThreads, 0, s>>>(x, P, dout, g, stride, touched, e->prm, l0, nl);
    return check_launch("encode_bwd_agg");
  }
  encode_bwd_kernel<SIMPLEX, D, F><<<grid_for(P, nl), kThreads, 0, s>>>(x, P, dout, g, stride, touched, e->prm,
                                                                       l0, nl);
  return check_launch("encode_bwd");
}

template <bool SIMPLEX, int D>
sxe_status bwd_fd(const sxe_encoder* e, const float* x, int64_t P, const float* dout, float* g, int64_t stride,
                  uint32_t* t, cudaStream_t s, int lb, int le) {
  switch (e->desc.n_features) {
    case 1: return bwd_f<SIMPLEX, D, 1>(e, x, P, dout, g, stride, t, s, lb, le);
    case 2: return bwd_f<SIMPLEX, D, 2>(e, x, P, dout, g, stride, t, s, lb, le);
    case 4: return bwd_f<SIMPLEX, D, 4>(e, x, P, dout, g, stride, t, s, lb, le);
    default: return bwd_f<SIMPLEX, D, 8>(e, x, P, dout, g, stride, t, s, lb, le);
  }
}

template <bool SIMPLEX>
sxe_status bwd_d(const sxe_encoder* e, const float* x, int64_t P, const float* dout, float* g, int64_t stride,
                 uint32_t* t, cudaStream_t s, int lb, int le) {
  switch (e->desc.d) {
    case 2: return bwd_fd<SIMPLEX, 2>(e, x, P, dout, g, stride, t, s, lb, le);
    case 3: return bwd_fd<SIMPLEX, 3>(e, x, P, dout, g, stride, t, s, lb, le);
    case 4: return bwd_fd<SIMPLEX, 4>(e, x, P, dout, g, stride, t, s, lb, le);
    default: return bwd_fd<SIMPLEX, 5>(e, x, P, dout, g, stride, t, s, lb, le);
  }
}

template <bool SIMPLEX>
sxe_status verts_d(const sxe_encoder* e, const float* x, int64_t P, uint32_t* sl, float* w, cudaStream_t s) {
  const unsigned g = grid_for(P, e->prm.n_levels);
  switch (e->desc.d) {
    case 2: encode_vertices_kernel<SIMPLEX, 2><<<g, kThreads, 0, s>>>(x, P, sl, w, e->prm); break;
    case 3: encode_vertices_kernel<SIMPLEX, 3><<<g, kThreads, 0, s>>>(x, P, sl, w, e->prm); break;
    case 4: encode_vertices_kernel<SIMPLEX, 4><<<g, kThreads, 0, s>>>(x, P, sl, w, e->prm); break;
    default: encode_vertices_kernel<SIMPLEX, 5><<<g, kThreads, 0, s>>>(x, P, sl, w, e->prm); break;
  }
  return check_launch("encode_vertices");
}

}  // namespace

sxe_status launch_encode_fwd(const sxe_encoder* enc, const float* x, int64_t P, const void* tables, void* out,
                             cudaStream_t s, int64_t table_stride, uint32_t* touched) {
  if (table_stride <= 0) table_stride = enc->desc.n_features;
  return enc->desc.kind == SXE_SIMPLEX ? fwd_d<true>(enc, x, P, tables, table_stride, out, touched, s)
                                       : fwd_d<false>(enc, x, P, tables, table_stride, out, touched, s);
}

sxe_status launch_encode_bwd(const sxe_encoder* enc, const float* x, int64_t P, const float* dout, float* grad,
                             int64_t stride, uint32_t* touched, cudaStream_t s, int level_begin, int level_end) {
  if (level_end < 0) level_end = enc->prm.n_levels;
  return enc->desc.kind == SXE_SIMPLEX ? bwd_d<true>(enc, x, P, dout, grad, stride, touched, s, level_begin, level_end)
                                       : bwd_d<false>(enc, x, P, dout, grad, stride, touched, s, level_begin, level_end);
}

int encode_bwd_coarse_levels(const sxe_encoder* enc, int64_t P) { return coarse_plan(enc, P).n; }

int encode_bwd_launches(const sxe_encoder* enc, int64_t P, int level_begin, int level_end) {
  if (level_end < 0) level_end = enc->prm.n_levels;
  if (P == 0 || level_begin >= level_end) return 0;
  const CoarsePlan full = coarse_plan(enc, P);
  const CoarsePlan plan = slice_plan(full, level_begin, level_end);
  return (plan.n > 0 ? 1 : 0) + (std::max(level_begin, full.n) < level_end ? 1 : 0);
}

sxe_status launch_encode_vertices(const sxe_encoder* enc, const float* x, int64_t P, uint32_t* slots,
                                  float* weights, cudaStream_t s) {
  return enc->desc.kind == SXE_SIMPLEX ? verts_d<true>(enc, x, P, slots, weights, s)
                                       : verts_d<false>(enc, x, P, slots, weights, s);
}

}  // namespace sxe
