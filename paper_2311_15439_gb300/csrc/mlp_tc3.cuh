// Kernel and launchers (templates) of the three-tile network training pass, instantiated by
// mlp_tc3.cu (n_out <= 8) and mlp_tc3_wide.cu (n_out <= 16).
//
// Tiny fully connected network, training pass (forward, L2 loss or upstream gradient, backward,
// weight gradients) on the 5th-generation tensor cores -- Sec. 5 (d)-(e) and Sec. 6.1 of
// arXiv 2311.15439 -- for networks with a narrow output layer (n_out <= 16), up to three 128-point
// tiles in flight per CTA.
//
// Each 128-thread group (warps 4g .. 4g+3) owns one tile at a time, its shared-memory buffers,
// its TMEM columns, an mbarrier and a named barrier; thread q*32 + lane of a group holds row
// 32 q + lane of its tile, which is TMEM lane 32 q + lane.  The tile's chain of tcgen05 products
// (M = 128 rows = points, fp32 accumulators in TMEM, issued by one thread of the group) is
//   H_0 = relu(X W_0^T),  H_h = relu(H_{h-1} W_h^T)                        NH products
//   dH_{h-1} = (dH_h W_h) * [H_{h-1} > 0],  with dW_h += dH_h^T H_{h-1}     NH - 1 products
//   dX = dH_0 W_0,  with dW_0 += dH_0^T X                                  1 product
// The output layer Y = H_last W_out^T, the loss dY = 2 (Y - target) / (count n_out) * loss_scale
// (or dY = dout * loss_scale) and dH_last = (dY W_out) * [H_last > 0] run in the last hidden
// layer's epilogue on warp-level mma.sync, each warp on its own 32 rows with no group barrier, and
// dW_out += dY^T H_last runs on mma.sync into registers while the next tcgen05 product is in
// flight: the narrow output layer adds no tensor-core round trip to the chain (2 NH products per
// tile instead of 2 NH + 2).  The weight gradients dW_h, dW_0 (M = 64 products over the tile's
// points, reading the K-major activation and delta tiles as MN-major operands) accumulate in the
// group's TMEM columns over the persistent loop.  The ReLU masks are applied to packed 16-bit
// pairs, with the mask taken from the stored (rounded) activations as in the other kernels.
//
// Each CTA writes one partial row of weight gradients: the groups' accumulators summed in group
// order (the tiles of a group and of a CTA are fixed by the launch shape), then the rows of all
// CTAs in a fixed order by the reduction kernel, so results are deterministic.
//
// Every mbarrier wait is bounded: on timeout the error word is raised, the group leaves its loop
// as a whole, the CTA writes its partials, frees TMEM and returns.
#pragma once

#include <algorithm>
#include <type_traits>

#include "mlp_tc_common.cuh"

namespace sxe {

int* tc3_error_word();   // device address of the tensor-core error word (current device)
sxe_status launch_mlp_bwd_tc3_wide(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                                   const float* target, float loss_scale, int64_t P, float* din, float* dW,
                                   float* sq_sum, float* ws, int grid, cudaStream_t s, int din_group, int64_t lc);
sxe_status launch_mlp_fwd_tc3(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out,
                              void* act, cudaStream_t s);   // n_out <= 16 (mlp_tc3_fwd.cu)

namespace {

using namespace mlpc;

constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr uint32_t kSleepNs = 20000;             // longest suspension of one mbarrier poll
constexpr uint64_t kLimitNs = 2000000000ull;     // a wait gives up after 2 s of global time
constexpr uint32_t kSleepPolls = 1u << 20;       // or after this many polls (at most 21 s suspended)

// Shared memory and TMEM plan of one CTA (G groups).
template <int N_IN, int NH>
struct Tc3 {
  static constexpr int COLS = (64 + 64 * (NH - 1) + N_IN + 31) / 32 * 32;   // TMEM columns per group
  static constexpr int X = 0;                                  // [128][N_IN]
  static constexpr int H = X + kM * N_IN * 2;                  // NH x [128][64]: H_h, dH_h in place (h < NH-1)
  static constexpr int DH = H + NH * kM * kW * 2;              // [128][64]: dH_{NH-1}
  static constexpr int DY = DH + kM * kW * 2;                  // [128][16]: dY, outputs >= n_out zero
  static constexpr int GROUP = DY + kM * 16 * 2;
  static constexpr int WBYTES = (2 * kW * N_IN + 2 * (NH - 1) * kW * kW + 2 * 16 * kW) * 2;
  static constexpr int G = cmin(3, cmin(512 / COLS, (227 * 1024 - WBYTES) / GROUP));
  static constexpr int W0 = G * GROUP;                         // [64][N_IN]   B of the first layer
  static constexpr int W0T = W0 + kW * N_IN * 2;               // [N_IN][64]   B of dX
  static constexpr int WH = W0T + N_IN * kW * 2;               // (NH-1) x [64][64]
  static constexpr int WHT = WH + (NH - 1) * kW * kW * 2;      // (NH-1) x [64][64] transposed
  static constexpr int WO = WHT + (NH - 1) * kW * kW * 2;      // [16][64]   W_out, rows >= n_out zero
  static constexpr int WOT = WO + 16 * kW * 2;                 // [64][16]   W_out transposed
  static constexpr int END = WOT + kW * 16 * 2;
  static constexpr int THREADS = 128 * G;
  // the input gradient is staged in the group's first activation buffer (16 KB) while dW_0 still
  // reads dH_0 (EARLY), or in the first two (or the first and DH) after dW_0 completed
  static constexpr bool EARLY = kM * N_IN * 4 <= kM * kW * 2;
  // a group's weight-gradient partial in shared memory (floats): dW_h rows padded to 68, dW_0 rows
  // to N_IN + 4, then dW_out [16][64]
  static constexpr int PH = 0;
  static constexpr int P0 = PH + (NH - 1) * kW * (kW + 4);
  static constexpr int PO = P0 + kW * (N_IN + 4);
  static constexpr int PSTRIDE = PO + 16 * kW;
  // at least 116 KB, so that one CTA (holding all 512 TMEM columns) runs per SM
  static constexpr int SMEM = END > 116 * 1024 ? END : 116 * 1024;
  static_assert(G >= 2, "two tiles per CTA at least");
  static_assert(kM * N_IN * 4 <= GROUP - H, "input-gradient staging fits the group's activation buffers");
  static_assert(G * PSTRIDE * 4 <= END, "the groups' partials fit the shared buffers");
};

template <typename T> __device__ __forceinline__ uint32_t bits16(T v);
template <> __device__ __forceinline__ uint32_t bits16<__half>(__half v) { return __half_as_ushort(v); }
template <> __device__ __forceinline__ uint32_t bits16<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }

// two 16-bit values of W as one fragment register (lo in the low half), zero where `keep` is false
template <typename T>
__device__ __forceinline__ uint32_t wpair(const T* W, int i_lo, int i_hi, bool keep_lo, bool keep_hi) {
  return (keep_lo ? bits16<T>(W[i_lo]) : 0u) | ((keep_hi ? bits16<T>(W[i_hi]) : 0u) << 16);
}

// relu(lo), relu(hi) rounded to a packed 16-bit pair (one conversion with relu clamping)
template <typename T> __device__ __forceinline__ uint32_t pack2_relu(float lo, float hi);
template <> __device__ __forceinline__ uint32_t pack2_relu<__half>(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
template <> __device__ __forceinline__ uint32_t pack2_relu<__nv_bfloat16>(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// the packed pair d where the packed activations h are positive, zero elsewhere
template <typename T> __device__ __forceinline__ uint32_t keep_where_positive(uint32_t d, uint32_t h);
template <> __device__ __forceinline__ uint32_t keep_where_positive<__half>(uint32_t d, uint32_t h) {
  return d & __hgt2_mask(*reinterpret_cast<const __half2*>(&h), __float2half2_rn(0.f));
}
template <> __device__ __forceinline__ uint32_t keep_where_positive<__nv_bfloat16>(uint32_t d, uint32_t h) {
  return d & __hgt2_mask(*reinterpret_cast<const __nv_bfloat162*>(&h), __float2bfloat162_rn(0.f));
}

template <typename T, int N_IN, int NH, typename S>
__device__ void load_weights_tc3(const T* __restrict__ W, int n_out, unsigned char* sm) {
  constexpr int P0 = kW * N_IN / 8, PH = (NH - 1) * kW * kW / 8;     // 8-element pieces
  constexpr int NP = (P0 + PH + S::THREADS - 1) / S::THREADS;
  uint4 v[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const int i = threadIdx.x + j * S::THREADS;
    v[j] = i < P0 + PH ? __ldg(reinterpret_cast<const uint4*>(W) + i) : make_uint4(0, 0, 0, 0);
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const int i = threadIdx.x + j * S::THREADS;
    if (i >= P0 + PH) break;
    const T* e = reinterpret_cast<const T*>(&v[j]);
    if (i < P0) {
      const int o = i / (N_IN / 8), c = (i % (N_IN / 8)) * 8;
      *reinterpret_cast<uint4*>(sm + S::W0 + tc::cm_offset(o, c, N_IN)) = v[j];
#pragma unroll
      for (int k = 0; k < 8; ++k) *cm<T>(sm + S::W0T, c + k, o, kW) = e[k];
    } else {
      const int ih = i - P0, h = ih / (kW * kW / 8), o = (ih / (kW / 8)) % kW, c = (ih % (kW / 8)) * 8;
      *reinterpret_cast<uint4*>(sm + S::WH + h * kW * kW * 2 + tc::cm_offset(o, c, kW)) = v[j];
#pragma unroll
      for (int k = 0; k < 8; ++k) *cm<T>(sm + S::WHT + h * kW * kW * 2, c + k, o, kW) = e[k];
    }
  }
  const T* Wo = W + kW * N_IN + (NH - 1) * kW * kW;
  constexpr int NO = (16 * kW + S::THREADS - 1) / S::THREADS;
  T wo[NO];
#pragma unroll
  for (int j = 0; j < NO; ++j) {
    const int i = threadIdx.x + j * S::THREADS, o = i / kW;
    wo[j] = (i < 16 * kW && o < n_out) ? Wo[i] : from_f32<T>(0.f);
  }
#pragma unroll
  for (int j = 0; j < NO; ++j) {
    const int i = threadIdx.x + j * S::THREADS, o = i / kW, c = i % kW;
    if (i < 16 * kW) {
      *cm<T>(sm + S::WO, o, c, kW) = wo[j];
      *cm<T>(sm + S::WOT, c, o, 16) = wo[j];
    }
  }
}

template <typename T, int N_IN, int NH, int MODE, int NT>
__global__ void __launch_bounds__(Tc3<N_IN, NH>::THREADS, 1)
mlp_train_tc3_kernel(const T* __restrict__ W, const T* __restrict__ in, int64_t P, int n_out,
                     const float* __restrict__ dout, const float* __restrict__ target, float loss_scale,
                     float inv_count, float* __restrict__ din, int din_group, float* __restrict__ ws,
                     int64_t n_params, int* __restrict__ err, float* __restrict__ yout, T* __restrict__ act) {
  using S = Tc3<N_IN, NH>;
  constexpr int G = S::G;
  constexpr bool BF16 = std::is_same<T, __nv_bfloat16>::value;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2 * G];   // per group: products of the chain, dW_0
  __shared__ uint32_t tmem_base;
  __shared__ float sq_part[4 * G];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 2, q = warp & 3, bar_id = 1 + g;
  const bool issuer = (tid & 127) == 0;
  const int r = q * 32 + lane;                          // this thread's tile row / TMEM lane
  const int gq = lane >> 2, t4 = lane & 3;              // mma.sync fragment coordinates
  const int lrow = (lane & 7) + 8 * ((lane >> 3) & 1), lcol = 8 * (lane >> 4);   // ldmatrix/stmatrix rows
  const int64_t n_tiles = (P + kM - 1) / kM;
  const float inv_scale = 1.f / loss_scale;
  unsigned char* gs = sm + g * S::GROUP;                // this group's buffers

  // the tile's inputs are loaded into registers one tile ahead, each thread its own row
  constexpr int kPieces = N_IN / 8;
  uint4 pf[kPieces];
  auto prefetch = [&](int64_t t) {
#pragma unroll
    for (int j = 0; j < kPieces; ++j) {                 // row r, columns 8 j .. 8 j + 7
      const int64_t row = t * kM + r;
      pf[j] = (t < n_tiles && row < P) ? __ldg(reinterpret_cast<const uint4*>(in + row * N_IN + 8 * j))
                                       : make_uint4(0, 0, 0, 0);
    }
  };
  const int64_t stride = (int64_t)G * gridDim.x;
  // tiles: CTA b takes b, b + grid, b + 2 grid, ... (so that the CTAs' counts differ by at most one)
  // and its group g every G-th of them, from b + g grid on
  const int64_t first = (int64_t)blockIdx.x + (int64_t)g * gridDim.x;
  prefetch(first);                                      // the first tile's loads overlap the set-up
  load_weights_tc3<T, N_IN, NH, S>(W, n_out, sm);
  // NT = 1 (n_out <= 8): the output layer's weights as mma.sync B fragments in registers, by for
  // Y = H W_out^T (n = output gq, k = hidden) and bd for dH = dY W_out (k = output, n = hidden).
  // NT = 2 (n_out <= 16): the same fragments read from the W_out tiles with ldmatrix when needed.
  const T* Wo = W + kW * N_IN + (NH - 1) * kW * kW;
  uint32_t by[NT == 1 ? 4 : 1][2], bd[NT == 1 ? 8 : 1];
  if constexpr (NT == 1) {
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int k = 16 * ks + 2 * t4, base = gq * kW;
      by[ks][0] = wpair<T>(Wo, base + k, base + k + 1, gq < n_out, gq < n_out);
      by[ks][1] = wpair<T>(Wo, base + k + 8, base + k + 9, gq < n_out, gq < n_out);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = 8 * nt + gq;
      bd[nt] = wpair<T>(Wo, (2 * t4) * kW + c, (2 * t4 + 1) * kW + c, 2 * t4 < n_out, 2 * t4 + 1 < n_out);
    }
  }
  // lane offsets of the ldmatrix / stmatrix addresses (the per-call parts are constants):
  //   lm_h: [128][64] tile, rows 32 q + lrow, columns lcol   (+ 2048 mt + 256 ks)
  //   lm_y: [128][16] tile, rows 32 q + lrow, columns lcol   (+ 512 mt)
  //   lm_wo: W_out [16][64] as B fragments of Y = H W_out^T (+ 256 ks)
  //   lm_wot: W_out^T [64][16] as B fragments of dH = dY W_out (+ 512 p: hidden columns 16 p ..)
  const uint32_t lm_h = (uint32_t)tc::cm_offset(32 * q + lrow, lcol, kW);
  const uint32_t lm_y = (uint32_t)tc::cm_offset(32 * q + lrow, lcol, 16);
  const int brow8 = (lane & 7) + 8 * (lane >> 4), bcol8 = 8 * ((lane >> 3) & 1);
  const uint32_t lm_wo = tc::smem_u32(sm + S::WO) + (uint32_t)tc::cm_offset(brow8, bcol8, kW);
  const uint32_t lm_wot = tc::smem_u32(sm + S::WOT) + (uint32_t)tc::cm_offset(brow8, bcol8, 16);
  if (tid == 0)
    for (int i = 0; i < 2 * G; ++i) tc::mbar_init(&mbar[i], 1);
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base + (uint32_t)(g * S::COLS);
  const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
  const uint32_t c_first = tmem + 64u + 64u * (NH - 1);     // dW_0; dW_h at 64 + 64 (h - 1)
  uint32_t phase = 0, phase_w = 0;
  bool failed = false, any_tile = false, w_pending = false;
  float dwo[2][4];                                      // dW_out tiles (m = outputs, n = q + 4 j)
#pragma unroll
  for (int j = 0; j < 2; ++j) dwo[j][0] = dwo[j][1] = dwo[j][2] = dwo[j][3] = 0.f;
  float sq = 0.f;

  auto issue_then = [&](auto&& body) {
    tc::fence_smem_async();
    tc::fence_before_sync();
    group_sync(bar_id);
    if (issuer) {
      tc::fence_after_sync();
      body();
      tc::commit(&mbar[g]);
    }
  };
  auto wait = [&]() -> bool {
    const bool ok = tc::mbar_wait_sleep(&mbar[g], phase, kSleepNs, kLimitNs, kSleepPolls);
    phase ^= 1u;
    tc::fence_after_sync();
    return !group_any(bar_id, !ok);
  };
  // the first-layer weight gradient of the previous tile (it reads X and dH_0)
  auto wait_w = [&]() -> bool {
    if (!w_pending) return true;
    w_pending = false;
    const bool ok = tc::mbar_wait_sleep(&mbar[G + g], phase_w, kSleepNs, kLimitNs, kSleepPolls);
    phase_w ^= 1u;
    tc::fence_after_sync();
    return !group_any(bar_id, !ok);
  };
  // M = 64 weight-gradient product over the tile's 128 points (8 MMAs of K = 16) from MN-major
  // views of two [points][features] core-matrix tiles (kA / kB bytes per 8 points); the descriptors
  // of consecutive K steps differ only in their start-address field (bytes / 16)
  auto wgrad = [&](uint32_t d, const unsigned char* A, uint32_t kA, const unsigned char* B, uint32_t kB, int N,
                   bool first) {
    const uint64_t da = tc::smem_desc(tc::smem_u32(A), kA, 128u), db = tc::smem_desc(tc::smem_u32(B), kB, 128u);
    const uint32_t id = tc::idesc_f16_mn(64, N, BF16);
#pragma unroll
    for (int ks = 0; ks < kM / 16; ++ks)
      tc::mma_f16(d, da + (uint64_t)(ks * 2 * kA / 16), db + (uint64_t)(ks * 2 * kB / 16), id, !(first && ks == 0));
  };
  // D = A B^T over K (multiple of 16) from two K-major core-matrix tiles (A: [128][K], B: [N][K])
  auto gemm = [&](const unsigned char* A, const unsigned char* B, int K, int N) {
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    const uint64_t da = tc::smem_desc(tc::smem_u32(A), 128u, sbo), db = tc::smem_desc(tc::smem_u32(B), 128u, sbo);
    const uint32_t id = tc::idesc_f16(kM, N, BF16);
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) tc::mma_f16(tmem, da + (uint64_t)(ks * 16), db + (uint64_t)(ks * 16), id, ks > 0);
  };
  // dW_out += dY^T H_last over the tile's points on mma.sync (warp q: hidden columns 8 q.., 8 (q + 4)..)
  auto dwout = [&]() {
    const int lo = lane >> 3, rr = lane & 7;
    const int arow = (lo >> 1) * 8 + rr, acol = (lo & 1) * 8, brow = (lo & 1) * 8 + rr;
    const uint32_t dl = tc::smem_u32(gs + S::DY) + (uint32_t)tc::cm_offset(arow, acol, 16);
    const uint32_t il = tc::smem_u32(gs + S::H + (NH - 1) * kM * kW * 2) + (uint32_t)tc::cm_offset(brow, 8 * q, kW);
#pragma unroll
    for (int ks = 0; ks < kM / 16; ++ks) {
      uint32_t a[4];
      ldsm_x4_trans(a, dl + 512u * ks);                 // points 16 ks .., outputs 0-15
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        uint32_t b0, b1;
        ldsm_x2_trans(b0, b1, il + 2048u * ks + 512u * j);   // hidden columns 8 (q + 4 j) ..
        mma16816<T>(dwo[j], a, b0, b1);
      }
    }
  };

  for (int64_t tile = first; tile < n_tiles; tile += stride) {
    const int64_t row0 = tile * kM;
    if (!wait_w()) { failed = true; break; }
#pragma unroll
    for (int j = 0; j < kPieces; ++j) *reinterpret_cast<uint4*>(gs + S::X + tc::cm_offset(r, 8 * j, N_IN)) = pf[j];
    prefetch(tile + stride);
    // targets (or upstream gradients) at this thread's output-fragment positions: rows
    // 32 q + 16 mt + gq (+ 8), outputs 2 t4 (+ 1)
    const int rows = (int)(P - row0 < kM ? P - row0 : kM);   // rows of this tile inside the batch
    float yin[2][NT][4];                                // [m-tile][output tile][fragment element]
    if constexpr (MODE == 2) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) yin[mt][nt][0] = yin[mt][nt][1] = yin[mt][nt][2] = yin[mt][nt][3] = 0.f;
    } else {
      const float* src = (MODE == 0 ? dout : target) + row0 * n_out;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int rl = 32 * q + 16 * mt + gq + 8 * (e >> 1), o = 8 * nt + 2 * t4 + (e & 1);
            yin[mt][nt][e] = (rl < rows && o < n_out) ? __ldg(src + rl * n_out + o) : 0.f;
          }
    }
    // ---- forward
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      unsigned char* Hh = gs + S::H + h * kM * kW * 2;
      issue_then([&] {
        if (h == 0) gemm(gs + S::X, sm + S::W0, N_IN, kW);
        else gemm(gs + S::H + (h - 1) * kM * kW * 2, sm + S::WH + (h - 1) * kW * kW * 2, kW, kW);
      });
      if (!wait()) { failed = true; break; }
      {
        float v[64];
        tc::tmem_ld64(lane_addr, v);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          uint4 u;
          u.x = pack2_relu<T>(v[8 * k + 0], v[8 * k + 1]);
          u.y = pack2_relu<T>(v[8 * k + 2], v[8 * k + 3]);
          u.z = pack2_relu<T>(v[8 * k + 4], v[8 * k + 5]);
          u.w = pack2_relu<T>(v[8 * k + 6], v[8 * k + 7]);
          *reinterpret_cast<uint4*>(Hh + tc::cm_offset(r, 8 * k, kW)) = u;
          if constexpr (MODE == 2)                      // the forward's hidden activations, if asked
            if (act && r < rows) *reinterpret_cast<uint4*>(act + ((int64_t)h * P + row0 + r) * kW + 8 * k) = u;
        }
      }
      if (h < NH - 1) continue;
      // ---- output layer, loss and dH_last on this warp's 32 rows (mma.sync)
      __syncwarp();
      const uint32_t sHh = tc::smem_u32(Hh) + lm_h;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        uint32_t ha[4][4];                              // A fragments of H_last, rows 32 q + 16 mt ..
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) ldsm_x4(ha[ks], sHh + 2048u * mt + 256u * ks);
        float y[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) y[nt][0] = y[nt][1] = y[nt][2] = y[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          if constexpr (NT == 1) {
            mma16816<T>(y[0], ha[ks], by[ks][0], by[ks][1]);
          } else {
            uint32_t b[4];                              // outputs 0-7 (b[0], b[1]) and 8-15 (b[2], b[3])
            ldsm_x4(b, lm_wo + 256u * ks);
            mma16816<T>(y[0], ha[ks], b[0], b[1]);
            mma16816<T>(y[NT - 1], ha[ks], b[2], b[3]);
          }
        }
        if constexpr (MODE == 2) {                      // forward only: the outputs, then the next m-tile
#pragma unroll
          for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int rl = 32 * q + 16 * mt + gq + 8 * (e >> 1), o = 8 * nt + 2 * t4 + (e & 1);
              if (rl < rows && o < n_out) yout[(row0 + rl) * n_out + o] = y[nt][e];
            }
          continue;
        }
        float dy[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const bool valid = 32 * q + 16 * mt + gq + 8 * (e >> 1) < rows && 8 * nt + 2 * t4 + (e & 1) < n_out;
            if (MODE == 0) {
              dy[nt][e] = valid ? yin[mt][nt][e] * loss_scale : 0.f;
            } else {
              const float res = y[nt][e] - yin[mt][nt][e];
              if (valid) sq = fmaf(res, res, sq);
              dy[nt][e] = valid ? res * inv_count * loss_scale : 0.f;
            }
          }
        // dY as the A operand of dH = dY W_out (k = outputs 0-15) and into the DY tile
        uint32_t da[4] = {pack2<T>(dy[0][0], dy[0][1]), pack2<T>(dy[0][2], dy[0][3]), pack2<T>(dy[1][0], dy[1][1]),
                          pack2<T>(dy[1][2], dy[1][3])};
        stsm_x4(tc::smem_u32(gs + S::DY) + lm_y + 512u * mt, da[0], da[1], da[2], da[3]);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          uint32_t b[4];                                // hidden columns 16 ks .. + 7 (b[0], b[1]), + 8 .. (b[2], b[3])
          if constexpr (NT == 1) {
            b[0] = bd[2 * ks];
            b[2] = bd[2 * ks + 1];
            b[1] = b[3] = 0u;                           // outputs 8-15
          } else {
            ldsm_x4(b, lm_wot + 512u * ks);
          }
          uint32_t u[4];
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma16816<T>(c, da, b[2 * j], b[2 * j + 1]);
            u[2 * j] = keep_where_positive<T>(pack2<T>(c[0], c[1]), ha[ks][2 * j]);
            u[2 * j + 1] = keep_where_positive<T>(pack2<T>(c[2], c[3]), ha[ks][2 * j + 1]);
          }
          stsm_x4(tc::smem_u32(gs + S::DH) + lm_h + 2048u * mt + 256u * ks, u[0], u[1], u[2], u[3]);
        }
      }
    }
    if (failed) break;
    if constexpr (MODE == 2) continue;                  // forward only
    // ---- backward through the hidden layers: dH_{h-1} = (dH_h W_h) * [H_{h-1} > 0].  The chain
    // product is committed alone and dW_h += dH_h^T H_{h-1} is issued after it (the next commit
    // covers it), so the epilogue does not wait for the weight gradient; dH_{h-1} goes into H_h's
    // buffer, whose readers have all completed (dW_{h+1} before this commit, dW_out on the warps).
    constexpr uint32_t kH = (kW / 8) * 128, kX = (N_IN / 8) * 128;
#pragma unroll
    for (int h = NH - 1; h >= 1; --h) {
      const unsigned char* A = h == NH - 1 ? gs + S::DH : gs + S::H + (h + 1) * kM * kW * 2;   // dH_h
      const unsigned char* Hp = gs + S::H + (h - 1) * kM * kW * 2;                             // H_{h-1}
      unsigned char* out = gs + S::H + h * kM * kW * 2;                                        // dH_{h-1}
      tc::fence_smem_async();
      tc::fence_before_sync();
      group_sync(bar_id);
      if (issuer) {
        tc::fence_after_sync();
        gemm(A, sm + S::WHT + (h - 1) * kW * kW * 2, kW, kW);
        tc::commit(&mbar[g]);
        wgrad(tmem + 64u + 64u * (h - 1), A, kH, Hp, kH, kW, !any_tile);
      }
      if (h == NH - 1) dwout();
      if (!wait()) { failed = true; break; }
      {
        float v[64];
        tc::tmem_ld64(lane_addr, v);
        const int c0 = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint4 hv = *reinterpret_cast<const uint4*>(Hp + tc::cm_offset(r, c0 + 8 * k, kW));
          uint4 u;
          u.x = keep_where_positive<T>(pack2<T>(v[8 * k + 0], v[8 * k + 1]), hv.x);
          u.y = keep_where_positive<T>(pack2<T>(v[8 * k + 2], v[8 * k + 3]), hv.y);
          u.z = keep_where_positive<T>(pack2<T>(v[8 * k + 4], v[8 * k + 5]), hv.z);
          u.w = keep_where_positive<T>(pack2<T>(v[8 * k + 6], v[8 * k + 7]), hv.w);
          *reinterpret_cast<uint4*>(out + tc::cm_offset(r, c0 + 8 * k, kW)) = u;
        }
      }
    }
    if (failed) break;
    // ---- dX = dH_0 W_0, committed alone; dW_0 += dH_0^T X after it with its own commit, waited
    // for before the next tile overwrites X (or, where the input-gradient staging needs dH_0's
    // buffer, before the epilogue)
    {
      const unsigned char* dH0 = NH == 1 ? gs + S::DH : gs + S::H + kM * kW * 2;
      tc::fence_smem_async();
      tc::fence_before_sync();
      group_sync(bar_id);
      if (issuer) {
        tc::fence_after_sync();
        gemm(dH0, sm + S::W0T, kW, N_IN);
        tc::commit(&mbar[g]);
        wgrad(c_first, dH0, kH, gs + S::X, kX, N_IN, !any_tile);
        tc::commit(&mbar[G + g]);
      }
      w_pending = true;
      if (NH == 1) dwout();
      any_tile = true;
      if (!wait()) { failed = true; break; }
      if (!S::EARLY && !wait_w()) { failed = true; break; }
    }
    // ---- input gradient (row-major output staged in the group's activation buffers, then
    // written as contiguous 16-byte pieces of the tile)
    if (din && din_group == 0) {
      // row r's 16-byte chunk c at chunk r * N_IN / 4 + (c ^ (r & SWZ)), SWZ + 1 = min(8, chunks per
      // row): the rows of eight lanes land in different bank groups (two-way for N_IN = 16)
      constexpr int SWZ = (N_IN / 4 < 8 ? N_IN / 4 : 8) - 1;
      float* st = reinterpret_cast<float*>(gs + S::H);
      float v[N_IN];
      tc::tmem_ld_cols<N_IN>(lane_addr, v);
#pragma unroll
      for (int j = 0; j < N_IN; j += 4)
        *reinterpret_cast<float4*>(st + (r * (N_IN / 4) + ((j >> 2) ^ (r & SWZ))) * 4) =
            make_float4(v[j] * inv_scale, v[j + 1] * inv_scale, v[j + 2] * inv_scale, v[j + 3] * inv_scale);
      group_sync(bar_id);
#pragma unroll
      for (int j = 0; j < N_IN / 4; ++j) {
        const int i = r + 128 * j, rr = i / (N_IN / 4), c4 = i % (N_IN / 4);
        if (rr < rows)
          *reinterpret_cast<float4*>(din + row0 * N_IN + rr * N_IN + c4 * 4) =
              *reinterpret_cast<const float4*>(st + (rr * (N_IN / 4) + (c4 ^ (rr & SWZ))) * 4);
      }
    } else {
      const int64_t row = row0 + r;
#pragma unroll
      for (int c0 = 0; c0 < N_IN; c0 += 16) {
        float v[16];
        tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
        if (din && row < P) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int col = c0 + j;
            const float2 val = make_float2(v[j] * inv_scale, v[j + 1] * inv_scale);
            if (din_group == 1) {
              din[(int64_t)col * P + row] = val.x;
              din[(int64_t)(col + 1) * P + row] = val.y;
            } else {
              *reinterpret_cast<float2*>(din + ((int64_t)(col / din_group) * P + row) * din_group + col % din_group) =
                  val;
            }
          }
        }
      }
    }
    // the next tile's first product is issued after a group barrier (issue_then), which orders
    // these reads of the staging buffers and of the accumulator before anything overwrites them
  }

  // ---- partials: each group's accumulators into its own shared row, then their sum in group
  // order as this CTA's row (every group reaches this point; a failed group left its loop whole)
  // the reduction of the CTAs' partial rows may be scheduled from here on (it waits for this grid)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (!failed && !wait_w()) failed = true;
  if (failed && (tid & 127) == 0 && err) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if constexpr (MODE == 2) {                            // no weight gradients
    if (warp == 0) tc::tmem_dealloc(tmem_base, 512);
    return;
  }
  // this group's partial in shared memory, rows padded (dW_h rows of 68 floats, dW_0 rows of
  // N_IN + 4) so that the accumulator rows of eight lanes land in eight different bank groups
  float* part = reinterpret_cast<float*>(sm) + g * S::PSTRIDE;
  {
    const int m = 16 * q + lane;                        // row of an M = 64 accumulator (lanes < 16)
    const uint32_t la = (uint32_t)(q * 32) << 16;
    float v[16];
#pragma unroll
    for (int h = 1; h < NH; ++h)
#pragma unroll
      for (int c0 = 0; c0 < kW; c0 += 16) {
        tc::tmem_ld16(tmem + 64u + 64u * (h - 1) + la + (uint32_t)c0, v);
        if (lane < 16)
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(part + S::PH + (h - 1) * kW * (kW + 4) + m * (kW + 4) + c0 + j) =
                any_tile ? make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
    for (int c0 = 0; c0 < N_IN; c0 += 16) {
      tc::tmem_ld16(c_first + la + (uint32_t)c0, v);
      if (lane < 16)
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(part + S::P0 + m * (N_IN + 4) + c0 + j) =
              any_tile ? make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int mo = gq + (e >> 1) * 8, n = (q + 4 * j) * 8 + 2 * t4 + (e & 1);
        if (mo < n_out) part[S::PO + mo * kW + n] = dwo[j][e];
      }
  }
  if (MODE == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) sq_part[warp] = sq;
  }
  tc::fence_before_sync();
  __syncthreads();
  // the CTA's row: the groups' partials summed in group order, in the parameter order
  // [W_0 | W_1 .. W_{NH-1} | W_out]
  float* row = ws + (int64_t)blockIdx.x * n_params;
  const float* p0 = reinterpret_cast<const float*>(sm);
  const int n_first = kW * N_IN, n_hid = (NH - 1) * kW * kW;
  for (int i = tid; i < (int)n_params; i += blockDim.x) {
    int at;
    if (i < n_first) {
      at = S::P0 + (i / N_IN) * (N_IN + 4) + i % N_IN;
    } else if (i < n_first + n_hid) {
      const int j = i - n_first;
      at = S::PH + (j / (kW * kW)) * kW * (kW + 4) + ((j / kW) % kW) * (kW + 4) + j % kW;
    } else {
      at = S::PO + (i - n_first - n_hid);
    }
    float sum = 0.f;
#pragma unroll
    for (int gg = 0; gg < G; ++gg) sum += p0[gg * S::PSTRIDE + at];
    row[i] = sum;
  }
  if (MODE == 1 && tid == 0) {
    float sum = 0.f;
    for (int w = 0; w < 4 * G; ++w) sum += sq_part[w];
    ws[(int64_t)gridDim.x * n_params + blockIdx.x] = sum;
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, 512);
  }
}

template <typename T, int N_IN, int NH, int NT>
sxe_status tc3_launch(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                      float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid,
                      cudaStream_t s, int64_t lc) {
  using S = Tc3<N_IN, NH>;
  const int64_t n_params = sxe_mlp_n_params(d);
  const int64_t n_tiles = (P + kM - 1) / kM;
  const int g3 = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)device_sm_count(), (int64_t)grid, (n_tiles + S::G - 1) / S::G}));
  const float ic = l2_inv_count(lc, d->n_out);
  int* err = tc3_error_word();
  if (target) {
    kernel_ctas_per_sm((const void*)mlp_train_tc3_kernel<T, N_IN, NH, 1, NT>, S::THREADS, S::SMEM);
    mlp_train_tc3_kernel<T, N_IN, NH, 1, NT><<<g3, S::THREADS, S::SMEM, s>>>(
        (const T*)W, (const T*)in, P, d->n_out, dout, target, ls, ic, din, dg, ws, n_params, err, nullptr,
        nullptr);
  } else {
    kernel_ctas_per_sm((const void*)mlp_train_tc3_kernel<T, N_IN, NH, 0, NT>, S::THREADS, S::SMEM);
    mlp_train_tc3_kernel<T, N_IN, NH, 0, NT><<<g3, S::THREADS, S::SMEM, s>>>(
        (const T*)W, (const T*)in, P, d->n_out, dout, target, ls, ic, din, dg, ws, n_params, err, nullptr,
        nullptr);
  }
  sxe_status st = check_launch("mlp_train_tc3");
  if (st != SXE_OK) return st;
  return launch_mlp_reduce(ws, g3, n_params, 1.f / ls, dW, target ? sq : nullptr, s);
}

// Forward only (MODE 2): the network's outputs out [P][n_out] binary32 and, if act is given, the
// hidden activations act [NH][P][64]; the same grid and plan as the training pass.
template <typename T, int N_IN, int NH, int NT>
sxe_status tc3_fwd_launch(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out, void* act,
                          cudaStream_t s) {
  using S = Tc3<N_IN, NH>;
  const int64_t n_tiles = (P + kM - 1) / kM;
  const int g3 = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)device_sm_count(), (n_tiles + S::G - 1) / S::G));
  kernel_ctas_per_sm((const void*)mlp_train_tc3_kernel<T, N_IN, NH, 2, NT>, S::THREADS, S::SMEM);
  mlp_train_tc3_kernel<T, N_IN, NH, 2, NT><<<g3, S::THREADS, S::SMEM, s>>>(
      (const T*)W, (const T*)in, P, d->n_out, nullptr, nullptr, 1.f, 0.f, nullptr, 0, nullptr, 0, tc3_error_word(),
      out, (T*)act);
  return check_launch("mlp_fwd_tc3");
}

template <typename T, int NT>
sxe_status tc3_fwd_in(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out, void* act,
                      cudaStream_t s) {
  switch (d->n_in * 4 + d->n_hidden) {
    case 16 * 4 + 1: return tc3_fwd_launch<T, 16, 1, NT>(d, W, in, P, out, act, s);
    case 16 * 4 + 2: return tc3_fwd_launch<T, 16, 2, NT>(d, W, in, P, out, act, s);
    case 16 * 4 + 3: return tc3_fwd_launch<T, 16, 3, NT>(d, W, in, P, out, act, s);
    case 32 * 4 + 1: return tc3_fwd_launch<T, 32, 1, NT>(d, W, in, P, out, act, s);
    case 32 * 4 + 2: return tc3_fwd_launch<T, 32, 2, NT>(d, W, in, P, out, act, s);
    case 32 * 4 + 3: return tc3_fwd_launch<T, 32, 3, NT>(d, W, in, P, out, act, s);
    case 64 * 4 + 1: return tc3_fwd_launch<T, 64, 1, NT>(d, W, in, P, out, act, s);
    case 64 * 4 + 2: return tc3_fwd_launch<T, 64, 2, NT>(d, W, in, P, out, act, s);
    default: return tc3_fwd_launch<T, 64, 3, NT>(d, W, in, P, out, act, s);
  }
}

template <typename T, int N_IN, int NT>
sxe_status tc3_nh(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                  float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid, cudaStream_t s,
                  int64_t lc) {
  switch (d->n_hidden) {
    case 1: return tc3_launch<T, N_IN, 1, NT>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    case 2: return tc3_launch<T, N_IN, 2, NT>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    default: return tc3_launch<T, N_IN, 3, NT>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
  }
}

template <typename T, int NT>
sxe_status tc3_in(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                  float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid, cudaStream_t s,
                  int64_t lc) {
  switch (d->n_in) {
    case 16: return tc3_nh<T, 16, NT>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    case 32: return tc3_nh<T, 32, NT>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    default: return tc3_nh<T, 64, NT>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
  }
}

}  // namespace
}  // namespace sxe
