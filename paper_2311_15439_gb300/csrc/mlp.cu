// Tiny fully connected ReLU network on the tensor cores (Sec. 5 d-e, Sec. 6.1 of
// arXiv 2311.15439: the encoding feeds a ~7k-weight network; the loss gradient flows
// back through it into the encoding).
//
// Shapes: n_in -> NH hidden layers of 64 ReLU units -> n_out (<= 16) linear outputs,
// no biases.  One CTA = 8 warps works on tiles of 128 points (16 per warp); the whole
// network lives in shared memory, activations stay in registers between layers (the
// C fragment of one m16n8k16 product is the A fragment of the next).
//
// The backward kernel recomputes the forward pass of its tile (cheaper than writing
// and re-reading activations), stages inputs, activations and deltas of the tile in
// shared memory and accumulates the weight gradients dW_l = Delta_l^T In_l for the
// whole persistent loop in registers; per-CTA partials go to a workspace and a second
// kernel sums them in a fixed order (deterministic).
#include <algorithm>
#include <type_traits>

#include "sxe_internal.cuh"

namespace sxe {
namespace {

constexpr int kWidth = 64;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kTile = kWarps * 16;   // points per tile
constexpr int kSW = kWidth + 8;      // padded row stride (halves) of 64-wide tiles
constexpr int kSO = 16 + 8;          // padded row stride of 16-wide tiles

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
  if constexpr (sizeof(T) == 2 && std::is_same<T, __half>::value) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

__device__ __forceinline__ uint32_t lds32(const void* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ void sts32(void* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t& r0, uint32_t& r1, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

// B fragments (k16 x n8) of n-tiles nt and nt+1 of a row-major [n][k] shared array (row stride
// ld halves, rows 16-byte aligned) with one ldmatrix: r = {b0, b1} of nt, then of nt+1.
template <typename T>
__device__ __forceinline__ void bfrag_pair(const T* W, int ld, int nt, int kk, int lane, uint32_t (&r)[4]) {
  const int m = lane >> 3;
  ldsm_x4(r, W + ((nt + (m >> 1)) * 8 + (lane & 7)) * ld + kk * 16 + (m & 1) * 8);
}

// B fragment (k16 x n8) of a row-major [n][k] shared array with row stride `ld` (halves).
template <typename T>
__device__ __forceinline__ void bfrag(const T* W, int ld, int nt, int kk, int g, int t, uint32_t& b0, uint32_t& b1) {
  const T* row = W + (nt * 8 + g) * ld + kk * 16 + 2 * t;
  b0 = lds32(row);
  b1 = lds32(row + 8);
}

// Shared-memory plan of one CTA (offsets in halves).
template <int N_IN, int NH>
struct Smem {
  static constexpr int SX = N_IN + 8;
  static constexpr int W0 = 0;                                  // [64][SX]      W_0
  static constexpr int WH = W0 + kWidth * SX;                   // (NH-1) x [64][kSW]  W_h
  static constexpr int WO = WH + (NH - 1) * kWidth * kSW;       // [16][kSW]     W_out (zero padded)
  static constexpr int X = WO + 16 * kSW;                       // [128][SX]     inputs of the tile
  static constexpr int A = X + kTile * SX;                      // NH x [128][kSW] hidden activations
  static constexpr int D = A + NH * kTile * kSW;                // NH x [128][kSW] hidden deltas
  static constexpr int DY = D + NH * kTile * kSW;               // [128][kSO]    output delta
  static constexpr int FWD_END = A;                             // forward-only kernels stop here
  static constexpr int END = DY + kTile * kSO;
  // training kernel: an unpadded [128][N_IN] staging buffer that cp.async fills with the next
  // tile's inputs while the current tile computes, where two CTAs per SM still fit with it
  static constexpr int XS = END;
  static constexpr bool PF = (END + kTile * N_IN) * 2 <= 113 * 1024;
  static constexpr int BWD_END = END + (PF ? kTile * N_IN : 0);
  // weight-gradient tiles: output layer 1x8, hidden 4x8 each, first layer 4x(N_IN/8)
  static constexpr int N_WTILES = 8 + (NH - 1) * 32 + 4 * (N_IN / 8);
  static constexpr int TILES_PER_WARP = (N_WTILES + kWarps - 1) / kWarps;
};

// Load W (global, [fan_out][fan_in] back to back) into padded row-major shared copies.
// The forward pass reads B fragments from them directly (k contiguous); the backward
// pass needs the transposed operand and reads it with ldmatrix.trans.
template <typename T, int N_IN, int NH>
__device__ void load_weights(const T* __restrict__ W, int n_out, T* sm) {
  using S = Smem<N_IN, NH>;
  const T zero = from_f32<T>(0.f);
  for (int i = threadIdx.x; i < kWidth * N_IN; i += blockDim.x) sm[S::W0 + (i / N_IN) * S::SX + i % N_IN] = W[i];
  const T* Wh = W + kWidth * N_IN;
  for (int i = threadIdx.x; i < (NH - 1) * kWidth * kWidth; i += blockDim.x) {
    const int h = i / (kWidth * kWidth), r = (i / kWidth) % kWidth, c = i % kWidth;
    sm[S::WH + h * kWidth * kSW + r * kSW + c] = Wh[i];
  }
  const T* Wo = Wh + (NH - 1) * kWidth * kWidth;
  for (int i = threadIdx.x; i < 16 * kWidth; i += blockDim.x) {
    const int r = i / kWidth, c = i % kWidth;
    sm[S::WO + r * kSW + c] = r < n_out ? Wo[r * kWidth + c] : zero;
  }
}

// B fragments of n-tiles nt and nt+1 of a row-major [k][n] shared array with one ldmatrix.trans:
// r = {b0, b1} of nt, then of nt+1 (lanes 16..31 address the second pair).
__device__ __forceinline__ void bfrag_kn_pair(const void* base, int ld_halves, int kk, int nt, int lane,
                                              uint32_t (&r)[4]) {
  const int q = lane >> 3, rr = lane & 7;
  ldsm_x4_trans(r, reinterpret_cast<const __half*>(base) + (kk * 16 + (q & 1) * 8 + rr) * ld_halves +
                       (nt + (q >> 1)) * 8);
}

// Stage the tile's inputs [128][N_IN] into shared memory (zero rows past P).
template <typename T, int N_IN, int NH>
__device__ __forceinline__ void load_inputs(const T* __restrict__ in, int64_t row0, int64_t P, T* sm) {
  using S = Smem<N_IN, NH>;
  constexpr int VPR = N_IN * 2 / 16;  // 16-byte vectors per row
  for (int i = threadIdx.x; i < kTile * VPR; i += blockDim.x) {
    const int r = i / VPR, c = i % VPR;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (row0 + r < P) v = __ldg(reinterpret_cast<const uint4*>(in + (row0 + r) * N_IN) + c);
    *reinterpret_cast<uint4*>(sm + S::X + r * S::SX + c * 8) = v;
  }
}

// Forward pass of the warp's 16 rows.  Writes hidden activations to sm (if `keep`)
// and returns the 16 output columns as two C fragments.
template <typename T, int N_IN, int NH>
__device__ __forceinline__ void forward_rows(T* sm, int r0, int g, int t, bool keep, float (&y)[2][4],
                                             uint32_t (&hfr)[NH][4][4]) {
  using S = Smem<N_IN, NH>;
  uint32_t afr[4][4];
  const int lane = g * 4 + t;
  // input fragments (one ldmatrix per 16 x 16 block)
#pragma unroll
  for (int kk = 0; kk < N_IN / 16; ++kk) {
    const int m = lane >> 3;
    ldsm_x4(afr[kk], sm + S::X + (r0 + (m & 1) * 8 + (lane & 7)) * S::SX + kk * 16 + (m >> 1) * 8);
  }
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    const T* Wl = h == 0 ? sm + S::W0 : sm + S::WH + (h - 1) * kWidth * kSW;
    const int ld = h == 0 ? S::SX : kSW;
    const int nk = h == 0 ? N_IN / 16 : 4;
#pragma unroll
    for (int np = 0; np < 4; ++np) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        if (kk >= nk) break;
        uint32_t b[4];
        bfrag_pair<T>(Wl, ld, 2 * np, kk, lane, b);
        mma16816<T>(acc[2 * np], afr[kk], b[0], b[1]);
        mma16816<T>(acc[2 * np + 1], afr[kk], b[2], b[3]);
      }
    }
    // ReLU, round to the operand type; the rounded values are both the next layer's
    // input and what the backward pass sees.
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      afr[kk][0] = pack2<T>(fmaxf(acc[2 * kk][0], 0.f), fmaxf(acc[2 * kk][1], 0.f));
      afr[kk][1] = pack2<T>(fmaxf(acc[2 * kk][2], 0.f), fmaxf(acc[2 * kk][3], 0.f));
      afr[kk][2] = pack2<T>(fmaxf(acc[2 * kk + 1][0], 0.f), fmaxf(acc[2 * kk + 1][1], 0.f));
      afr[kk][3] = pack2<T>(fmaxf(acc[2 * kk + 1][2], 0.f), fmaxf(acc[2 * kk + 1][3], 0.f));
#pragma unroll
      for (int j = 0; j < 4; ++j) hfr[h][kk][j] = afr[kk][j];
      if (keep) {
        T* a = sm + S::A + h * kTile * kSW;
        sts32(a + (r0 + g) * kSW + kk * 16 + 2 * t, afr[kk][0]);
        sts32(a + (r0 + g + 8) * kSW + kk * 16 + 2 * t, afr[kk][1]);
        sts32(a + (r0 + g) * kSW + kk * 16 + 8 + 2 * t, afr[kk][2]);
        sts32(a + (r0 + g + 8) * kSW + kk * 16 + 8 + 2 * t, afr[kk][3]);
      }
    }
  }
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) y[nt][0] = y[nt][1] = y[nt][2] = y[nt][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    uint32_t b[4];
    bfrag_pair<T>(sm + S::WO, kSW, 0, kk, lane, b);
    mma16816<T>(y[0], afr[kk], b[0], b[1]);
    mma16816<T>(y[1], afr[kk], b[2], b[3]);
  }
}

template <typename T, int N_IN, int NH>
__global__ void __launch_bounds__(kThreads)
mlp_fwd_kernel(const T* __restrict__ W, const T* __restrict__ in, int64_t P, int n_out, float* __restrict__ out,
               T* __restrict__ act) {
  using S = Smem<N_IN, NH>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  load_weights<T, N_IN, NH>(W, n_out, sm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = warp * 16;
  const int64_t n_tiles = (P + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTile;
    __syncthreads();
    load_inputs<T, N_IN, NH>(in, row0, P, sm);
    __syncthreads();
    float y[2][4];
    uint32_t hfr[NH][4][4];
    forward_rows<T, N_IN, NH>(sm, r0, g, t, false, y, hfr);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t row = row0 + r0 + g + half * 8;
      if (row >= P) continue;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int o = nt * 8 + 2 * t + j;
          if (o < n_out) out[row * n_out + o] = y[nt][half * 2 + j];
        }
      if (act) {
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            T* a = act + ((int64_t)h * P + row) * kWidth + kk * 16 + 2 * t;
            sts32(a, hfr[h][kk][half]);
            sts32(a + 8, hfr[h][kk][2 + half]);
          }
      }
    }
  }
}

// Volumetric field of a tile of samples in one pass (Sec. 6.2): the density network, then
// sigma = exp(min(v_0, 15)) and the colour network's input row [v_0..v_15, SH(d)] written to
// shared memory by the warp that owns the rows, then the colour network.  The arithmetic is
// that of sxe_mlp_fwd, sxe_vr_field and sxe_mlp_fwd in sequence; nothing but sigma and the
// colour logits leaves the chip.
template <typename T, int N_IN, int NHC>
__global__ void __launch_bounds__(kThreads)
vr_field_mlp_kernel(const T* __restrict__ Wd, const T* __restrict__ Wc, const T* __restrict__ enc,
                    const float* __restrict__ dirs, int64_t P, int S, int n_out_c, float* __restrict__ sigma,
                    float* __restrict__ logits) {
  using SD = Smem<N_IN, 1>;
  using SC = Smem<32, NHC>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smd = reinterpret_cast<T*>(smem_raw);
  T* smc = smd + SD::FWD_END;
  load_weights<T, N_IN, 1>(Wd, 16, smd);
  load_weights<T, 32, NHC>(Wc, n_out_c, smc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = warp * 16;
  const int64_t n_tiles = (P + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTile;
    __syncthreads();
    load_inputs<T, N_IN, 1>(enc, row0, P, smd);
    __syncthreads();
    float y[2][4];
    uint32_t hfr[1][4][4];
    forward_rows<T, N_IN, 1>(smd, r0, g, t, false, y, hfr);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int rl = r0 + g + 8 * half;
      const int64_t row = row0 + rl;
      if (t == 0 && row < P) sigma[row] = vr_density(y[0][2 * half]);
      T* xr = smc + SC::X + rl * SC::SX;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) sts32(xr + nt * 8 + 2 * t, pack2<T>(y[nt][2 * half], y[nt][2 * half + 1]));
      const int64_t ray = (row < P ? row : P - 1) / S;
      float h[16];
      sh16(__ldg(dirs + ray * 3), __ldg(dirs + ray * 3 + 1), __ldg(dirs + ray * 3 + 2), h);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (t == q) {
          sts32(xr + 16 + 4 * q, pack2<T>(h[4 * q], h[4 * q + 1]));
          sts32(xr + 18 + 4 * q, pack2<T>(h[4 * q + 2], h[4 * q + 3]));
        }
    }
    __syncwarp();
    float y2[2][4];
    uint32_t hfr2[NHC][4][4];
    forward_rows<T, 32, NHC>(smc, r0, g, t, false, y2, hfr2);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t row = row0 + r0 + g + half * 8;
      if (row >= P) continue;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int o = nt * 8 + 2 * t + j;
          if (o < n_out_c) logits[row * n_out_c + o] = y2[nt][half * 2 + j];
        }
    }
  }
}

// MODE 0: dy = dout * loss_scale.  MODE 1: dy = loss_scale * 2 (y - target) / (P n_out),
// and the squared residuals are summed into *sq_sum.
// Two CTAs per SM where the shared-memory plan allows it (then at most 128 registers).
template <int N_IN, int NH>
struct BwdOcc { static constexpr int value = Smem<N_IN, NH>::BWD_END * 2 <= 113 * 1024 ? 2 : 1; };

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T, int N_IN, int NH, int MODE>
__global__ void __launch_bounds__(kThreads, BwdOcc<N_IN, NH>::value)
mlp_bwd_kernel(const T* __restrict__ W, const T* __restrict__ in, int64_t P, int n_out,
               const float* __restrict__ dout, const float* __restrict__ target, float loss_scale, float inv_count,
               float* __restrict__ din, float* __restrict__ ws, int64_t n_params, float* __restrict__ sq_sum,
               int din_group) {
  using S = Smem<N_IN, NH>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  load_weights<T, N_IN, NH>(W, n_out, sm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = warp * 16;
  const int64_t n_tiles = (P + kTile - 1) / kTile;
  float dw[S::TILES_PER_WARP][4];
#pragma unroll
  for (int i = 0; i < S::TILES_PER_WARP; ++i) dw[i][0] = dw[i][1] = dw[i][2] = dw[i][3] = 0.f;
  float sq = 0.f;
  // inputs one tile ahead: each thread cp.asyncs its own 16-byte pieces of the next tile into the
  // staging buffer and later moves exactly those pieces into the padded tile, so it waits only for
  // its own copies (rows past P are zero-filled)
  constexpr int VPR = N_IN * 2 / 16;
  constexpr int PIECES = kTile * VPR / kThreads;
  static_assert(!S::PF || (kTile * VPR) % kThreads == 0, "staging pieces per thread");
  auto stage = [&](int64_t tl) {
#pragma unroll
    for (int j = 0; j < PIECES; ++j) {
      const int i = threadIdx.x + j * kThreads, rr = i / VPR, c = i % VPR;
      const int64_t row = tl * kTile + rr;
      const bool valid = tl < n_tiles && row < P;
      cp_async16(sm + S::XS + rr * N_IN + c * 8, valid ? in + row * N_IN + c * 8 : in, valid);
    }
    cp_async_commit();
  };
  if constexpr (S::PF) stage(blockIdx.x);

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTile;
    __syncthreads();
    if constexpr (S::PF) {
      cp_async_wait_all();
#pragma unroll
      for (int j = 0; j < PIECES; ++j) {
        const int i = threadIdx.x + j * kThreads, rr = i / VPR, c = i % VPR;
        *reinterpret_cast<uint4*>(sm + S::X + rr * S::SX + c * 8) =
            *reinterpret_cast<const uint4*>(sm + S::XS + rr * N_IN + c * 8);
      }
      stage(tile + gridDim.x);
    } else {
      load_inputs<T, N_IN, NH>(in, row0, P, sm);
    }
    __syncthreads();
    float y[2][4];
    uint32_t hfr[NH][4][4];
    forward_rows<T, N_IN, NH>(sm, r0, g, t, true, y, hfr);
    // ---- output delta
    uint32_t afr[4][4];
    {
      float dy[2][4];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t row = row0 + r0 + g + (e >> 1) * 8;
          const int o = nt * 8 + 2 * t + (e & 1);
          float v = 0.f;
          if (row < P && o < n_out) {
            if (MODE == 0) {
              v = dout[row * n_out + o] * loss_scale;
            } else {
              const float r = y[nt][e] - target[row * n_out + o];
              sq = fmaf(r, r, sq);
              v = r * inv_count * loss_scale;
            }
          }
          dy[nt][e] = v;
        }
      afr[0][0] = pack2<T>(dy[0][0], dy[0][1]);
      afr[0][1] = pack2<T>(dy[0][2], dy[0][3]);
      afr[0][2] = pack2<T>(dy[1][0], dy[1][1]);
      afr[0][3] = pack2<T>(dy[1][2], dy[1][3]);
      T* d = sm + S::DY;
      sts32(d + (r0 + g) * kSO + 2 * t, afr[0][0]);
      sts32(d + (r0 + g + 8) * kSO + 2 * t, afr[0][1]);
      sts32(d + (r0 + g) * kSO + 8 + 2 * t, afr[0][2]);
      sts32(d + (r0 + g + 8) * kSO + 8 + 2 * t, afr[0][3]);
    }
    // ---- hidden deltas, top layer down: dH_h = (dH_{h+1} W_{h+1}) * [a_h > 0]
#pragma unroll
    for (int h = NH - 1; h >= 0; --h) {
      float acc[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
      for (int np = 0; np < 8; np += 2) {
        if (h == NH - 1) {          // dY W_out: B[k = o][n = j] = W_out[o][j]
          uint32_t b[4];
          bfrag_kn_pair(sm + S::WO, kSW, 0, np, lane, b);
          mma16816<T>(acc[np], afr[0], b[0], b[1]);
          mma16816<T>(acc[np + 1], afr[0], b[2], b[3]);
        } else {                    // dH_{h+1} W_{h+1}: B[k = j][n = j'] = W_{h+1}[j][j']
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            uint32_t b[4];
            bfrag_kn_pair(sm + S::WH + h * kWidth * kSW, kSW, kk, np, lane, b);
            mma16816<T>(acc[np], afr[kk], b[0], b[1]);
            mma16816<T>(acc[np + 1], afr[kk], b[2], b[3]);
          }
        }
      }
      // mask by the ReLU derivative and round to the operand type
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int nt = 2 * kk + (j >> 1);
          const float2 a = unpack2<T>(hfr[h][kk][j]);
          const float lo = a.x > 0.f ? acc[nt][(j & 1) * 2] : 0.f;
          const float hi = a.y > 0.f ? acc[nt][(j & 1) * 2 + 1] : 0.f;
          afr[kk][j] = pack2<T>(lo, hi);
        }
        T* d = sm + S::D + h * kTile * kSW;
        sts32(d + (r0 + g) * kSW + kk * 16 + 2 * t, afr[kk][0]);
        sts32(d + (r0 + g + 8) * kSW + kk * 16 + 2 * t, afr[kk][1]);
        sts32(d + (r0 + g) * kSW + kk * 16 + 8 + 2 * t, afr[kk][2]);
        sts32(d + (r0 + g + 8) * kSW + kk * 16 + 8 + 2 * t, afr[kk][3]);
      }
    }
    // ---- input gradient dX = dH_0 W_0
    if (din) {
      const float inv_scale = 1.f / loss_scale;
#pragma unroll
      for (int np = 0; np < N_IN / 8; np += 2) {
        float acc2[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {    // dH_0 W_0: B[k = j][n = i] = W_0[j][i]
          uint32_t b[4];
          bfrag_kn_pair(sm + S::W0, S::SX, kk, np, lane, b);
          mma16816<T>(acc2[0], afr[kk], b[0], b[1]);
          mma16816<T>(acc2[1], afr[kk], b[2], b[3]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int nt = np + (u >> 1), half = u & 1;
          const float* acc = acc2[u >> 1];
          const int64_t row = row0 + r0 + g + half * 8;
          if (row >= P) continue;
          const int c = nt * 8 + 2 * t;                 // columns c, c + 1
          const float2 v = make_float2(acc[half * 2] * inv_scale, acc[half * 2 + 1] * inv_scale);
          if (din_group == 0) {                          // [P][n_in]
            *reinterpret_cast<float2*>(din + row * N_IN + c) = v;
          } else if (din_group == 1) {                   // [n_in][P]
            din[(int64_t)c * P + row] = v.x;
            din[(int64_t)(c + 1) * P + row] = v.y;
          } else {                                       // [n_in / g][P][g], c and c + 1 in one group
            *reinterpret_cast<float2*>(din + ((int64_t)(c / din_group) * P + row) * din_group + c % din_group) = v;
          }
        }
      }
    }
    __syncthreads();
    // ---- weight gradients of the tile: dW_l += Delta_l^T In_l, K = 128 rows.  Warp w owns the
    // m16n8 tiles w, w + 8, w + 16, ... of the list [output layer 1x8, hidden h 4x8 each, first
    // layer 4x(N_IN/8)] (dw[i] = tile w + 8i).  Since N_IN/8 divides 8, all of a warp's tiles of
    // one hidden or first layer have the same input columns nt: their B fragment is loaded once
    // per k step and used by every m-tile.
    {
      const int q = lane >> 3, rr = lane & 7;
      const int arow = (q >> 1) * 8 + rr, acol = (q & 1) * 8, brow = (q & 1) * 8 + rr;
      {                                                   // output layer [16][64]: tile 0, nt = warp
        const T* Dl = sm + S::DY;
        const T* In = sm + S::A + (NH - 1) * kTile * kSW;
#pragma unroll
        for (int ks = 0; ks < kTile / 16; ++ks) {
          uint32_t a[4], b0, b1;
          ldsm_x4_trans(a, Dl + (ks * 16 + arow) * kSO + acol);
          ldsm_x2_trans(b0, b1, In + (ks * 16 + brow) * kSW + warp * 8);
          mma16816<T>(dw[0], a, b0, b1);
        }
      }
#pragma unroll
      for (int h = 1; h < NH; ++h) {                      // hidden h [64][64]: mt = 0..3, nt = warp
        const T* Dl = sm + S::D + h * kTile * kSW;
        const T* In = sm + S::A + (h - 1) * kTile * kSW;
#pragma unroll
        for (int ks = 0; ks < kTile / 16; ++ks) {
          uint32_t b0, b1;
          ldsm_x2_trans(b0, b1, In + (ks * 16 + brow) * kSW + warp * 8);
#pragma unroll
          for (int mt = 0; mt < 4; ++mt) {
            uint32_t a[4];
            ldsm_x4_trans(a, Dl + (ks * 16 + arow) * kSW + mt * 16 + acol);
            mma16816<T>(dw[1 + 4 * (h - 1) + mt], a, b0, b1);
          }
        }
      }
      {                                                   // first layer [64][N_IN]
        constexpr int n8 = N_IN / 8, FT = N_IN / 16;      // n-tiles, tiles per warp
        static_assert(8 % n8 == 0 && 1 + 4 * (NH - 1) + FT == S::TILES_PER_WARP, "tile plan");
        const T* Dl = sm + S::D;
        const T* In = sm + S::X;
        const int nt = warp % n8, mt0 = warp / n8;
#pragma unroll
        for (int ks = 0; ks < kTile / 16; ++ks) {
          uint32_t b0, b1;
          ldsm_x2_trans(b0, b1, In + (ks * 16 + brow) * S::SX + nt * 8);
#pragma unroll
          for (int i = 0; i < FT; ++i) {
            uint32_t a[4];
            ldsm_x4_trans(a, Dl + (ks * 16 + arow) * kSW + (mt0 + i * (8 / n8)) * 16 + acol);
            mma16816<T>(dw[1 + 4 * (NH - 1) + i], a, b0, b1);
          }
        }
      }
    }
  }
  if constexpr (S::PF) cp_async_wait_all();     // the last staging copies (zero fill) have landed
  // ---- per-CTA partials to the workspace
  float* wsb = ws + (int64_t)blockIdx.x * n_params;
  const int off_h = kWidth * N_IN;
  const int off_o = off_h + (NH - 1) * kWidth * kWidth;
#pragma unroll
  for (int i = 0; i < S::TILES_PER_WARP; ++i) {
    const int id = warp + i * kWarps;
    if (id >= S::N_WTILES) break;
    int base, fan_in, mt, nt, rows;
    if (id < 8) { base = off_o; fan_in = kWidth; mt = 0; nt = id; rows = n_out; }
    else if (id < 8 + (NH - 1) * 32) {
      const int j = id - 8, h = 1 + j / 32, r = j % 32;
      base = off_h + (h - 1) * kWidth * kWidth; fan_in = kWidth; mt = r / 8; nt = r % 8; rows = kWidth;
    } else {
      const int j = id - 8 - (NH - 1) * 32;
      base = 0; fan_in = N_IN; mt = j / (N_IN / 8); nt = j % (N_IN / 8); rows = kWidth;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int m = mt * 16 + g + (e >> 1) * 8, n = nt * 8 + 2 * t + (e & 1);
      if (m < rows) wsb[base + m * fan_in + n] = dw[i][e];
    }
  }
  if (MODE == 1) {   // per-CTA sum of squared residuals after the weight partials
    __shared__ float sq_part[kWarps];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) sq_part[warp] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < kWarps; ++w) s += sq_part[w];
      ws[(int64_t)gridDim.x * n_params + blockIdx.x] = s;
    }
  }
}

// dW[j] += (sum_b ws[b][j]) / loss_scale, summed over b in increasing order; the loss
// partials (after the nb x n weight partials) are summed the same way into *sq_sum.
// Sums the per-CTA partial weight gradients: one CTA per 32 consecutive parameters, its 16
// warps take interleaved slices of the partials (coalesced 128-byte rows, eight in flight per
// warp), and the 16 warp sums are added in a fixed order, so the result does not depend on
// scheduling.
constexpr int kReduceCols = 32, kReduceWarps = 16, kReduceUnroll = 8;
__global__ void __launch_bounds__(kReduceCols * kReduceWarps)
reduce_partials_kernel(const float* __restrict__ ws, int nb, int64_t n, float inv_scale,
                       float* __restrict__ dW, float* __restrict__ sq_sum) {
  __shared__ float part[kReduceWarps][kReduceCols];
  // launched as a programmatic dependent of the training pass: wait until that grid has completed
  // and its writes are visible (a no-op for an ordinary launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * kReduceCols + lane;
  // warp w takes partial rows w, w + 16, ...; kReduceUnroll independent loads in flight, each
  // into its own accumulator, combined pairwise in a fixed order
  float acc[kReduceUnroll];
#pragma unroll
  for (int u = 0; u < kReduceUnroll; ++u) acc[u] = 0.f;
  if (j < n) {
    int b = w;
    for (; b + (kReduceUnroll - 1) * kReduceWarps < nb; b += kReduceUnroll * kReduceWarps) {
      float v[kReduceUnroll];
#pragma unroll
      for (int u = 0; u < kReduceUnroll; ++u) v[u] = __ldcs(ws + (int64_t)(b + u * kReduceWarps) * n + j);
#pragma unroll
      for (int u = 0; u < kReduceUnroll; ++u) acc[u] += v[u];
    }
    for (; b < nb; b += kReduceWarps) acc[0] += __ldcs(ws + (int64_t)b * n + j);
  }
#pragma unroll
  for (int width = kReduceUnroll / 2; width > 0; width >>= 1)
#pragma unroll
    for (int u = 0; u < width; ++u) acc[u] += acc[u + width];
  part[w][lane] = acc[0];
  __syncthreads();
  if (w == 0 && j < n) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kReduceWarps; ++k) s += part[k][lane];
    dW[j] += s * inv_scale;
  }
  if (sq_sum && blockIdx.x == 0 && w == 1) {
    float s = 0.f;
    for (int b = lane; b < nb; b += 32) s += ws[(int64_t)nb * n + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) *sq_sum = s;
  }
}

int reduce_blocks(int64_t n_params) { return (int)((n_params + kReduceCols - 1) / kReduceCols); }

}  // namespace

// Launched with programmatic stream serialisation: the reduction grid may be scheduled while the
// training pass before it on the stream is still running (its launch latency hidden behind that
// pass); the kernel's first instruction waits for the pass to complete.
sxe_status launch_mlp_reduce(const float* ws, int nb, int64_t n_params, float inv_scale, float* dW, float* sq_sum,
                             cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)reduce_blocks(n_params));
  cfg.blockDim = dim3(kReduceCols * kReduceWarps);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, reduce_partials_kernel, ws, nb, n_params, inv_scale, dW, sq_sum);
  if (e != cudaSuccess) return set_error(SXE_ECUDA, "mlp_bwd_reduce: %s", cudaGetErrorString(e));
  return check_launch("mlp_bwd_reduce");
}

int g_mlp_kernel = SXE_MLP_KERNEL_AUTO;

namespace {

int num_sms();

// CTAs of the backward kernel that fit on one SM (shared memory and registers), cached.
template <typename T, int N_IN, int NH, int MODE>
int bwd_ctas_per_sm() {
  return kernel_ctas_per_sm((const void*)mlp_bwd_kernel<T, N_IN, NH, MODE>, kThreads,
                            Smem<N_IN, NH>::BWD_END * (int)sizeof(T));
}

int num_sms() { return device_sm_count(); }

template <typename T, int N_IN, int NH>
sxe_status fwd_launch(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out, void* act,
                      cudaStream_t s) {
  using S = Smem<N_IN, NH>;
  const size_t bytes = (size_t)S::FWD_END * sizeof(T);   // weights + input tile
  auto k = mlp_fwd_kernel<T, N_IN, NH>;
  const int per_sm = kernel_ctas_per_sm((const void*)k, kThreads, (int)bytes);   // registers, shared memory
  const int64_t n_tiles = (P + kTile - 1) / kTile;
  const int grid = (int)std::min<int64_t>(n_tiles, (int64_t)per_sm * num_sms());
  k<<<grid, kThreads, bytes, s>>>((const T*)W, (const T*)in, P, d->n_out, out, (T*)act);
  return check_launch("mlp_fwd");
}

template <typename T, int N_IN, int NHC>
sxe_status field_launch(const void* Wd, const void* Wc, const void* enc, const float* dirs, int64_t P, int S,
                        int n_out_c, float* sigma, float* logits, cudaStream_t s) {
  const size_t bytes = (size_t)(Smem<N_IN, 1>::FWD_END + Smem<32, NHC>::FWD_END) * sizeof(T);
  auto k = vr_field_mlp_kernel<T, N_IN, NHC>;
  const int per_sm = kernel_ctas_per_sm((const void*)k, kThreads, (int)bytes);
  const int64_t n_tiles = (P + kTile - 1) / kTile;
  const int grid = (int)std::min<int64_t>(n_tiles, (int64_t)per_sm * num_sms());
  k<<<grid, kThreads, bytes, s>>>((const T*)Wd, (const T*)Wc, (const T*)enc, dirs, P, S, n_out_c, sigma, logits);
  return check_launch("vr_field_mlp");
}

template <typename T, int N_IN>
sxe_status field_nh(int nhc, const void* Wd, const void* Wc, const void* enc, const float* dirs, int64_t P, int S,
                    int n_out_c, float* sigma, float* logits, cudaStream_t s) {
  switch (nhc) {
    case 1: return field_launch<T, N_IN, 1>(Wd, Wc, enc, dirs, P, S, n_out_c, sigma, logits, s);
    case 2: return field_launch<T, N_IN, 2>(Wd, Wc, enc, dirs, P, S, n_out_c, sigma, logits, s);
    default: return field_launch<T, N_IN, 3>(Wd, Wc, enc, dirs, P, S, n_out_c, sigma, logits, s);
  }
}

template <typename T>
sxe_status field_in(int n_in, int nhc, const void* Wd, const void* Wc, const void* enc, const float* dirs, int64_t P,
                    int S, int n_out_c, float* sigma, float* logits, cudaStream_t s) {
  switch (n_in) {
    case 16: return field_nh<T, 16>(nhc, Wd, Wc, enc, dirs, P, S, n_out_c, sigma, logits, s);
    case 32: return field_nh<T, 32>(nhc, Wd, Wc, enc, dirs, P, S, n_out_c, sigma, logits, s);
    default: return field_nh<T, 64>(nhc, Wd, Wc, enc, dirs, P, S, n_out_c, sigma, logits, s);
  }
}

template <typename T, int N_IN, int NH>
sxe_status bwd_launch(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                      float loss_scale, int64_t P, float* din, float* dW, float* sq_sum, float* ws, int grid,
                      cudaStream_t s, int din_group, int64_t lc) {
  using S = Smem<N_IN, NH>;
  const size_t bytes = (size_t)S::BWD_END * sizeof(T);
  const int64_t n_params = sxe_mlp_n_params(d);
  if (target) {
    auto k = mlp_bwd_kernel<T, N_IN, NH, 1>;
    kernel_ctas_per_sm((const void*)k, kThreads, (int)bytes);
    k<<<grid, kThreads, bytes, s>>>((const T*)W, (const T*)in, P, d->n_out, dout, target, loss_scale,
                                    l2_inv_count(lc, d->n_out), din, ws, n_params, sq_sum, din_group);
  } else {
    auto k = mlp_bwd_kernel<T, N_IN, NH, 0>;
    kernel_ctas_per_sm((const void*)k, kThreads, (int)bytes);
    k<<<grid, kThreads, bytes, s>>>((const T*)W, (const T*)in, P, d->n_out, dout, target, loss_scale,
                                    l2_inv_count(lc, d->n_out), din, ws, n_params, sq_sum, din_group);
  }
  sxe_status st = check_launch("mlp_bwd");
  if (st != SXE_OK) return st;
  return launch_mlp_reduce(ws, grid, n_params, 1.f / loss_scale, dW, target ? sq_sum : nullptr, s);
}

template <typename T, int N_IN>
sxe_status fwd_nh(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out, void* act, cudaStream_t s) {
  switch (d->n_hidden) {
    case 1: return fwd_launch<T, N_IN, 1>(d, W, in, P, out, act, s);
    case 2: return fwd_launch<T, N_IN, 2>(d, W, in, P, out, act, s);
    default: return fwd_launch<T, N_IN, 3>(d, W, in, P, out, act, s);
  }
}
template <typename T>
sxe_status fwd_in(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out, void* act, cudaStream_t s) {
  switch (d->n_in) {
    case 16: return fwd_nh<T, 16>(d, W, in, P, out, act, s);
    case 32: return fwd_nh<T, 32>(d, W, in, P, out, act, s);
    default: return fwd_nh<T, 64>(d, W, in, P, out, act, s);
  }
}
template <typename T, int N_IN>
sxe_status bwd_nh(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                  float ls, int64_t P, float* din, float* dW, float* sq, float* ws, int grid, cudaStream_t s, int dg,
                  int64_t lc) {
  switch (d->n_hidden) {
    case 1: return bwd_launch<T, N_IN, 1>(d, W, in, dout, target, ls, P, din, dW, sq, ws, grid, s, dg, lc);
    case 2: return bwd_launch<T, N_IN, 2>(d, W, in, dout, target, ls, P, din, dW, sq, ws, grid, s, dg, lc);
    default: return bwd_launch<T, N_IN, 3>(d, W, in, dout, target, ls, P, din, dW, sq, ws, grid, s, dg, lc);
  }
}
template <typename T>
sxe_status bwd_in(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                  float ls, int64_t P, float* din, float* dW, float* sq, float* ws, int grid, cudaStream_t s, int dg,
                  int64_t lc) {
  switch (d->n_in) {
    case 16: return bwd_nh<T, 16>(d, W, in, dout, target, ls, P, din, dW, sq, ws, grid, s, dg, lc);
    case 32: return bwd_nh<T, 32>(d, W, in, dout, target, ls, P, din, dW, sq, ws, grid, s, dg, lc);
    default: return bwd_nh<T, 64>(d, W, in, dout, target, ls, P, din, dW, sq, ws, grid, s, dg, lc);
  }
}

template <typename T, int N_IN>
int ctas_nh(int nh) {
  switch (nh) {
    case 1: return std::min(bwd_ctas_per_sm<T, N_IN, 1, 0>(), bwd_ctas_per_sm<T, N_IN, 1, 1>());
    case 2: return std::min(bwd_ctas_per_sm<T, N_IN, 2, 0>(), bwd_ctas_per_sm<T, N_IN, 2, 1>());
    default: return std::min(bwd_ctas_per_sm<T, N_IN, 3, 0>(), bwd_ctas_per_sm<T, N_IN, 3, 1>());
  }
}
template <typename T>
int ctas_in(const sxe_mlp_desc* d) {
  switch (d->n_in) {
    case 16: return ctas_nh<T, 16>(d->n_hidden);
    case 32: return ctas_nh<T, 32>(d->n_hidden);
    default: return ctas_nh<T, 64>(d->n_hidden);
  }
}

}  // namespace

// Persistent grid of the backward kernel: every resident CTA slot of the device, at most
// one CTA per tile of 128 points.
int mlp_grid_blocks(const sxe_mlp_desc* d, int64_t P) {
  const int64_t n_tiles = (P + kTile - 1) / kTile;
  const int per_sm = d->dtype == SXE_F16 ? ctas_in<__half>(d) : ctas_in<__nv_bfloat16>(d);
  return (int)std::max<int64_t>(1, std::min<int64_t>(n_tiles, (int64_t)num_sms() * per_sm));
}

sxe_status launch_mlp_fwd(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out, void* act,
                          cudaStream_t s, bool shared_gpu) {
  // the three-tile tcgen05 kernel's forward-only form for n_out <= 16 (automatic choice), else
  // mma.sync.  A caller whose launches run beside other streams' kernels (the serving loop) gets
  // mma.sync under the automatic choice: each CTA of the persistent tcgen05 kernel needs a whole
  // SM (213 KB of shared memory, 384 threads of 155 registers), so it starts only where the other
  // streams' blocks have drained and then holds that SM to itself.  Serving mixed-d queries from
  // four streams: 2.6 against 2.0 G points/s for the simplex encoder, 0.98 against 0.59 for the grid.
  const bool tc3 = g_mlp_kernel == SXE_MLP_KERNEL_TCGEN05_3TILE || (g_mlp_kernel == SXE_MLP_KERNEL_AUTO && !shared_gpu);
  if (tc3 && mlp_tc3_applies(d)) return launch_mlp_fwd_tc3(d, W, in, P, out, act, s);
  return d->dtype == SXE_F16 ? fwd_in<__half>(d, W, in, P, out, act, s)
                             : fwd_in<__nv_bfloat16>(d, W, in, P, out, act, s);
}

sxe_status launch_vr_field_mlp(const sxe_mlp_desc* dd, const void* Wd, const sxe_mlp_desc* dc, const void* Wc,
                               const void* enc, const float* dirs, int64_t R, int S, float* sigma, float* logits,
                               float* dens_out, void* color_in, cudaStream_t s) {
  // the tcgen05 form (three sample tiles per SM) under the automatic and three-tile settings
  if ((g_mlp_kernel == SXE_MLP_KERNEL_AUTO || g_mlp_kernel == SXE_MLP_KERNEL_TCGEN05_3TILE) && dc->n_out <= 8)
    return launch_vr_field_tc3(dd, Wd, dc, Wc, enc, dirs, R, S, sigma, logits, dens_out, color_in, s);
  const int64_t P = R * S;
  if (dens_out && color_in) {      // the intermediates asked for: the three launches, which write them
    sxe_status st = launch_mlp_fwd(dd, Wd, enc, P, dens_out, nullptr, s);
    if (st == SXE_OK) st = launch_vr_field(dens_out, dirs, R, S, dd->dtype, sigma, color_in, s);
    if (st == SXE_OK) st = launch_mlp_fwd(dc, Wc, color_in, P, logits, nullptr, s);
    return st;
  }
  return dd->dtype == SXE_F16
             ? field_in<__half>(dd->n_in, dc->n_hidden, Wd, Wc, enc, dirs, P, S, dc->n_out, sigma, logits, s)
             : field_in<__nv_bfloat16>(dd->n_in, dc->n_hidden, Wd, Wc, enc, dirs, P, S, dc->n_out, sigma, logits, s);
}

sxe_status launch_mlp_bwd(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                          const float* target, float loss_scale, int64_t P, float* din, float* dW, float* sq_sum,
                          float* ws, int grid, cudaStream_t s, int din_group, int64_t loss_count) {
  const int64_t lc = loss_count > 0 ? loss_count : P;   // the L2 gradient's 2 / (count * n_out)
  // automatic choice: for a narrow output layer (n_out <= 8) the three-tile tcgen05 kernel (image
  // network, 2^18 points: 43.8 us per pass, against 62.4 us for the two-tile kernel and 62.5 us
  // for mma.sync), else the two-tile tcgen05 kernel where its plan fits, else mma.sync
  if (g_mlp_kernel == SXE_MLP_KERNEL_AUTO && mlp_tc3_applies(d))
    return launch_mlp_bwd_tc3(d, W, in, dout, target, loss_scale, P, din, dW, sq_sum, ws, grid, s, din_group, lc);
  if (g_mlp_kernel == SXE_MLP_KERNEL_TCGEN05_PIPELINED)
    return launch_mlp_bwd_ws(d, W, in, dout, target, loss_scale, P, din, dW, sq_sum, ws, grid, s, din_group, lc);
  if (g_mlp_kernel == SXE_MLP_KERNEL_TCGEN05_3TILE && mlp_tc3_applies(d))
    return launch_mlp_bwd_tc3(d, W, in, dout, target, loss_scale, P, din, dW, sq_sum, ws, grid, s, din_group, lc);
  if (g_mlp_kernel == SXE_MLP_KERNEL_TCGEN05_3TILE)
    return launch_mlp_bwd_tc(d, W, in, dout, target, loss_scale, P, din, dW, sq_sum, ws, grid, s, din_group, lc);
  if (g_mlp_kernel == SXE_MLP_KERNEL_TCGEN05 || (g_mlp_kernel == SXE_MLP_KERNEL_AUTO && mlp_tc2_applies(d, grid)))
    return launch_mlp_bwd_tc(d, W, in, dout, target, loss_scale, P, din, dW, sq_sum, ws, grid, s, din_group, lc);
  return d->dtype == SXE_F16
             ? bwd_in<__half>(d, W, in, dout, target, loss_scale, P, din, dW, sq_sum, ws, grid, s, din_group, lc)
             : bwd_in<__nv_bfloat16>(d, W, in, dout, target, loss_scale, P, din, dW, sq_sum, ws, grid, s, din_group, lc);
}

}  // namespace sxe
