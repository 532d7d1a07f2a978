// Volumetric field of a batch of samples in one pass on the 5th-generation tensor cores (Sec. 6.2):
// density network (encoding -> 64 -> 16), sigma = exp(min(v_0, 15)), colour input [v_0..v_15, SH(d)],
// colour network (32 -> 64 -> ... -> n_out), the same arithmetic as vr_field_mlp_kernel's
// mma.sync form.  Three 128-sample tiles are in flight per SM, one per 128-thread group, each
// issuing its own tcgen05 products (the hidden layers, fp32 accumulators in TMEM); the two
// narrow output layers run on warp-level mma.sync in the epilogues, each warp on its own 32 rows.
// Per tile: density hidden layer, colour hidden layers on tcgen05; density outputs, sigma and
// the colour input's first 16 columns from the first epilogue (the spherical-harmonics half is
// written at the tile's start); the colour logits from the last.  On request the density outputs
// (binary32) and the colour input rows are written out too, for a backward pass that reads them.
// Every wait is bounded.
#include "mlp_tc3.cuh"

namespace sxe {
namespace {

// Shared memory of one CTA: per group the density input, the colour input and two hidden-layer
// buffers (density hidden, then the colour hidden layers alternating), then the weights.
template <int N_IN, int NHC>
struct Fd3 {
  static constexpr int G = 3;
  static constexpr int X = 0;                                // [128][N_IN] encoding rows
  static constexpr int X2 = X + kM * N_IN * 2;               // [128][32] colour input
  static constexpr int HA = X2 + kM * 32 * 2;                // [128][64]
  static constexpr int HB = HA + kM * kW * 2;                // [128][64]
  static constexpr int GROUP = HB + kM * kW * 2;
  static constexpr int W0D = G * GROUP;                      // [64][N_IN] density hidden layer
  static constexpr int WOD = W0D + kW * N_IN * 2;            // [16][64] density outputs
  static constexpr int W0C = WOD + 16 * kW * 2;              // [64][32] colour hidden layer 0
  static constexpr int WHC = W0C + kW * 32 * 2;              // (NHC-1) x [64][64]
  static constexpr int END = WHC + (NHC - 1) * kW * kW * 2;
  static constexpr int SMEM = END > 116 * 1024 ? END : 116 * 1024;   // one CTA (and TMEM owner) per SM
  static constexpr int THREADS = 128 * G;
  static_assert(END <= 227 * 1024, "shared-memory plan");
};

template <typename T, int N_IN, int NHC, typename S>
__device__ void load_field_weights(const T* __restrict__ Wd, const T* __restrict__ Wc, unsigned char* sm) {
  for (int i = threadIdx.x; i < kW * N_IN; i += S::THREADS) *cm<T>(sm + S::W0D, i / N_IN, i % N_IN, N_IN) = Wd[i];
  const T* Wdo = Wd + kW * N_IN;
  for (int i = threadIdx.x; i < 16 * kW; i += S::THREADS) *cm<T>(sm + S::WOD, i / kW, i % kW, kW) = Wdo[i];
  for (int i = threadIdx.x; i < kW * 32; i += S::THREADS) *cm<T>(sm + S::W0C, i / 32, i % 32, 32) = Wc[i];
  const T* Wch = Wc + kW * 32;
  for (int i = threadIdx.x; i < (NHC - 1) * kW * kW; i += S::THREADS) {
    const int h = i / (kW * kW), o = (i / kW) % kW, c = i % kW;
    *cm<T>(sm + S::WHC + h * kW * kW * 2, o, c, kW) = Wch[i];
  }
}

template <typename T, int N_IN, int NHC>
__global__ void __launch_bounds__(Fd3<N_IN, NHC>::THREADS, 1)
vr_field_tc3_kernel(const T* __restrict__ Wd, const T* __restrict__ Wc, const T* __restrict__ enc,
                    const float* __restrict__ dirs, int64_t P, int S_, int n_out_c, float* __restrict__ sigma,
                    float* __restrict__ logits, float* __restrict__ dens_out, T* __restrict__ color_in,
                    int* __restrict__ err) {
  using S = Fd3<N_IN, NHC>;
  constexpr int G = S::G;
  constexpr bool BF16 = std::is_same<T, __nv_bfloat16>::value;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[G];
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 2, q = warp & 3, bar_id = 1 + g;
  const bool issuer = (tid & 127) == 0;
  const int r = q * 32 + lane;
  const int gq = lane >> 2, t4 = lane & 3;
  const int lrow = (lane & 7) + 8 * ((lane >> 3) & 1), lcol = 8 * (lane >> 4);
  const int64_t n_tiles = (P + kM - 1) / kM;
  unsigned char* gs = sm + g * S::GROUP;

  constexpr int kPieces = N_IN / 8;
  uint4 pf[kPieces];
  auto prefetch = [&](int64_t t) {
#pragma unroll
    for (int j = 0; j < kPieces; ++j) {
      const int64_t row = t * kM + r;
      pf[j] = (t < n_tiles && row < P) ? __ldg(reinterpret_cast<const uint4*>(enc + row * N_IN + 8 * j))
                                       : make_uint4(0, 0, 0, 0);
    }
  };
  const int64_t stride = (int64_t)G * gridDim.x;
  const int64_t first = (int64_t)blockIdx.x + (int64_t)g * gridDim.x;
  prefetch(first);
  load_field_weights<T, N_IN, NHC, S>(Wd, Wc, sm);
  // the colour output layer's weights as mma.sync B fragments (n = output gq, k = hidden)
  const T* Wco = Wc + kW * 32 + (NHC - 1) * kW * kW;
  uint32_t by[4][2];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int k = 16 * ks + 2 * t4, base = gq * kW;
    by[ks][0] = wpair<T>(Wco, base + k, base + k + 1, gq < n_out_c, gq < n_out_c);
    by[ks][1] = wpair<T>(Wco, base + k + 8, base + k + 9, gq < n_out_c, gq < n_out_c);
  }
  const uint32_t lm_h = (uint32_t)tc::cm_offset(32 * q + lrow, lcol, kW);
  const uint32_t lm_x2 = (uint32_t)tc::cm_offset(32 * q + lrow, lcol, 32);   // + 1024 mt (16 rows of 64 bytes)
  const int brow8 = (lane & 7) + 8 * (lane >> 4), bcol8 = 8 * ((lane >> 3) & 1);
  const uint32_t lm_wod = tc::smem_u32(sm + S::WOD) + (uint32_t)tc::cm_offset(brow8, bcol8, kW);
  if (tid == 0)
    for (int i = 0; i < G; ++i) tc::mbar_init(&mbar[i], 1);
  if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base + (uint32_t)(g * 64);
  const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
  uint32_t phase = 0;
  bool failed = false;

  auto issue = [&](const unsigned char* A, const unsigned char* B, int K) {
    tc::fence_smem_async();
    tc::fence_before_sync();
    group_sync(bar_id);
    if (issuer) {
      tc::fence_after_sync();
      const uint32_t sbo = (uint32_t)(K / 8) * 128u;
      const uint64_t da = tc::smem_desc(tc::smem_u32(A), 128u, sbo), db = tc::smem_desc(tc::smem_u32(B), 128u, sbo);
      const uint32_t id = tc::idesc_f16(kM, kW, BF16);
      for (int ks = 0; ks < K / 16; ++ks) tc::mma_f16(tmem, da + (uint64_t)(ks * 16), db + (uint64_t)(ks * 16), id, ks > 0);
      tc::commit(&mbar[g]);
    }
  };
  auto wait = [&]() -> bool {
    const bool ok = tc::mbar_wait_sleep(&mbar[g], phase, 20000u, 2000000000ull, 1u << 20);
    phase ^= 1u;
    tc::fence_after_sync();
    return !group_any(bar_id, !ok);
  };
  // relu of the 64-column accumulator into row r of a [128][64] tile
  auto relu_out = [&](unsigned char* H) {
    float v[64];
    tc::tmem_ld64(lane_addr, v);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint4 u;
      u.x = pack2_relu<T>(v[8 * k + 0], v[8 * k + 1]);
      u.y = pack2_relu<T>(v[8 * k + 2], v[8 * k + 3]);
      u.z = pack2_relu<T>(v[8 * k + 4], v[8 * k + 5]);
      u.w = pack2_relu<T>(v[8 * k + 6], v[8 * k + 7]);
      *reinterpret_cast<uint4*>(H + tc::cm_offset(r, 8 * k, kW)) = u;
    }
  };

  for (int64_t tile = first; tile < n_tiles; tile += stride) {
    const int64_t row0 = tile * kM;
    const int rows = (int)(P - row0 < kM ? P - row0 : kM);
#pragma unroll
    for (int j = 0; j < kPieces; ++j) *reinterpret_cast<uint4*>(gs + S::X + tc::cm_offset(r, 8 * j, N_IN)) = pf[j];
    prefetch(tile + stride);
    {                                                   // colour input columns 16-31: SH(d) of the ray
      const int64_t ray = (row0 + r < P ? row0 + r : P - 1) / S_;
      float h[16];
      sh16(__ldg(dirs + ray * 3), __ldg(dirs + ray * 3 + 1), __ldg(dirs + ray * 3 + 2), h);
      uint4 a, b;
      a.x = pack2<T>(h[0], h[1]);   a.y = pack2<T>(h[2], h[3]);   a.z = pack2<T>(h[4], h[5]);   a.w = pack2<T>(h[6], h[7]);
      b.x = pack2<T>(h[8], h[9]);   b.y = pack2<T>(h[10], h[11]); b.z = pack2<T>(h[12], h[13]); b.w = pack2<T>(h[14], h[15]);
      *reinterpret_cast<uint4*>(gs + S::X2 + tc::cm_offset(r, 16, 32)) = a;
      *reinterpret_cast<uint4*>(gs + S::X2 + tc::cm_offset(r, 24, 32)) = b;
    }
    // ---- density network: hidden layer on tcgen05, the 16 outputs on mma.sync
    issue(gs + S::X, sm + S::W0D, N_IN);
    if (!wait()) { failed = true; break; }
    relu_out(gs + S::HA);
    __syncwarp();
    {
      const uint32_t sH = tc::smem_u32(gs + S::HA) + lm_h;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        uint32_t ha[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) ldsm_x4(ha[ks], sH + 2048u * mt + 256u * ks);
        float y[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          uint32_t b[4];                                // outputs 0-7 (b[0], b[1]) and 8-15 (b[2], b[3])
          ldsm_x4(b, lm_wod + 256u * ks);
          mma16816<T>(y[0], ha[ks], b[0], b[1]);
          mma16816<T>(y[1], ha[ks], b[2], b[3]);
        }
        if (t4 == 0) {                                  // output 0 of rows gq, gq + 8: the density
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int rl = 32 * q + 16 * mt + gq + 8 * half;
            if (rl < rows) sigma[row0 + rl] = vr_density(y[0][2 * half]);
          }
        }
        if (dens_out) {                                 // the 16 outputs in binary32, if asked
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int rl = 32 * q + 16 * mt + gq + 8 * half;
            if (rl < rows)
#pragma unroll
              for (int nt = 0; nt < 2; ++nt)
                *reinterpret_cast<float2*>(dens_out + (row0 + rl) * 16 + 8 * nt + 2 * t4) =
                    make_float2(y[nt][2 * half], y[nt][2 * half + 1]);
          }
        }
        // the 16 outputs, rounded, are the colour input's columns 0-15
        stsm_x4(tc::smem_u32(gs + S::X2) + lm_x2 + 1024u * mt, pack2<T>(y[0][0], y[0][1]), pack2<T>(y[0][2], y[0][3]),
                pack2<T>(y[1][0], y[1][1]), pack2<T>(y[1][2], y[1][3]));
      }
    }
    if (color_in) {                                     // the colour input row, if asked (this warp's rows)
      __syncwarp();
      if (r < rows)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          *reinterpret_cast<uint4*>(color_in + (row0 + r) * 32 + 8 * j) =
              *reinterpret_cast<const uint4*>(gs + S::X2 + tc::cm_offset(r, 8 * j, 32));
    }
    // ---- colour network: hidden layers on tcgen05 (HA, HB alternating), outputs on mma.sync
    issue(gs + S::X2, sm + S::W0C, 32);
    if (!wait()) { failed = true; break; }
    relu_out(gs + S::HA);
#pragma unroll
    for (int hc = 1; hc < NHC; ++hc) {
      issue(gs + ((hc & 1) ? S::HA : S::HB), sm + S::WHC + (hc - 1) * kW * kW * 2, kW);
      if (!wait()) { failed = true; break; }
      relu_out(gs + ((hc & 1) ? S::HB : S::HA));
    }
    if (failed) break;
    __syncwarp();
    {
      const uint32_t sH = tc::smem_u32(gs + (((NHC - 1) & 1) ? S::HB : S::HA)) + lm_h;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        uint32_t ha[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) ldsm_x4(ha[ks], sH + 2048u * mt + 256u * ks);
        float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) mma16816<T>(y, ha[ks], by[ks][0], by[ks][1]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int rl = 32 * q + 16 * mt + gq + 8 * (e >> 1), o = 2 * t4 + (e & 1);
          if (rl < rows && o < n_out_c) logits[(row0 + rl) * n_out_c + o] = y[e];
        }
      }
    }
  }
  if (failed && (tid & 127) == 0 && err) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, 256);
  }
}

template <typename T, int N_IN, int NHC>
sxe_status field_tc3_launch(const void* Wd, const void* Wc, const void* enc, const float* dirs, int64_t P, int S_,
                            int n_out_c, float* sigma, float* logits, float* dens_out, void* color_in,
                            cudaStream_t s) {
  using S = Fd3<N_IN, NHC>;
  const int64_t n_tiles = (P + kM - 1) / kM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)device_sm_count(), (n_tiles + S::G - 1) / S::G));
  kernel_ctas_per_sm((const void*)vr_field_tc3_kernel<T, N_IN, NHC>, S::THREADS, S::SMEM);
  vr_field_tc3_kernel<T, N_IN, NHC><<<grid, S::THREADS, S::SMEM, s>>>((const T*)Wd, (const T*)Wc, (const T*)enc, dirs,
                                                                       P, S_, n_out_c, sigma, logits, dens_out,
                                                                       (T*)color_in, tc3_error_word());
  return check_launch("vr_field_tc3");
}

template <typename T>
sxe_status field_tc3_in(int n_in, int nhc, const void* Wd, const void* Wc, const void* enc, const float* dirs,
                        int64_t P, int S_, int n_out_c, float* sigma, float* logits, float* dens_out,
                        void* color_in, cudaStream_t s) {
  switch (n_in * 4 + nhc) {
    case 16 * 4 + 1: return field_tc3_launch<T, 16, 1>(Wd, Wc, enc, dirs, P, S_, n_out_c, sigma, logits, dens_out, color_in, s);
    case 16 * 4 + 2: return field_tc3_launch<T, 16, 2>(Wd, Wc, enc, dirs, P, S_, n_out_c, sigma, logits, dens_out, color_in, s);
    case 16 * 4 + 3: return field_tc3_launch<T, 16, 3>(Wd, Wc, enc, dirs, P, S_, n_out_c, sigma, logits, dens_out, color_in, s);
    case 32 * 4 + 1: return field_tc3_launch<T, 32, 1>(Wd, Wc, enc, dirs, P, S_, n_out_c, sigma, logits, dens_out, color_in, s);
    case 32 * 4 + 2: return field_tc3_launch<T, 32, 2>(Wd, Wc, enc, dirs, P, S_, n_out_c, sigma, logits, dens_out, color_in, s);
    case 32 * 4 + 3: return field_tc3_launch<T, 32, 3>(Wd, Wc, enc, dirs, P, S_, n_out_c, sigma, logits, dens_out, color_in, s);
    case 64 * 4 + 1: return field_tc3_launch<T, 64, 1>(Wd, Wc, enc, dirs, P, S_, n_out_c, sigma, logits, dens_out, color_in, s);
    case 64 * 4 + 2: return field_tc3_launch<T, 64, 2>(Wd, Wc, enc, dirs, P, S_, n_out_c, sigma, logits, dens_out, color_in, s);
    default: return field_tc3_launch<T, 64, 3>(Wd, Wc, enc, dirs, P, S_, n_out_c, sigma, logits, dens_out, color_in, s);
  }
}

}  // namespace

sxe_status launch_vr_field_tc3(const sxe_mlp_desc* dd, const void* Wd, const sxe_mlp_desc* dc, const void* Wc,
                               const void* enc, const float* dirs, int64_t R, int S_, float* sigma, float* logits,
                               float* dens_out, void* color_in, cudaStream_t s) {
  if (dc->n_out > 8) return set_error(SXE_EUNSUPPORTED, "vr_field_tc3: colour n_out=%d > 8", dc->n_out);
  const int64_t P = R * S_;
  return dd->dtype == SXE_F16
             ? field_tc3_in<__half>(dd->n_in, dc->n_hidden, Wd, Wc, enc, dirs, P, S_, dc->n_out, sigma, logits,
                                    dens_out, color_in, s)
             : field_tc3_in<__nv_bfloat16>(dd->n_in, dc->n_hidden, Wd, Wc, enc, dirs, P, S_, dc->n_out, sigma, logits,
                                           dens_out, color_in, s);
}

}  // namespace sxe
