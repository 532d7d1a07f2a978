// Tiny fully connected network, forward + L2 loss + backward, on the 5th-generation tensor
// cores (tcgen05) -- Sec. 5 (d)-(e) and Sec. 6.1 of arXiv 2311.15439.
//
// One CTA (8 warps) owns one 128-point tile at a time (persistent loop).  The tile's row r is
// TMEM lane r: every GEMM whose rows are points runs as tcgen05.mma with M = 128, fp16/bf16
// operands from shared memory (core-matrix layout, see tc_ptx.cuh) and an fp32 accumulator
// in TMEM, issued by one thread and completed through an mbarrier:
//   forward   H_0 = relu(X W_0^T), H_h = relu(H_{h-1} W_h^T), Y = H_last W_out^T
//   loss      dY = 2 (Y - target) / (P n_out) * loss_scale            (per row, in registers)
//   backward  dH_last = (dY W_out) * [H_last > 0], dH_{h-1} = (dH_h W_h) * [H_{h-1} > 0],
//             dX = dH_0 W_0
// The epilogues read the accumulator with tcgen05.ld (warp w reads lanes 32 (w % 4)..+31,
// half the columns each), apply ReLU / mask / loss, and write the next operand tile.
// The weight gradients dW_l = Delta_l^T In_l reduce over the points, so their rows are not
// points; they run as mma.sync m16n8k16 over the same shared-memory tiles (ldmatrix.trans)
// while the last tcgen05 product of the tile is in flight, and accumulate across the
// persistent loop in registers (per-CTA partials, summed in a fixed order afterwards).
//
// Every mbarrier wait is bounded: on timeout the kernel raises the device error word, all
// threads leave the loop together, TMEM is freed and the kernel returns.
#include <algorithm>
#include <type_traits>

#include "mlp_tc_common.cuh"

namespace sxe {

__device__ int g_tc_error;   // nonzero once a tensor-core wait timed out

namespace {

using namespace mlpc;
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 64;

template <int N_IN, int NH>
struct TcSmem {
  static constexpr int X = 0;                                 // [128][N_IN]
  static constexpr int H = X + kM * N_IN * 2;                 // NH x [128][64]
  static constexpr int DH = H + NH * kM * kW * 2;             // NH x [128][64]
  static constexpr int DY = DH + NH * kM * kW * 2;            // [128][16]
  static constexpr int W0 = DY + kM * 16 * 2;                 // [64][N_IN]
  static constexpr int WH = W0 + kW * N_IN * 2;               // (NH-1) x [64][64]
  static constexpr int WO = WH + (NH - 1) * kW * kW * 2;      // [16][64]
  static constexpr int WOT = WO + 16 * kW * 2;                // [64][16]
  static constexpr int WHT = WOT + kW * 16 * 2;               // (NH-1) x [64][64]
  static constexpr int W0T = WHT + (NH - 1) * kW * kW * 2;    // [N_IN][64]
  static constexpr int END = W0T + N_IN * kW * 2;
  static constexpr int N_WTILES = 8 + (NH - 1) * 32 + 4 * (N_IN / 8);
  static constexpr int TILES_PER_WARP = (N_WTILES + 7) / 8;
};

// Write W (global [fan_out][fan_in]) as B operand [fan_out][fan_in] and its transpose
// [fan_in][fan_out], rows of the output layer past n_out zero.
template <typename T, int N_IN, int NH, typename S = TcSmem<N_IN, NH>>
__device__ void load_weights_cm(const T* __restrict__ W, int n_out, unsigned char* sm) {
  const T zero = from_f32<T>(0.f);
  for (int i = threadIdx.x; i < kW * N_IN; i += blockDim.x) {
    const int o = i / N_IN, c = i % N_IN;
    const T v = W[i];
    *cm<T>(sm + S::W0, o, c, N_IN) = v;
    *cm<T>(sm + S::W0T, c, o, kW) = v;
  }
  const T* Wh = W + kW * N_IN;
  for (int i = threadIdx.x; i < (NH - 1) * kW * kW; i += blockDim.x) {
    const int h = i / (kW * kW), o = (i / kW) % kW, c = i % kW;
    const T v = Wh[i];
    *cm<T>(sm + S::WH + h * kW * kW * 2, o, c, kW) = v;
    *cm<T>(sm + S::WHT + h * kW * kW * 2, c, o, kW) = v;
  }
  const T* Wo = Wh + (NH - 1) * kW * kW;
  for (int i = threadIdx.x; i < 16 * kW; i += blockDim.x) {
    const int o = i / kW, c = i % kW;
    const T v = o < n_out ? Wo[o * kW + c] : zero;
    *cm<T>(sm + S::WO, o, c, kW) = v;
    *cm<T>(sm + S::WOT, c, o, 16) = v;
  }
}

// MODE 0: dy = dout * loss_scale.  MODE 1: L2 loss against target.
template <typename T, int N_IN, int NH, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
mlp_train_tc_kernel(const T* __restrict__ W, const T* __restrict__ in, int64_t P, int n_out,
                    const float* __restrict__ dout, const float* __restrict__ target, float loss_scale, float inv_count,
                    float* __restrict__ din, int din_group, float* __restrict__ ws, int64_t n_params) {
  using S = TcSmem<N_IN, NH>;
  constexpr bool BF16 = std::is_same<T, __nv_bfloat16>::value;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float sq_part[8];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;
  const int r = quad * 32 + lane;                       // this thread's tile row / TMEM lane
  const int64_t n_tiles = (P + kM - 1) / kM;
  const float inv_scale = 1.f / loss_scale;

  load_weights_cm<T, N_IN, NH>(W, n_out, sm);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
  uint32_t phase = 0;
  bool failed = false;

  float dw[S::TILES_PER_WARP][4];
#pragma unroll
  for (int i = 0; i < S::TILES_PER_WARP; ++i) dw[i][0] = dw[i][1] = dw[i][2] = dw[i][3] = 0.f;
  float sq = 0.f;

  // issue (one thread) after all operand writes, then every thread waits for the product
  auto gemm = [&](const unsigned char* A, const unsigned char* B, int K, int N) -> bool {
    tc::fence_smem_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_gemm(tmem, A, B, K, tc::idesc_f16(kM, N, BF16));
      tc::commit(&mbar);
    }
    const bool ok = tc::mbar_wait(&mbar, phase, kWaitPolls);
    phase ^= 1u;
    tc::fence_after_sync();
    return ok;
  };

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kM;
    // ---- stage the tile's inputs
    for (int i = tid; i < kM * (N_IN / 8); i += kThreads) {
      const int rr = i / (N_IN / 8), c = (i % (N_IN / 8)) * 8;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (row0 + rr < P) v = __ldg(reinterpret_cast<const uint4*>(in + (row0 + rr) * N_IN + c));
      *reinterpret_cast<uint4*>(sm + S::X + tc::cm_offset(rr, c, N_IN)) = v;
    }
    // ---- forward
    bool ok = true;
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      if (h == 0) ok = gemm(sm + S::X, sm + S::W0, N_IN, kW);
      else ok = gemm(sm + S::H + (h - 1) * kM * kW * 2, sm + S::WH + (h - 1) * kW * kW * 2, kW, kW);
      if (__syncthreads_or(!ok)) { failed = true; break; }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int c0 = half * 32 + c * 16;
        float v[16];
        tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
        store16<T>(sm + S::H + h * kM * kW * 2, r, c0, kW, v);
      }
    }
    if (failed) break;
    ok = gemm(sm + S::H + (NH - 1) * kM * kW * 2, sm + S::WO, kW, 16);
    if (__syncthreads_or(!ok)) { failed = true; break; }
    // ---- output delta (warps 0-3 hold the 16 output columns of their rows)
    if (half == 0) {
      float v[16];
      tc::tmem_ld16(lane_addr, v);
      const int64_t row = row0 + r;
#pragma unroll
      for (int o = 0; o < 16; ++o) {
        float dyo = 0.f;
        if (row < P && o < n_out) {
          if (MODE == 0) {
            dyo = dout[row * n_out + o] * loss_scale;
          } else {
            const float res = v[o] - target[row * n_out + o];
            sq = fmaf(res, res, sq);
            dyo = res * inv_count * loss_scale;
          }
        }
        v[o] = dyo;
      }
      store16<T>(sm + S::DY, r, 0, 16, v);
    }
    // ---- hidden deltas, top layer down
#pragma unroll
    for (int h = NH - 1; h >= 0; --h) {
      if (h == NH - 1) ok = gemm(sm + S::DY, sm + S::WOT, 16, kW);
      else ok = gemm(sm + S::DH + (h + 1) * kM * kW * 2, sm + S::WHT + h * kW * kW * 2, kW, kW);
      if (__syncthreads_or(!ok)) { failed = true; break; }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int c0 = half * 32 + c * 16;
        float v[16], a[16];
        tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
        load16<T>(sm + S::H + h * kM * kW * 2, r, c0, kW, a);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = a[j] > 0.f ? v[j] : 0.f;
        store16<T>(sm + S::DH + h * kM * kW * 2, r, c0, kW, v);
      }
    }
    if (failed) break;
    // ---- dX = dH_0 W_0 on the tensor cores, weight gradients on mma.sync meanwhile
    tc::fence_smem_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_gemm(tmem, sm + S::DH, sm + S::W0T, kW, tc::idesc_f16(kM, N_IN, BF16));
      tc::commit(&mbar);
    }
    {
      const int g = lane >> 2, t = lane & 3, q = lane >> 3, rr = lane & 7;
      (void)g; (void)t;
#pragma unroll
      for (int i = 0; i < S::TILES_PER_WARP; ++i) {
        const int id = warp + i * 8;
        if (id >= S::N_WTILES) break;
        const unsigned char *Dl, *In;
        int Kd, Ki, mt, nt;
        if (id < 8) {
          Dl = sm + S::DY; Kd = 16; In = sm + S::H + (NH - 1) * kM * kW * 2; Ki = kW; mt = 0; nt = id;
        } else if (id < 8 + (NH - 1) * 32) {
          const int j = id - 8, h = 1 + j / 32, rem = j % 32;
          Dl = sm + S::DH + h * kM * kW * 2; Kd = kW; In = sm + S::H + (h - 1) * kM * kW * 2; Ki = kW;
          mt = rem / 8; nt = rem % 8;
        } else {
          const int j = id - 8 - (NH - 1) * 32;
          Dl = sm + S::DH; Kd = kW; In = sm + S::X; Ki = N_IN; mt = j / (N_IN / 8); nt = j % (N_IN / 8);
        }
        const uint32_t dl = tc::smem_u32(Dl), il = tc::smem_u32(In);
#pragma unroll
        for (int ks = 0; ks < kM / 16; ++ks) {
          uint32_t a[4], b0, b1;
          ldsm_x4_trans(a, dl + tc::cm_offset(ks * 16 + (q >> 1) * 8 + rr, mt * 16 + (q & 1) * 8, Kd));
          ldsm_x2_trans(b0, b1, il + tc::cm_offset(ks * 16 + (q & 1) * 8 + rr, nt * 8, Ki));
          mma16816<T>(dw[i], a, b0, b1);
        }
      }
    }
    ok = tc::mbar_wait(&mbar, phase, kWaitPolls);
    phase ^= 1u;
    tc::fence_after_sync();
    if (__syncthreads_or(!ok)) { failed = true; break; }
    // ---- input gradient
    {
      constexpr int PER_WARP = N_IN / 2;          // columns per warp half (16 or 32; 8 -> one half)
      const int64_t row = row0 + r;
      if (N_IN >= 32 || half == 0) {
#pragma unroll
        for (int c = 0; c < (N_IN >= 32 ? PER_WARP / 16 : 1); ++c) {
          const int c0 = (N_IN >= 32 ? half * PER_WARP : 0) + c * 16;
          float v[16];
          tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
          if (din && row < P) {
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
              const int col = c0 + j;
              const float2 val = make_float2(v[j] * inv_scale, v[j + 1] * inv_scale);
              if (din_group == 0) {
                *reinterpret_cast<float2*>(din + row * N_IN + col) = val;
              } else if (din_group == 1) {
                din[(int64_t)col * P + row] = val.x;
                din[(int64_t)(col + 1) * P + row] = val.y;
              } else {
                *reinterpret_cast<float2*>(din + ((int64_t)(col / din_group) * P + row) * din_group + col % din_group) = val;
              }
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }

  // ---- per-CTA partials (all threads reach this point together)
  if (failed && tid == 0) atomicExch(&g_tc_error, 1);
  float* wsb = ws + (int64_t)blockIdx.x * n_params;
  const int off_h = kW * N_IN;
  const int off_o = off_h + (NH - 1) * kW * kW;
  {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < S::TILES_PER_WARP; ++i) {
      const int id = warp + i * 8;
      if (id >= S::N_WTILES) break;
      int base, fan_in, mt, nt, rows;
      if (id < 8) { base = off_o; fan_in = kW; mt = 0; nt = id; rows = n_out; }
      else if (id < 8 + (NH - 1) * 32) {
        const int j = id - 8, h = 1 + j / 32, rem = j % 32;
        base = off_h + (h - 1) * kW * kW; fan_in = kW; mt = rem / 8; nt = rem % 8; rows = kW;
      } else {
        const int j = id - 8 - (NH - 1) * 32;
        base = 0; fan_in = N_IN; mt = j / (N_IN / 8); nt = j % (N_IN / 8); rows = kW;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = mt * 16 + g + (e >> 1) * 8, n = nt * 8 + 2 * t + (e & 1);
        if (m < rows) wsb[base + m * fan_in + n] = dw[i][e];
      }
    }
  }
  if (MODE == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) sq_part[warp] = sq;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (MODE == 1 && tid == 0) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += sq_part[w];
    ws[(int64_t)gridDim.x * n_params + blockIdx.x] = s;
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// ---- two tiles in flight per CTA ----------------------------------------------------------
// The kernel above runs each tile's products strictly in sequence (issue, wait, epilogue, next
// product), so the tensor cores idle during the epilogues and the mma.sync weight gradients.
// This one runs two tiles per CTA at once: warps 0-3 (group 0) and warps 4-7 (group 1) each
// own a tile, its shared-memory buffers, 64 TMEM columns, an mbarrier and a named barrier, and
// step through the same sequence independently, so that one group's products run on the tensor
// cores while the other group is in an epilogue or in its weight gradients.  Thread q*32 + lane
// of a group (warp 4g + q) holds row 32 q + lane of its tile, which is TMEM lane 32 q + lane.
// The weights are staged once and shared.  Each group writes its own row of weight-gradient
// partials (rows 2 b and 2 b + 1 of CTA b), summed in a fixed order afterwards.
template <int N_IN, int NH>
struct Tc2Smem {
  static constexpr int X = 0;                                 // per group: [128][N_IN]
  static constexpr int H = X + kM * N_IN * 2;                 // NH x [128][64]
  static constexpr int DH = H + NH * kM * kW * 2;             // NH x [128][64]
  static constexpr int DY = DH + NH * kM * kW * 2;            // [128][16]
  static constexpr int GROUP = DY + kM * 16 * 2;              // bytes of one group's buffers
  static constexpr int W0 = 2 * GROUP;                        // shared weights, as TcSmem
  static constexpr int WH = W0 + kW * N_IN * 2;
  static constexpr int WO = WH + (NH - 1) * kW * kW * 2;
  static constexpr int WOT = WO + 16 * kW * 2;
  static constexpr int WHT = WOT + kW * 16 * 2;
  static constexpr int W0T = WHT + (NH - 1) * kW * kW * 2;
  static constexpr int END = W0T + N_IN * kW * 2;
  // weight-gradient m16n8 tiles per warp of a group: output layer 2 (nt = q, q + 4), hidden
  // layer 8 each (nt = q, q + 4; mt = 0..3), first layer N_IN / 8 (see first_tile)
  static constexpr int N8 = N_IN / 8;
  static constexpr int T_OUT = 2, T_HID = 8, T_FIRST = N8;
  static constexpr int TILES = T_OUT + (NH - 1) * T_HID + T_FIRST;
  static constexpr int FIRST_NT = N8 >= 4 ? N8 / 4 : 1;      // n-tiles of the first layer per warp
  static constexpr int FIRST_MT = N8 >= 4 ? 4 : 2;            // m-tiles per n-tile
};

// (mt, nt) of weight-gradient tile `i` of warp q of a group, and where its values go in the
// [fan_out][fan_in] parameter block: base offset, fan_in, rows kept
template <int N_IN, int NH>
__device__ __forceinline__ void tc2_tile(int i, int q, int n_out, int& mt, int& nt, int& base, int& fan_in,
                                         int& rows) {
  using S = Tc2Smem<N_IN, NH>;
  const int off_h = kW * N_IN, off_o = off_h + (NH - 1) * kW * kW;
  if (i < S::T_OUT) {
    mt = 0; nt = q + 4 * i; base = off_o; fan_in = kW; rows = n_out;
  } else if (i < S::T_OUT + (NH - 1) * S::T_HID) {
    const int j = i - S::T_OUT, h = j / S::T_HID, r = j % S::T_HID;
    mt = r % 4; nt = q + 4 * (r / 4); base = off_h + h * kW * kW; fan_in = kW; rows = kW;
  } else {
    const int r = i - S::T_OUT - (NH - 1) * S::T_HID;
    const int j = r / S::FIRST_MT, k = r % S::FIRST_MT;
    nt = S::N8 >= 4 ? q + 4 * j : q % 2;
    mt = S::N8 >= 4 ? k : q / 2 + 2 * k;
    base = 0; fan_in = N_IN; rows = kW;
  }
}

// TCW: the weight gradients on tcgen05 as well.  dW_out^T = H_last^T dY (64 x 16), dW_h = dH_h^T
// H_{h-1} (64 x 64) and dW_0 = dH_0^T X (64 x N_IN) are M = 64 products over the tile's 128
// points, whose operands are the tile's activation, delta and input buffers read as MN-major
// operands; they accumulate in TMEM (256 columns per group) over the whole persistent loop and
// are read out once at the end.  Without TCW they run on mma.sync into registers.
template <typename T, int N_IN, int NH, int MODE, bool TCW>
__global__ void __launch_bounds__(kThreads, 1)
mlp_train_tc2_kernel(const T* __restrict__ W, const T* __restrict__ in, int64_t P, int n_out,
                     const float* __restrict__ dout, const float* __restrict__ target, float loss_scale, float inv_count,
                     float* __restrict__ din, int din_group, float* __restrict__ ws, int64_t n_params) {
  using S = Tc2Smem<N_IN, NH>;
  constexpr bool BF16 = std::is_same<T, __nv_bfloat16>::value;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ float sq_part[8];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 2, q = warp & 3, bar_id = 1 + g;
  const bool issuer = (tid & 127) == 0;
  const int r = q * 32 + lane;                          // this thread's tile row / TMEM lane
  const int64_t n_tiles = (P + kM - 1) / kM;
  const float inv_scale = 1.f / loss_scale;
  unsigned char* gs = sm + g * S::GROUP;                // this group's buffers

  load_weights_cm<T, N_IN, NH, S>(W, n_out, sm);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  constexpr uint32_t kGroupCols = TCW ? 256u : kTmemCols;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * kGroupCols);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base + (uint32_t)g * kGroupCols;
  const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
  // TCW accumulators: dW_out^T at column 64, dW_h at 80 + 64 (h - 1), dW_0 after them
  const uint32_t c_out = tmem + 64u, c_first = tmem + 80u + 64u * (NH - 1);
  static_assert(!TCW || 80 + 64 * (NH - 1) + N_IN <= 256, "TMEM columns of one group");
  uint32_t phase = 0;
  bool failed = false, any_tile = false;

  float dw[TCW ? 1 : S::TILES][4];
#pragma unroll
  for (int i = 0; i < (TCW ? 1 : S::TILES); ++i) dw[i][0] = dw[i][1] = dw[i][2] = dw[i][3] = 0.f;
  float sq = 0.f;

  // M = 64 weight-gradient product over the tile's 128 points (8 MMAs of K = 16): A' and B' are
  // MN-major views of [points][features] tiles whose 8-point core-matrix rows are kA / kB bytes
  // apart per 8 points; the 8-feature blocks are 128 bytes apart
  auto wgrad = [&](uint32_t d, const unsigned char* A, uint32_t kA, const unsigned char* B, uint32_t kB, int N,
                   bool first) {
    const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B), id = tc::idesc_f16_mn(64, N, BF16);
#pragma unroll
    for (int ks = 0; ks < kM / 16; ++ks)
      tc::mma_f16(d, tc::smem_desc(a0 + ks * 2 * kA, kA, 128u), tc::smem_desc(b0 + ks * 2 * kB, kB, 128u), id,
                  !(first && ks == 0));
  };

  auto issue = [&](const unsigned char* A, const unsigned char* B, int K, int N) {
    tc::fence_smem_async();
    tc::fence_before_sync();
    group_sync(bar_id);
    if (issuer) {
      tc::fence_after_sync();
      issue_gemm(tmem, A, B, K, tc::idesc_f16(kM, N, BF16));
      tc::commit(&mbar[g]);
    }
  };
  auto wait = [&]() -> bool {
    const bool ok = tc::mbar_wait(&mbar[g], phase, kWaitPolls);
    phase ^= 1u;
    tc::fence_after_sync();
    return !group_any(bar_id, !ok);
  };

  // the tile's inputs are loaded into registers one tile ahead (item i = r + 128 j of the
  // tile's 128 x N_IN / 8 sixteen-byte pieces), so their latency hides behind a whole tile
  constexpr int kPieces = N_IN / 8;                     // per thread: 128 rows x N_IN / 8 / 128
  uint4 pf[kPieces];
  auto prefetch = [&](int64_t t) {
#pragma unroll
    for (int j = 0; j < kPieces; ++j) {
      const int i = r + 128 * j, rr = i / (N_IN / 8), c = (i % (N_IN / 8)) * 8;
      const int64_t row = t * kM + rr;
      pf[j] = (t < n_tiles && row < P) ? __ldg(reinterpret_cast<const uint4*>(in + row * N_IN + c))
                                       : make_uint4(0, 0, 0, 0);
    }
  };
  prefetch(2 * (int64_t)blockIdx.x + g);
  for (int64_t tile = 2 * (int64_t)blockIdx.x + g; tile < n_tiles; tile += 2 * (int64_t)gridDim.x) {
    const int64_t row0 = tile * kM;
#pragma unroll
    for (int j = 0; j < kPieces; ++j) {
      const int i = r + 128 * j, rr = i / (N_IN / 8), c = (i % (N_IN / 8)) * 8;
      *reinterpret_cast<uint4*>(gs + S::X + tc::cm_offset(rr, c, N_IN)) = pf[j];
    }
    prefetch(tile + 2 * (int64_t)gridDim.x);
    // this row's targets (L2 loss) or upstream gradients, needed after the forward products
    float yin[16];
    {
      const int64_t row = row0 + r;
      const float* src = MODE == 0 ? dout : target;
#pragma unroll
      for (int o = 0; o < 16; ++o) yin[o] = (row < P && o < n_out) ? __ldg(src + row * n_out + o) : 0.f;
    }
    // ---- forward
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      if (h == 0) issue(gs + S::X, sm + S::W0, N_IN, kW);
      else issue(gs + S::H + (h - 1) * kM * kW * 2, sm + S::WH + (h - 1) * kW * kW * 2, kW, kW);
      if (!wait()) { failed = true; break; }
#pragma unroll
      for (int c0 = 0; c0 < kW; c0 += 32) {
        float v[32];
        tc::tmem_ld32(lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float u[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) u[j] = fmaxf(v[16 * half + j], 0.f);
          store16<T>(gs + S::H + h * kM * kW * 2, r, c0 + 16 * half, kW, u);
        }
      }
    }
    if (failed) break;
    issue(gs + S::H + (NH - 1) * kM * kW * 2, sm + S::WO, kW, 16);
    if (!wait()) { failed = true; break; }
    // ---- output delta
    {
      float v[16];
      tc::tmem_ld16(lane_addr, v);
      const int64_t row = row0 + r;
#pragma unroll
      for (int o = 0; o < 16; ++o) {
        float dyo = 0.f;
        if (row < P && o < n_out) {
          if (MODE == 0) {
            dyo = yin[o] * loss_scale;
          } else {
            const float res = v[o] - yin[o];
            sq = fmaf(res, res, sq);
            dyo = res * inv_count * loss_scale;
          }
        }
        v[o] = dyo;
      }
      store16<T>(gs + S::DY, r, 0, 16, v);
    }
    // ---- hidden deltas, top layer down
#pragma unroll
    for (int h = NH - 1; h >= 0; --h) {
      if (h == NH - 1) issue(gs + S::DY, sm + S::WOT, 16, kW);
      else issue(gs + S::DH + (h + 1) * kM * kW * 2, sm + S::WHT + h * kW * kW * 2, kW, kW);
      if (!wait()) { failed = true; break; }
#pragma unroll
      for (int c0 = 0; c0 < kW; c0 += 32) {
        float v[32];
        tc::tmem_ld32(lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float a[16], u[16];
          load16<T>(gs + S::H + h * kM * kW * 2, r, c0 + 16 * half, kW, a);
#pragma unroll
          for (int j = 0; j < 16; ++j) u[j] = a[j] > 0.f ? v[16 * half + j] : 0.f;
          store16<T>(gs + S::DH + h * kM * kW * 2, r, c0 + 16 * half, kW, u);
        }
      }
    }
    if (failed) break;
    // ---- dX = dH_0 W_0 on the tensor cores; the weight gradients on tcgen05 with it (TCW) or on
    // mma.sync meanwhile
    if constexpr (TCW) {
      tc::fence_smem_async();
      tc::fence_before_sync();
      group_sync(bar_id);
      if (issuer) {
        tc::fence_after_sync();
        constexpr uint32_t kH = (kW / 8) * 128, kDY = (16 / 8) * 128, kX = (N_IN / 8) * 128;
        wgrad(c_out, gs + S::H + (NH - 1) * kM * kW * 2, kH, gs + S::DY, kDY, 16, !any_tile);
#pragma unroll
        for (int h = 1; h < NH; ++h)
          wgrad(tmem + 80u + 64u * (h - 1), gs + S::DH + h * kM * kW * 2, kH, gs + S::H + (h - 1) * kM * kW * 2, kH,
                kW, !any_tile);
        wgrad(c_first, gs + S::DH, kH, gs + S::X, kX, N_IN, !any_tile);
        issue_gemm(tmem, gs + S::DH, sm + S::W0T, kW, tc::idesc_f16(kM, N_IN, BF16));
        tc::commit(&mbar[g]);
      }
      any_tile = true;
    } else {
    issue(gs + S::DH, sm + S::W0T, kW, N_IN);
    {
      const int gq = lane >> 2, t4 = lane & 3, lo = lane >> 3, rr = lane & 7;
      (void)gq; (void)t4;
      const int arow = (lo >> 1) * 8 + rr, acol = (lo & 1) * 8, brow = (lo & 1) * 8 + rr;
      {                                                 // output layer: tiles 0, 1 (nt = q, q + 4)
        const uint32_t dl = tc::smem_u32(gs + S::DY), il = tc::smem_u32(gs + S::H + (NH - 1) * kM * kW * 2);
#pragma unroll
        for (int ks = 0; ks < kM / 16; ++ks) {
          uint32_t a[4];
          ldsm_x4_trans(a, dl + tc::cm_offset(ks * 16 + arow, acol, 16));
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            uint32_t b0, b1;
            ldsm_x2_trans(b0, b1, il + tc::cm_offset(ks * 16 + brow, (q + 4 * j) * 8, kW));
            mma16816<T>(dw[j], a, b0, b1);
          }
        }
      }
#pragma unroll
      for (int h = 1; h < NH; ++h) {                   // hidden h: nt = q, q + 4; mt = 0..3
        const uint32_t dl = tc::smem_u32(gs + S::DH + h * kM * kW * 2);
        const uint32_t il = tc::smem_u32(gs + S::H + (h - 1) * kM * kW * 2);
#pragma unroll
        for (int ks = 0; ks < kM / 16; ++ks) {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            uint32_t b0, b1;
            ldsm_x2_trans(b0, b1, il + tc::cm_offset(ks * 16 + brow, (q + 4 * j) * 8, kW));
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
              uint32_t a[4];
              ldsm_x4_trans(a, dl + tc::cm_offset(ks * 16 + arow, mt * 16 + acol, kW));
              mma16816<T>(dw[S::T_OUT + (h - 1) * S::T_HID + j * 4 + mt], a, b0, b1);
            }
          }
        }
      }
      {                                                 // first layer
        const uint32_t dl = tc::smem_u32(gs + S::DH), il = tc::smem_u32(gs + S::X);
        constexpr int base = S::T_OUT + (NH - 1) * S::T_HID;
#pragma unroll
        for (int ks = 0; ks < kM / 16; ++ks) {
#pragma unroll
          for (int j = 0; j < S::FIRST_NT; ++j) {
            const int nt = S::N8 >= 4 ? q + 4 * j : q % 2;
            uint32_t b0, b1;
            ldsm_x2_trans(b0, b1, il + tc::cm_offset(ks * 16 + brow, nt * 8, N_IN));
#pragma unroll
            for (int k = 0; k < S::FIRST_MT; ++k) {
              const int mt = S::N8 >= 4 ? k : q / 2 + 2 * k;
              uint32_t a[4];
              ldsm_x4_trans(a, dl + tc::cm_offset(ks * 16 + arow, mt * 16 + acol, kW));
              mma16816<T>(dw[base + j * S::FIRST_MT + k], a, b0, b1);
            }
          }
        }
      }
    }
    }
    if (!wait()) { failed = true; break; }
    // ---- input gradient.  Row-major output: staged in the (now free) activation and delta buffers
    // one row per thread, then written by the group as contiguous 16-byte pieces of the tile
    if (din && din_group == 0) {
      constexpr int LD = 128 * (N_IN + 4) * 4 <= 2 * NH * kM * kW * 2 ? N_IN + 4 : N_IN;   // floats per row
      float* st = reinterpret_cast<float*>(gs + S::H);
#pragma unroll
      for (int c0 = 0; c0 < N_IN; c0 += 16) {
        float v[16];
        tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(st + r * LD + c0 + j) =
              make_float4(v[j] * inv_scale, v[j + 1] * inv_scale, v[j + 2] * inv_scale, v[j + 3] * inv_scale);
      }
      group_sync(bar_id);
      for (int i = r; i < kM * (N_IN / 4); i += 128) {
        const int rr = i / (N_IN / 4), c4 = i % (N_IN / 4);
        if (row0 + rr < P)
          *reinterpret_cast<float4*>(din + (row0 + rr) * N_IN + c4 * 4) =
              *reinterpret_cast<const float4*>(st + rr * LD + c4 * 4);
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
            if (din_group == 0) {
              *reinterpret_cast<float2*>(din + row * N_IN + col) = val;
            } else if (din_group == 1) {
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
    tc::fence_before_sync();
    group_sync(bar_id);                                 // the tile's buffers are free again
  }

  // ---- per-group partials (both groups reach this point; a failed group left its loop whole)
  if (failed && (tid & 127) == 0) atomicExch(&g_tc_error, 1);
  float* wsb = ws + (2 * (int64_t)blockIdx.x + g) * n_params;
  if constexpr (TCW) {
    // row m = 16 q + lane of every M = 64 accumulator sits in lane 32 q + lane (lanes 0-15 of the
    // warp); a group without a tile never wrote its accumulators and writes zeros
    const int off_h = kW * N_IN, off_o = off_h + (NH - 1) * kW * kW;
    const int m = 16 * q + lane;
    const uint32_t la = (uint32_t)(q * 32) << 16;
    float v[16];
    tc::tmem_ld16(c_out + la, v);
    if (lane < 16)
#pragma unroll
      for (int o = 0; o < 16; ++o)
        if (o < n_out) wsb[off_o + o * kW + m] = any_tile ? v[o] : 0.f;
#pragma unroll
    for (int h = 1; h < NH; ++h)
#pragma unroll
      for (int c0 = 0; c0 < kW; c0 += 16) {
        tc::tmem_ld16(tmem + 80u + 64u * (h - 1) + la + (uint32_t)c0, v);
        if (lane < 16)
#pragma unroll
          for (int j = 0; j < 16; ++j) wsb[off_h + (h - 1) * kW * kW + m * kW + c0 + j] = any_tile ? v[j] : 0.f;
      }
#pragma unroll
    for (int c0 = 0; c0 < N_IN; c0 += 16) {
      tc::tmem_ld16(c_first + la + (uint32_t)c0, v);
      if (lane < 16)
#pragma unroll
        for (int j = 0; j < 16; ++j) wsb[m * N_IN + c0 + j] = any_tile ? v[j] : 0.f;
    }
  } else {
    const int gq = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int i = 0; i < S::TILES; ++i) {
      int mt, nt, base, fan_in, rows;
      tc2_tile<N_IN, NH>(i, q, n_out, mt, nt, base, fan_in, rows);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = mt * 16 + gq + (e >> 1) * 8, n = nt * 8 + 2 * t4 + (e & 1);
        if (m < rows) wsb[base + m * fan_in + n] = dw[TCW ? 0 : i][e];
      }
    }
  }
  if (MODE == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) sq_part[warp] = sq;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (MODE == 1 && (tid & 127) == 0) {
    float s = 0.f;
    for (int w = 4 * g; w < 4 * g + 4; ++w) s += sq_part[w];
    ws[(int64_t)2 * gridDim.x * n_params + 2 * blockIdx.x + g] = s;
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, 2 * kGroupCols);
  }
}

// ---- warp-specialised: one MMA-issuing warp feeding up to four tiles -------------------------
// The two kernels above issue each tile's products from the tile's own threads, so a tile's
// chain of products (2 NH + 2 of them, each waiting for the epilogue before it) leaves the tensor
// cores idle unless another tile happens to be ready.  Here one thread of a dedicated warp issues
// every product of the CTA: it polls the tiles' "operands ready" barriers in turn and issues the
// next product of whichever tile is ready, so up to SLOTS tiles (one per epilogue warpgroup) keep
// the tensor cores fed.  Because a single thread issues every product, the weight-gradient
// products of all tiles accumulate into one set of TMEM accumulators (products from one thread
// execute in order), which is what leaves TMEM room for four tiles.  Shared memory per tile is the
// input tile, one buffer per hidden layer and the output delta: each hidden layer's activations
// are overwritten in place by its delta once the products that read them have completed.
//
// Stages of one tile (one product each, weight-gradient products riding along on the backward):
//   0            acc = X W_0^T                               -> H_0 = relu(acc)
//   h < NH       acc = H_{h-1} W_h^T                         -> H_h = relu(acc)
//   NH           acc = H_{NH-1} W_out^T                      -> dY (loss) in registers, DY tile
//   NH+1         dW_out^T += H_{NH-1}^T DY; acc = DY W_out   -> dH_{NH-1} = acc * [H_{NH-1} > 0], in place
//   NH+1+j       dW_h += dH_h^T H_{h-1};    acc = dH_h W_h   -> dH_{h-1} = acc * [H_{h-1} > 0], in place
//   2 NH + 1     dW_0 += dH_0^T X;          acc = dH_0 W_0   -> dX (the input gradient)
// Barriers per tile slot: ready (one epilogue thread arrives, after a named barrier of the slot's
// 128 threads, once the stage's operands are in shared memory and the previous accumulator has been
// read) and full (the MMA thread's commit);
// every wait is bounded and a shared abort word lets all warps unwind together.
template <int N_IN, int NH>
struct WsSmem {
  static constexpr int X = 0;                                 // per slot: [128][N_IN]
  static constexpr int H = X + kM * N_IN * 2;                 // NH x [128][64], activations then deltas
  static constexpr int DY = H + NH * kM * kW * 2;             // [128][16]
  static constexpr int SLOT = DY + kM * 16 * 2;
  static constexpr int WBYTES = 2 * (kW * N_IN * 2) + 2 * ((NH - 1) * kW * kW * 2) + 2 * (16 * kW * 2);
  static constexpr int FIT = (227 * 1024 - WBYTES) / SLOT;
  static constexpr int SLOTS = FIT >= 4 ? 4 : FIT;
  static constexpr int W0 = SLOTS * SLOT;                     // weights, as TcSmem
  static constexpr int WH = W0 + kW * N_IN * 2;
  static constexpr int WO = WH + (NH - 1) * kW * kW * 2;
  static constexpr int WOT = WO + 16 * kW * 2;
  static constexpr int WHT = WOT + kW * 16 * 2;
  static constexpr int W0T = WHT + (NH - 1) * kW * kW * 2;
  static constexpr int END = W0T + N_IN * kW * 2;
  static constexpr int THREADS = SLOTS * 128 + 32;
  static constexpr int STAGES = 2 * NH + 2;
  // TMEM: one 64-column accumulator per slot, then dW_out^T (16), dW_1..dW_{NH-1} (64 each), dW_0
  static constexpr int C_OUT = SLOTS * 64;
  static constexpr int C_HID = C_OUT + 16;
  static constexpr int C_FIRST = C_HID + 64 * (NH - 1);
  static constexpr int COLS = C_FIRST + N_IN;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(mbar)) : "memory");
}

// non-blocking probe: has the phase with this parity completed?
__device__ __forceinline__ bool mbar_test(uint64_t* mbar, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(tc::smem_u32(mbar)), "r"(parity) : "memory");
  return done != 0;
}

// bounded wait (try_wait lets the hardware suspend the thread until the phase completes or a short
// time limit passes, instead of spinning on shared memory) that also gives up once another thread
// has raised the CTA's abort word, checked every 64 polls
__device__ __forceinline__ bool mbar_wait_abort(uint64_t* mbar, uint32_t parity, volatile int* abort_word) {
  for (uint32_t it = 0; it < kWaitPolls; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(tc::smem_u32(mbar)), "r"(parity) : "memory");
    if (done) return true;
    if ((it & 63u) == 63u && *abort_word) return false;
  }
  *abort_word = 1;
  return false;
}

template <typename T, int N_IN, int NH, int MODE>
__global__ void __launch_bounds__(WsSmem<N_IN, NH>::THREADS, 1)
mlp_train_ws_kernel(const T* __restrict__ W, const T* __restrict__ in, int64_t P, int n_out,
                    const float* __restrict__ dout, const float* __restrict__ target, float loss_scale,
                    float inv_count, float* __restrict__ din, int din_group, float* __restrict__ ws,
                    int64_t n_params) {
  using S = WsSmem<N_IN, NH>;
  constexpr int SL = S::SLOTS;
  constexpr bool BF16 = std::is_same<T, __nv_bfloat16>::value;
  static_assert(SL >= 1 && S::END <= 227 * 1024 && S::COLS <= 512, "shared memory / TMEM plan");
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t ready[SL], full[SL], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_word;
  __shared__ int n_done_tiles;
  __shared__ float sq_part[SL * 4];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n_tiles = (P + kM - 1) / kM;
  const int64_t stride = (int64_t)gridDim.x * SL;
  const float inv_scale = 1.f / loss_scale;

  load_weights_cm<T, N_IN, NH, S>(W, n_out, sm);
  if (tid == 0) {
    for (int s = 0; s < SL; ++s) {
      tc::mbar_init(&ready[s], 1);
      tc::mbar_init(&full[s], 1);
    }
    tc::mbar_init(&done, 1);
    abort_word = 0;
    n_done_tiles = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  volatile int* abort_p = &abort_word;
  float sq = 0.f;

  if (warp == 4 * SL) {
    // ---------------- the MMA-issuing warp (one thread)
    if (lane == 0) {
      int st[SL], rnd[SL];
      int64_t tile[SL];
      uint32_t rph[SL];
      int active = 0;
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        tile[s] = (int64_t)blockIdx.x * SL + s;
        st[s] = 0;
        rnd[s] = 0;
        rph[s] = 0;
        active += tile[s] < n_tiles;
      }
      // The weight-gradient stages (NH + 1 .. 2 NH + 1) of this CTA's tiles are issued in tile order
      // (ordinal rnd * SL + slot), one turn counter per stage, so that every TMEM accumulator sums
      // its tiles in the same order on every run: the partials, and dweights, are deterministic.
      // A tile only ever waits for lower ordinals, so the turns cannot deadlock.
      // (every per-slot and per-stage array is indexed only inside fully unrolled loops, so the
      // issuing thread's state stays in registers)
      int turn[NH + 1];
#pragma unroll
      for (int j = 0; j <= NH; ++j) turn[j] = 0;
      bool first_out = true, first_0 = true;
      uint32_t first_h = (1u << NH) - 1u;
      constexpr uint32_t kH = (kW / 8) * 128, kDY = (16 / 8) * 128, kX = (N_IN / 8) * 128;
      auto wgrad = [&](uint32_t d, const unsigned char* A, uint32_t kA, const unsigned char* B, uint32_t kB, int N,
                       bool first) {
        const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B), id = tc::idesc_f16_mn(64, N, BF16);
#pragma unroll
        for (int ks = 0; ks < kM / 16; ++ks)
          tc::mma_f16(d, tc::smem_desc(a0 + ks * 2 * kA, kA, 128u), tc::smem_desc(b0 + ks * 2 * kB, kB, 128u), id,
                      !(first && ks == 0));
      };
      uint32_t idle = 0;
      while (active > 0) {
        bool progressed = false;
#pragma unroll
        for (int s = 0; s < SL; ++s) {
          if (tile[s] >= n_tiles) continue;
          const int ord = rnd[s] * SL + s;
          const int j = st[s] - NH - 1;                // weight-gradient stage, or negative
          int tj = ord;
#pragma unroll
          for (int jj = 0; jj <= NH; ++jj)
            if (jj == j) tj = turn[jj];
          if (tj != ord) continue;
          if (!mbar_test(&ready[s], rph[s])) continue;
          rph[s] ^= 1u;
#pragma unroll
          for (int jj = 0; jj <= NH; ++jj)
            if (jj == j) turn[jj] = ord + 1;
          tc::fence_after_sync();
          unsigned char* b = sm + s * S::SLOT;
          const uint32_t acc = tmem + 64u * (uint32_t)s;
          const int k = st[s];
          if (k == 0) {
            issue_gemm(acc, b + S::X, sm + S::W0, N_IN, tc::idesc_f16(kM, kW, BF16));
          } else if (k < NH) {
            issue_gemm(acc, b + S::H + (k - 1) * kM * kW * 2, sm + S::WH + (k - 1) * kW * kW * 2, kW,
                       tc::idesc_f16(kM, kW, BF16));
          } else if (k == NH) {
            issue_gemm(acc, b + S::H + (NH - 1) * kM * kW * 2, sm + S::WO, kW, tc::idesc_f16(kM, 16, BF16));
          } else if (k == NH + 1) {
            wgrad(tmem + S::C_OUT, b + S::H + (NH - 1) * kM * kW * 2, kH, b + S::DY, kDY, 16, first_out);
            first_out = false;
            issue_gemm(acc, b + S::DY, sm + S::WOT, 16, tc::idesc_f16(kM, kW, BF16));
          } else if (k < 2 * NH + 1) {
            const int h = 2 * NH + 1 - k;              // delta of layer h known; dW_h, then dH_{h-1}
            wgrad(tmem + S::C_HID + 64u * (uint32_t)(h - 1), b + S::H + h * kM * kW * 2, kH,
                  b + S::H + (h - 1) * kM * kW * 2, kH, kW, (first_h >> h) & 1u);
            first_h &= ~(1u << h);
            issue_gemm(acc, b + S::H + h * kM * kW * 2, sm + S::WHT + (h - 1) * kW * kW * 2, kW,
                       tc::idesc_f16(kM, kW, BF16));
          } else {
            wgrad(tmem + S::C_FIRST, b + S::H, kH, b + S::X, kX, N_IN, first_0);
            first_0 = false;
            issue_gemm(acc, b + S::H, sm + S::W0T, kW, tc::idesc_f16(kM, N_IN, BF16));
          }
          tc::commit(&full[s]);
          if (++st[s] == S::STAGES) {
            st[s] = 0;
            ++rnd[s];
            tile[s] += stride;
            active -= tile[s] >= n_tiles;
          }
          progressed = true;
        }
        if (progressed) {
          idle = 0;
        } else if (++idle > kWaitPolls || *abort_p) {
          *abort_p = 1;
          break;
        }
      }
      tc::commit(&done);                               // arrives once every product has completed
      if (!tc::mbar_wait(&done, 0, kWaitPolls)) *abort_p = 1;   // TMEM is freed only after this
    }
    __syncwarp();
  } else {
    // ---------------- epilogue warpgroup `slot`: warp q reads TMEM lanes 32 q .. 32 q + 31
    const int slot = warp >> 2, q = warp & 3, r = q * 32 + lane;
    unsigned char* b = sm + slot * S::SLOT;
    const uint32_t lane_addr = tmem + 64u * (uint32_t)slot + ((uint32_t)(q * 32) << 16);
    uint32_t fph = 0;
    bool failed = false;
    // the warpgroup's writes are made visible to the tensor cores (proxy fence), its TMEM reads are
    // ordered before the barrier, and one thread arrives once all 128 have passed the named barrier
    auto operands_ready = [&]() {
      tc::fence_smem_async();
      tc::fence_before_sync();
      group_sync(1 + slot);
      if (r == 0) mbar_arrive(&ready[slot]);
    };
    // every thread of the warpgroup takes the same branch (group_any is a barrier of the 128), so
    // no thread can be left waiting at the warpgroup's named barrier for one that gave up
    auto acc_full = [&]() -> bool {
      const bool ok = mbar_wait_abort(&full[slot], fph, abort_p);
      fph ^= 1u;
      tc::fence_after_sync();
      return !group_any(1 + slot, !ok);
    };
    constexpr int kPieces = N_IN / 8;
    uint4 pf[kPieces];
    auto prefetch = [&](int64_t t) {
#pragma unroll
      for (int j = 0; j < kPieces; ++j) {
        const int i = r + 128 * j, rr = i / (N_IN / 8), c = (i % (N_IN / 8)) * 8;
        const int64_t row = t * kM + rr;
        pf[j] = (t < n_tiles && row < P) ? __ldg(reinterpret_cast<const uint4*>(in + row * N_IN + c))
                                         : make_uint4(0, 0, 0, 0);
      }
    };
    int tiles_here = 0;
    prefetch((int64_t)blockIdx.x * SL + slot);
    for (int64_t tile = (int64_t)blockIdx.x * SL + slot; tile < n_tiles && !failed; tile += stride) {
      const int64_t row0 = tile * kM;
#pragma unroll
      for (int j = 0; j < kPieces; ++j) {
        const int i = r + 128 * j, rr = i / (N_IN / 8), c = (i % (N_IN / 8)) * 8;
        *reinterpret_cast<uint4*>(b + S::X + tc::cm_offset(rr, c, N_IN)) = pf[j];
      }
      operands_ready();                                // stage 0: the input tile
      prefetch(tile + stride);
      float yin[16];
      {
        const int64_t row = row0 + r;
        const float* src = MODE == 0 ? dout : target;
#pragma unroll
        for (int o = 0; o < 16; ++o) yin[o] = (row < P && o < n_out) ? __ldg(src + row * n_out + o) : 0.f;
      }
      // ---- forward
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        if (!acc_full()) { failed = true; break; }
#pragma unroll
        for (int c0 = 0; c0 < kW; c0 += 32) {
          float v[32];
          tc::tmem_ld32(lane_addr + (uint32_t)c0, v);
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            float u[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) u[j] = fmaxf(v[16 * half + j], 0.f);
            store16<T>(b + S::H + h * kM * kW * 2, r, c0 + 16 * half, kW, u);
          }
        }
        operands_ready();
      }
      if (failed || !acc_full()) { failed = true; break; }
      // ---- output delta
      {
        float v[16];
        tc::tmem_ld16(lane_addr, v);
        const int64_t row = row0 + r;
#pragma unroll
        for (int o = 0; o < 16; ++o) {
          float dyo = 0.f;
          if (row < P && o < n_out) {
            if (MODE == 0) {
              dyo = yin[o] * loss_scale;
            } else {
              const float res = v[o] - yin[o];
              sq = fmaf(res, res, sq);
              dyo = res * inv_count * loss_scale;
            }
          }
          v[o] = dyo;
        }
        store16<T>(b + S::DY, r, 0, 16, v);
      }
      operands_ready();
      // ---- hidden deltas, top layer down, each written over its layer's activations (16 columns
      // at a time: fewer live registers than 32)
#pragma unroll
      for (int h = NH - 1; h >= 0; --h) {
        if (!acc_full()) { failed = true; break; }
#pragma unroll
        for (int c0 = 0; c0 < kW; c0 += 16) {
          float v[16], a[16];
          tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
          load16<T>(b + S::H + h * kM * kW * 2, r, c0, kW, a);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) v[jj] = a[jj] > 0.f ? v[jj] : 0.f;
          store16<T>(b + S::H + h * kM * kW * 2, r, c0, kW, v);
        }
        operands_ready();
      }
      if (failed || !acc_full()) { failed = true; break; }
      // ---- input gradient (the slot's buffers are free: every product of the tile has completed)
      if (din && din_group == 0 && kM * (N_IN + 4) * 4 <= NH * kM * kW * 2) {
        constexpr int LD = N_IN + 4;
        float* stg = reinterpret_cast<float*>(b + S::H);
#pragma unroll
        for (int c0 = 0; c0 < N_IN; c0 += 16) {
          float v[16];
          tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(stg + r * LD + c0 + j) =
                make_float4(v[j] * inv_scale, v[j + 1] * inv_scale, v[j + 2] * inv_scale, v[j + 3] * inv_scale);
        }
        group_sync(1 + slot);
        for (int i = r; i < kM * (N_IN / 4); i += 128) {
          const int rr = i / (N_IN / 4), c4 = i % (N_IN / 4);
          if (row0 + rr < P)
            *reinterpret_cast<float4*>(din + (row0 + rr) * N_IN + c4 * 4) =
                *reinterpret_cast<const float4*>(stg + rr * LD + c4 * 4);
        }
        group_sync(1 + slot);                          // staging read before the next tile's H_0
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
              if (din_group == 0) {
                *reinterpret_cast<float2*>(din + row * N_IN + col) = val;
              } else if (din_group == 1) {
                din[(int64_t)col * P + row] = val.x;
                din[(int64_t)(col + 1) * P + row] = val.y;
              } else {
                *reinterpret_cast<float2*>(din + ((int64_t)(col / din_group) * P + row) * din_group +
                                           col % din_group) = val;
              }
            }
          }
        }
      }
      ++tiles_here;
    }
    if (failed) *abort_p = 1;
    if (q == 0 && lane == 0 && tiles_here > 0) atomicAdd(&n_done_tiles, tiles_here);
    if (MODE == 1) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) sq_part[warp] = sq;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool failed_cta = abort_word != 0;
  if (failed_cta && tid == 0) atomicExch(&g_tc_error, 1);
  // ---- this CTA's partials: the weight-gradient accumulators (row m of an M = 64 accumulator in
  // TMEM lane 32 (m / 16) + m % 16, read by warps 0-3 from their lanes 0-15); zeros without a tile
  float* wsb = ws + (int64_t)blockIdx.x * n_params;
  const bool any = n_done_tiles > 0 && !failed_cta;
  if (warp < 4) {
    const int q = warp, off_h = kW * N_IN, off_o = off_h + (NH - 1) * kW * kW;
    const int m = 16 * q + lane;
    const uint32_t la = (uint32_t)(q * 32) << 16;
    float v[16];
    tc::tmem_ld16(tmem + S::C_OUT + la, v);
    if (lane < 16)
#pragma unroll
      for (int o = 0; o < 16; ++o)
        if (o < n_out) wsb[off_o + o * kW + m] = any ? v[o] : 0.f;
#pragma unroll
    for (int h = 1; h < NH; ++h)
#pragma unroll
      for (int c0 = 0; c0 < kW; c0 += 16) {
        tc::tmem_ld16(tmem + S::C_HID + 64u * (h - 1) + la + (uint32_t)c0, v);
        if (lane < 16)
#pragma unroll
          for (int j = 0; j < 16; ++j) wsb[off_h + (h - 1) * kW * kW + m * kW + c0 + j] = any ? v[j] : 0.f;
      }
#pragma unroll
    for (int c0 = 0; c0 < N_IN; c0 += 16) {
      tc::tmem_ld16(tmem + S::C_FIRST + la + (uint32_t)c0, v);
      if (lane < 16)
#pragma unroll
        for (int j = 0; j < 16; ++j) wsb[m * N_IN + c0 + j] = any ? v[j] : 0.f;
    }
  }
  if (MODE == 1 && tid == 0) {
    float s = 0.f;
    for (int w = 0; w < 4 * SL; ++w) s += sq_part[w];
    ws[(int64_t)gridDim.x * n_params + blockIdx.x] = s;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 512);
  }
}

}  // namespace
}  // namespace sxe

namespace sxe {
namespace {

template <typename T, int N_IN, int NH, int MODE>
int tc_ctas_per_sm() {
  return kernel_ctas_per_sm((const void*)mlp_train_tc_kernel<T, N_IN, NH, MODE>, kThreads, TcSmem<N_IN, NH>::END);
}

// Two-tile kernel: one CTA per SM, two partial rows per CTA (the workspace holds `grid` rows).
constexpr int kMaxDynSmem = 227 * 1024;

template <typename T, int N_IN, int NH>
sxe_status tc2_launch(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                      float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid, int sms,
                      cudaStream_t s, int64_t lc) {
  // at least 116 KB, so that one CTA (holding all 512 TMEM columns) runs per SM
  constexpr int bytes = Tc2Smem<N_IN, NH>::END > 116 * 1024 ? Tc2Smem<N_IN, NH>::END : 116 * 1024;
  const int64_t n_params = sxe_mlp_n_params(d);
  const int64_t n_tiles = (P + kM - 1) / kM;
  const int g2 = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)sms, (int64_t)(grid / 2), (n_tiles + 1) / 2}));
  kernel_ctas_per_sm((const void*)mlp_train_tc2_kernel<T, N_IN, NH, 0, true>, kThreads, bytes);
  kernel_ctas_per_sm((const void*)mlp_train_tc2_kernel<T, N_IN, NH, 1, true>, kThreads, bytes);
  if (target)
    mlp_train_tc2_kernel<T, N_IN, NH, 1, true><<<g2, kThreads, bytes, s>>>((const T*)W, (const T*)in, P, d->n_out,
                                                                          dout, target, ls, l2_inv_count(lc, d->n_out),
                                                                          din, dg, ws, n_params);
  else
    mlp_train_tc2_kernel<T, N_IN, NH, 0, true><<<g2, kThreads, bytes, s>>>((const T*)W, (const T*)in, P, d->n_out,
                                                                          dout, target, ls, l2_inv_count(lc, d->n_out),
                                                                          din, dg, ws, n_params);
  sxe_status st = check_launch("mlp_train_tc2");
  if (st != SXE_OK) return st;
  return launch_mlp_reduce(ws, 2 * g2, n_params, 1.f / ls, dW, target ? sq : nullptr, s);
}

// Warp-specialised kernel: one CTA per SM (its shared-memory plan takes the SM), SLOTS tiles per
// CTA in flight; one partial row per CTA (the workspace holds `grid` rows).
template <typename T, int N_IN, int NH>
sxe_status ws_launch(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                     float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid,
                     cudaStream_t s, int64_t lc) {
  using S = WsSmem<N_IN, NH>;
  const int64_t n_params = sxe_mlp_n_params(d);
  const int64_t n_tiles = (P + kM - 1) / kM;
  const int g = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)device_sm_count(), (int64_t)grid, (n_tiles + S::SLOTS - 1) / S::SLOTS}));
  const float ic = l2_inv_count(lc, d->n_out);
  if (target) {
    kernel_ctas_per_sm((const void*)mlp_train_ws_kernel<T, N_IN, NH, 1>, S::THREADS, S::END);
    mlp_train_ws_kernel<T, N_IN, NH, 1><<<g, S::THREADS, S::END, s>>>((const T*)W, (const T*)in, P, d->n_out, dout,
                                                                      target, ls, ic, din, dg, ws, n_params);
  } else {
    kernel_ctas_per_sm((const void*)mlp_train_ws_kernel<T, N_IN, NH, 0>, S::THREADS, S::END);
    mlp_train_ws_kernel<T, N_IN, NH, 0><<<g, S::THREADS, S::END, s>>>((const T*)W, (const T*)in, P, d->n_out, dout,
                                                                      target, ls, ic, din, dg, ws, n_params);
  }
  sxe_status st = check_launch("mlp_train_ws");
  if (st != SXE_OK) return st;
  return launch_mlp_reduce(ws, g, n_params, 1.f / ls, dW, target ? sq : nullptr, s);
}

template <typename T, int N_IN>
sxe_status ws_nh(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                 float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid, cudaStream_t s, int64_t lc) {
  switch (d->n_hidden) {
    case 1: return ws_launch<T, N_IN, 1>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    case 2: return ws_launch<T, N_IN, 2>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    default: return ws_launch<T, N_IN, 3>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
  }
}

template <typename T>
sxe_status ws_in(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                 float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid, cudaStream_t s, int64_t lc) {
  switch (d->n_in) {
    case 16: return ws_nh<T, 16>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    case 32: return ws_nh<T, 32>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    default: return ws_nh<T, 64>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
  }
}

template <typename T, int N_IN, int NH>
sxe_status tc_launch(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                     float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid, cudaStream_t s,
                     int64_t lc) {
  const int bytes = TcSmem<N_IN, NH>::END;
  const int64_t n_params = sxe_mlp_n_params(d);
  const int sms = device_sm_count();
  if constexpr (Tc2Smem<N_IN, NH>::END <= kMaxDynSmem) {
    if (grid >= 2) return tc2_launch<T, N_IN, NH>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, sms, s, lc);
  }
  if (target) {
    grid = std::min(grid, sms * tc_ctas_per_sm<T, N_IN, NH, 1>());
    mlp_train_tc_kernel<T, N_IN, NH, 1><<<grid, kThreads, bytes, s>>>((const T*)W, (const T*)in, P, d->n_out, dout,
                                                                     target, ls, l2_inv_count(lc, d->n_out), din, dg, ws, n_params);
  } else {
    grid = std::min(grid, sms * tc_ctas_per_sm<T, N_IN, NH, 0>());
    mlp_train_tc_kernel<T, N_IN, NH, 0><<<grid, kThreads, bytes, s>>>((const T*)W, (const T*)in, P, d->n_out, dout,
                                                                     target, ls, l2_inv_count(lc, d->n_out), din, dg, ws, n_params);
  }
  sxe_status st = check_launch("mlp_train_tc");
  if (st != SXE_OK) return st;
  return launch_mlp_reduce(ws, grid, n_params, 1.f / ls, dW, target ? sq : nullptr, s);
}

template <typename T, int N_IN>
sxe_status tc_nh(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                 float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid, cudaStream_t s, int64_t lc) {
  switch (d->n_hidden) {
    case 1: return tc_launch<T, N_IN, 1>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    case 2: return tc_launch<T, N_IN, 2>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    default: return tc_launch<T, N_IN, 3>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
  }
}

template <typename T>
sxe_status tc_in(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, const float* target,
                 float ls, int64_t P, float* din, int dg, float* dW, float* sq, float* ws, int grid, cudaStream_t s, int64_t lc) {
  switch (d->n_in) {
    case 16: return tc_nh<T, 16>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    case 32: return tc_nh<T, 32>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
    default: return tc_nh<T, 64>(d, W, in, dout, target, ls, P, din, dg, dW, sq, ws, grid, s, lc);
  }
}

}  // namespace

sxe_status launch_mlp_bwd_tc(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                             const float* target, float loss_scale, int64_t P, float* din, float* dW, float* sq_sum,
                             float* ws, int grid, cudaStream_t s, int din_group, int64_t lc) {
  return d->dtype == SXE_F16
             ? tc_in<__half>(d, W, in, dout, target, loss_scale, P, din, din_group, dW, sq_sum, ws, grid, s, lc)
             : tc_in<__nv_bfloat16>(d, W, in, dout, target, loss_scale, P, din, din_group, dW, sq_sum, ws, grid, s, lc);
}

sxe_status launch_mlp_bwd_ws(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                             const float* target, float loss_scale, int64_t P, float* din, float* dW, float* sq_sum,
                             float* ws, int grid, cudaStream_t s, int din_group, int64_t lc) {
  return d->dtype == SXE_F16
             ? ws_in<__half>(d, W, in, dout, target, loss_scale, P, din, din_group, dW, sq_sum, ws, grid, s, lc)
             : ws_in<__nv_bfloat16>(d, W, in, dout, target, loss_scale, P, din, din_group, dW, sq_sum, ws, grid, s, lc);
}

// Whether the two-tile tcgen05 kernel runs this network (its shared-memory plan fits and the
// workspace holds at least two partial rows); the automatic kernel choice prefers it then.
bool mlp_tc2_applies(const sxe_mlp_desc* d, int grid) {
  if (grid < 2) return false;
  auto fits = [](int n_in, int nh) {
    switch (n_in * 4 + nh) {
      case 16 * 4 + 1: return Tc2Smem<16, 1>::END <= kMaxDynSmem;
      case 16 * 4 + 2: return Tc2Smem<16, 2>::END <= kMaxDynSmem;
      case 16 * 4 + 3: return Tc2Smem<16, 3>::END <= kMaxDynSmem;
      case 32 * 4 + 1: return Tc2Smem<32, 1>::END <= kMaxDynSmem;
      case 32 * 4 + 2: return Tc2Smem<32, 2>::END <= kMaxDynSmem;
      case 32 * 4 + 3: return Tc2Smem<32, 3>::END <= kMaxDynSmem;
      case 64 * 4 + 1: return Tc2Smem<64, 1>::END <= kMaxDynSmem;
      case 64 * 4 + 2: return Tc2Smem<64, 2>::END <= kMaxDynSmem;
      default: return Tc2Smem<64, 3>::END <= kMaxDynSmem;
    }
  };
  return fits(d->n_in, d->n_hidden);
}

int* tc_error_word() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_tc_error) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<int*>(p);
}

sxe_status read_tc_error(int32_t* flag, bool clear) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int));
  if (e == cudaSuccess && clear) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
  }
  if (e != cudaSuccess) return set_error(SXE_ECUDA, "device_error: %s", cudaGetErrorString(e));
  *flag = v;
  return SXE_OK;
}

}  // namespace sxe
