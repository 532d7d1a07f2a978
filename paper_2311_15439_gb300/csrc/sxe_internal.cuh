// Internal declarations shared by the CUDA translation units of libsimplexenc.
//
// The lattice arithmetic here is the GPU side of the simplex-grid hash encoding
// (Wen & Yang, arXiv 2311.15439): scale + skew (Eq. 2, Sec. 5.1), simplicial
// subdivision by ranking the fractional parts (Sec. 4.2, Remark 2), barycentric
// weights (Sec. 4.3) and the vertex hash (Sec. 5 a); plus the 2^d grid corners of
// the comparator (Algorithm 1).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "simplexenc.h"

namespace sxe {

// ---------------------------------------------------------------------------
// host-side handle
// ---------------------------------------------------------------------------
struct EncParams {
  int32_t n_levels;
  int32_t log2_T;
  int32_t out_dtype;
  float skew_F;                    // F_n of Eq. 2 rounded to binary32 (simplex only)
  float scale[SXE_MAX_LEVELS];     // per-level input multiplier (binary32)
  uint32_t width[SXE_MAX_LEVELS];  // box width B of a directly indexed level, 0 = hashed
};

}  // namespace sxe

struct sxe_encoder {
  sxe_encoding_desc desc;
  int32_t level_res[SXE_MAX_LEVELS];
  uint32_t box_width[SXE_MAX_LEVELS];   // lattice coordinates per axis of [0,1]^d at each level
  sxe::EncParams prm;
  int32_t bwd_aggregate = 0;            // backward: warp-level sum of colliding terms (coherent batches)
};

namespace sxe {

// error reporting (defined in api.cu)
sxe_status set_error(sxe_status st, const char* fmt, ...);
sxe_status check_launch(const char* what);

// Launch set-up of the current device, cached per device (defined in api.cu): its SM count, and
// for a kernel the resident CTAs per SM at `threads` threads and `smem_bytes` of dynamic shared
// memory, after raising the kernel's dynamic shared-memory limit to `smem_bytes` on that device.
int device_sm_count();
int kernel_ctas_per_sm(const void* kernel, int threads, int smem_bytes);
// 2 / (P n_out), the factor of the L2 loss's gradient dy = 2 (y - t) / (P n_out), rounded on the
// host so that no kernel needs FP64 to form it exactly (P n_out exceeds 2^24).
inline float l2_inv_count(int64_t P, int n_out) { return 2.f / (float)((double)P * n_out); }
// Shape and dtype check of a network description, shared by every network entry point.
sxe_status check_mlp(const char* fn, const sxe_mlp_desc* d);

// launchers (defined in encode.cu / mlp.cu / optim.cu); arguments already validated
sxe_status launch_encode_fwd(const sxe_encoder* enc, const float* x, int64_t P, const void* tables,
                             void* out, cudaStream_t s, int64_t table_stride = 0);
// level_end < 0 means n_levels; only levels [level_begin, level_end) are accumulated
sxe_status launch_encode_bwd(const sxe_encoder* enc, const float* x, int64_t P, const float* dout,
                             float* grad, int64_t grad_stride, uint32_t* touched, cudaStream_t s,
                             int level_begin = 0, int level_end = -1);
int encode_bwd_launches(const sxe_encoder* enc, int64_t P, int level_begin = 0, int level_end = -1);
int encode_bwd_coarse_levels(const sxe_encoder* enc, int64_t P);
sxe_status launch_adam_advance(const sxe_adam_desc* a, int64_t* t, float* corrections, cudaStream_t s);
sxe_status launch_encode_plain(const sxe_encoder* enc, bool backward, const float* x, int64_t P, const float* a,
                               float* b, cudaStream_t s);
sxe_status launch_encode_vertices(const sxe_encoder* enc, const float* x, int64_t P, uint32_t* slots,
                                  float* weights, cudaStream_t s);
sxe_status launch_encode_bwd_input(const sxe_encoder* enc, const float* x, int64_t P, const void* tables,
                                   const float* dout, float* dx, cudaStream_t s);
sxe_status launch_vr_samples(const float* o, const float* d, const float* tn, const float* tf, int64_t R, int S,
                             float* x, float* delta, cudaStream_t s);
sxe_status launch_vr_field(const float* dens, const float* dirs, int64_t R, int S, int dtype, float* sigma,
                           void* cin, cudaStream_t s);
sxe_status launch_vr_field_mlp(const sxe_mlp_desc* dd, const void* Wd, const sxe_mlp_desc* dc, const void* Wc,
                               const void* enc, const float* dirs, int64_t R, int S, float* sigma, float* logits,
                               cudaStream_t s);
sxe_status launch_vr_composite_bwd(const float* sigma, const float* logits, const float* delta, const float* color,
                                   const float* dcolor, int64_t R, int S, float* dsigma, float* dlogits,
                                   cudaStream_t s);
sxe_status launch_vr_field_bwd(const float* dcin, const float* dsigma, const float* sigma, const float* dens,
                               int64_t P, float* dv, cudaStream_t s);
sxe_status launch_vr_composite(const float* sigma, const float* logits, const float* delta, int64_t R, int S,
                               float* color, float* trans, float* weights, cudaStream_t s);

int mlp_grid_blocks(const sxe_mlp_desc* d, int64_t P);
sxe_status launch_mlp_fwd(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out,
                          void* act, cudaStream_t s);
sxe_status launch_mlp_bwd(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                          const float* target, float loss_scale, int64_t P, float* din, float* dW,
                          float* sq_sum, float* ws, int grid, cudaStream_t s, int din_group = 0);
sxe_status launch_mlp_bwd_tc(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                             const float* target, float loss_scale, int64_t P, float* din, float* dW,
                             float* sq_sum, float* ws, int grid, cudaStream_t s, int din_group);
bool mlp_tc2_applies(const sxe_mlp_desc* d, int grid);
sxe_status launch_mlp_reduce(const float* ws, int nb, int64_t n_params, float inv_scale, float* dW, float* sq_sum,
                             cudaStream_t s);
sxe_status read_tc_error(int32_t* flag, bool clear);
extern int g_mlp_kernel;
sxe_status launch_loss_l2(const float* y, const float* target, int64_t P, int32_t n_out, float* dy,
                          float* sq_sum, cudaStream_t s);
sxe_status launch_adam_dense(const sxe_adam_desc* a, int64_t t, int64_t n, float* p, float* m, float* v,
                             float* g, void* lowp, int32_t lowp_dtype, cudaStream_t s,
                             const float* corrections = nullptr);
sxe_status launch_adam_touched(const sxe_adam_desc* a, int64_t t, int64_t n_entries, int32_t F,
                               float* state, uint32_t* touched, void* lowp, int32_t lowp_dtype,
                               cudaStream_t s,
                               const float* corrections = nullptr);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Hash multipliers per axis: 1, 2654435761, 805459861 (the Instant-NGP spatial hash
// the paper's backbone uses) and, for axes 4 and 5, the smallest primes not below
// frac(sqrt(5)) * 2^32 and frac(sqrt(7)) * 2^32.
__host__ __device__ constexpr uint32_t hash_prime(int axis) {
  return axis == 0 ? 1u : axis == 1 ? 2654435761u : axis == 2 ? 805459861u
       : axis == 3 ? 1013904263u : 2773480771u;
}

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Store `n` binary32 values as dtype `dt` at element offset `off` of `base`.
__device__ __forceinline__ void store_as(void* base, int64_t off, int32_t dt, float v) {
  if (dt == SXE_F32) reinterpret_cast<float*>(base)[off] = v;
  else if (dt == SXE_F16) reinterpret_cast<__half*>(base)[off] = __float2half_rn(v);
  else reinterpret_cast<__nv_bfloat16*>(base)[off] = __float2bfloat16_rn(v);
}

// Raw aligned vector of B bytes.
template <int B> struct RawVec;
template <> struct RawVec<2> { using type = unsigned short; };
template <> struct RawVec<4> { using type = unsigned int; };
template <> struct RawVec<8> { using type = uint2; };
template <> struct RawVec<16> { using type = uint4; };

// Gather the F features of one table entry through the read-only path.
template <typename T, int F>
__device__ __forceinline__ void load_entry(const T* __restrict__ p, float (&o)[F]) {
  constexpr int B = F * (int)sizeof(T);
  if constexpr (B <= 16) {
    using V = typename RawVec<B>::type;
    union { V v; T t[F]; } u;
    u.v = __ldg(reinterpret_cast<const V*>(p));
#pragma unroll
    for (int f = 0; f < F; ++f) o[f] = to_f32(u.t[f]);
  } else {
    union { uint4 v[B / 16]; T t[F]; } u;
#pragma unroll
    for (int j = 0; j < B / 16; ++j) u.v[j] = __ldg(reinterpret_cast<const uint4*>(p) + j);
#pragma unroll
    for (int f = 0; f < F; ++f) o[f] = to_f32(u.t[f]);
  }
}

// Vector atomic add of F binary32 values (8/16-byte vector atomics on sm_90+).
template <int F>
__device__ __forceinline__ void atomic_add_entry(float* p, const float (&v)[F]) {
  if constexpr (F == 1) {
    atomicAdd(p, v[0]);
  } else if constexpr (F == 2) {
    atomicAdd(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
  } else {
#pragma unroll
    for (int j = 0; j < F / 4; ++j)
      atomicAdd(reinterpret_cast<float4*>(p) + j, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
  }
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba, Algorithm 1) on binary32 state
// ---------------------------------------------------------------------------
struct AdamConst {
  float lr, b1, b2, eps, c1, c2;  // c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
  int skip;
  const float* cdev;              // if set: c1, c2 are read from device memory (cdev[0], cdev[1])
};

// The constants a kernel uses: the bias corrections from device memory where the step count
// lives on the device (captured training loops), else the host-computed ones.
__device__ __forceinline__ AdamConst adam_resolve(const AdamConst& k) {
  AdamConst r = k;
  if (k.cdev) {
    r.c1 = __ldg(k.cdev);
    r.c2 = __ldg(k.cdev + 1);
  }
  return r;
}

inline AdamConst make_adam_const(const sxe_adam_desc* a, int64_t t) {
  AdamConst k;
  k.lr = a->lr; k.b1 = a->beta1; k.b2 = a->beta2; k.eps = a->eps;
  k.c1 = (float)(1.0 / (1.0 - pow((double)a->beta1, (double)t)));
  k.c2 = (float)(1.0 / (1.0 - pow((double)a->beta2, (double)t)));
  k.skip = a->skip_zero_grad;
  k.cdev = nullptr;
  return k;
}

// m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr m c1 / (sqrt(v c2) + eps)
__device__ __forceinline__ void adam_one(const AdamConst& k, float g, float& p, float& m, float& v) {
  m = fmaf(k.b1, m, (1.f - k.b1) * g);
  v = fmaf(k.b2, v, (1.f - k.b2) * g * g);
  const float mh = m * k.c1;
  const float vh = v * k.c2;
  p = p - k.lr * mh / (sqrtf(vh) + k.eps);
}

// Low-precision copy of F consecutive parameters in one store where the type allows.
template <int F>
__device__ __forceinline__ void store_lowp(void* base, int64_t e, int ldt, const float (&p)[F]) {
  if (F == 2 && ldt == SXE_F16) {
    reinterpret_cast<__half2*>(base)[e] = __floats2half2_rn(p[0], p[1]);
  } else if (F == 2 && ldt == SXE_BF16) {
    reinterpret_cast<__nv_bfloat162*>(base)[e] = __floats2bfloat162_rn(p[0], p[1]);
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f) store_as(base, e * F + f, ldt, p[f]);
  }
}

// Compare-exchange of a descending sort of (f, axis) with ties broken by the lower axis first,
// carrying each axis's hash step along.
__device__ __forceinline__ void sort_cx(float& fa, int& ia, uint32_t& da, float& fb, int& ib, uint32_t& db) {
  const bool sw = (fb > fa) || (fb == fa && ib < ia);
  const float f = sw ? fb : fa;
  const int i = sw ? ib : ia;
  const uint32_t d = sw ? db : da;
  fb = sw ? fa : fb; ib = sw ? ia : ib; db = sw ? da : db;
  fa = f; ia = i; da = d;
}

// Sorting networks (1, 3, 5 and 9 comparators for 2, 3, 4 and 5 keys).
template <int D>
__device__ __forceinline__ void sort_desc(float (&f)[D], int (&ix)[D], uint32_t (&dl)[D]) {
#define SXE_CX(a, b) sort_cx(f[a], ix[a], dl[a], f[b], ix[b], dl[b])
  if constexpr (D == 2) {
    SXE_CX(0, 1);
  } else if constexpr (D == 3) {
    SXE_CX(0, 1); SXE_CX(1, 2); SXE_CX(0, 1);
  } else if constexpr (D == 4) {
    SXE_CX(0, 1); SXE_CX(2, 3); SXE_CX(0, 2); SXE_CX(1, 3); SXE_CX(1, 2);
  } else {
    static_assert(D == 5, "d = 2..5");
    SXE_CX(0, 1); SXE_CX(3, 4); SXE_CX(2, 4); SXE_CX(2, 3); SXE_CX(0, 3);
    SXE_CX(0, 2); SXE_CX(1, 4); SXE_CX(1, 3); SXE_CX(1, 2);
  }
#undef SXE_CX
}

// ---------------------------------------------------------------------------
// Simplex lattice of one point at one level.
//   Sec. 5.1 + Eq. 2: p_i = x_i * s, sigma = sum_i p_i (left to right), t = F * sigma,
//   q_i = p_i + t; each operation rounded once (no contraction).
//   Sec. 4.2: c = floor(q), f = q - c (exact); the fractional parts are sorted in decreasing
//   order, ties lower axis first (a sorting network carrying the axis and its hash step).
//   Remark 2: vertex k = c + the unit vectors of the first k sorted axes; its slot is the base
//   vertex's hash updated by the hash steps of those axes.
//   Sec. 4.3: w_0 = 1 - s_0, w_k = s_{k-1} - s_k, w_d = s_{d-1} on the sorted s.
//   Sec. 5 (a): slot = XOR_i (uint32(v_i) * prime_i) mod T; on a directly indexed level
//   (width B > 0) slot = (sum_i uint32(v_i) * B^i) mod T instead.  rank_i is the position of
//   axis i in the sorted order.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void simplex_lattice(const float (&x)[D], float s, float skewF, uint32_t mask,
                                                uint32_t width, uint32_t (&slot)[D + 1], float (&w)[D + 1],
                                                int (&rank)[D], int (&cell)[D]) {
  float p[D];
#pragma unroll
  for (int i = 0; i < D; ++i) p[i] = __fmul_rn(x[i], s);
  float sigma = p[0];
#pragma unroll
  for (int i = 1; i < D; ++i) sigma = __fadd_rn(sigma, p[i]);
  const float t = __fmul_rn(skewF, sigma);
  float f[D];
  int ix[D];
  uint32_t dl[D];
  uint32_t h = 0, pw = 1u;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const float q = __fadd_rn(p[i], t);
    const float fl = floorf(q);
    f[i] = __fsub_rn(q, fl);
    cell[i] = __float2int_rz(fl);
    const uint32_t c = (uint32_t)cell[i];
    const uint32_t mult = width ? pw : hash_prime(i);
    pw *= width;
    const uint32_t h0 = c * mult;
    h = width ? h + h0 : h ^ h0;
    dl[i] = width ? mult : (h0 ^ (h0 + mult));          // hash step of moving +1 along axis i
    ix[i] = i;
  }
  sort_desc<D>(f, ix, dl);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    int r = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) r = ix[k] == i ? k : r;
    rank[i] = r;
  }
  w[0] = __fsub_rn(1.f, f[0]);
#pragma unroll
  for (int k = 1; k < D; ++k) w[k] = __fsub_rn(f[k - 1], f[k]);
  w[D] = f[D - 1];
  slot[0] = h & mask;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    h = width ? h + dl[k] : h ^ dl[k];
    slot[k + 1] = h & mask;
  }
}

template <int D>
__device__ __forceinline__ void simplex_lattice(const float (&x)[D], float s, float skewF, uint32_t mask,
                                                uint32_t width, uint32_t (&slot)[D + 1], float (&w)[D + 1],
                                                int (&rank)[D]) {
  int cell[D];
  simplex_lattice<D>(x, s, skewF, mask, width, slot, w, rank, cell);
}

template <int D>
__device__ __forceinline__ void simplex_lattice(const float (&x)[D], float s, float skewF, uint32_t mask,
                                                uint32_t width, uint32_t (&slot)[D + 1], float (&w)[D + 1]) {
  int rank[D];
  simplex_lattice<D>(x, s, skewF, mask, width, slot, w, rank);
}

// 2^D grid corners of one point at one level (Algorithm 1's multilinear weights):
// p_i = x_i * N (binary32), c = floor(p), f = p - c; corner b (axis 0 = most
// significant bit) has weight prod_i (b_i ? f_i : 1 - f_i), multiplied in axis order.
template <int D>
__device__ __forceinline__ void grid_lattice(const float (&x)[D], float N, uint32_t mask, uint32_t width,
                                             uint32_t (&slot)[1 << D], float (&w)[1 << D], float (&f)[D],
                                             int (&cell)[D]) {
  uint32_t h0[D], h1[D];
  uint32_t pw = 1u;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const float p = __fmul_rn(x[i], N);
    const float fl = floorf(p);
    f[i] = __fsub_rn(p, fl);
    cell[i] = __float2int_rz(fl);
    const uint32_t c = (uint32_t)cell[i];
    const uint32_t mult = width ? pw : hash_prime(i);
    pw *= width;
    h0[i] = c * mult;
    h1[i] = (c + 1u) * mult;
  }
#pragma unroll
  for (int b = 0; b < (1 << D); ++b) {
    float wt = 1.f;
    uint32_t h = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const bool bi = (b >> (D - 1 - i)) & 1;
      wt = __fmul_rn(wt, bi ? f[i] : __fsub_rn(1.f, f[i]));
      const uint32_t v = bi ? h1[i] : h0[i];
      h = width ? h + v : h ^ v;
    }
    w[b] = wt;
    slot[b] = h & mask;
  }
}

template <int D>
__device__ __forceinline__ void grid_lattice(const float (&x)[D], float N, uint32_t mask, uint32_t width,
                                             uint32_t (&slot)[1 << D], float (&w)[1 << D], float (&f)[D]) {
  int cell[D];
  grid_lattice<D>(x, N, mask, width, slot, w, f, cell);
}

template <int D>
__device__ __forceinline__ void grid_lattice(const float (&x)[D], float N, uint32_t mask, uint32_t width,
                                             uint32_t (&slot)[1 << D], float (&w)[1 << D]) {
  float f[D];
  grid_lattice<D>(x, N, mask, width, slot, w, f);
}

// Table slot of lattice vertex v under a level's rule (hash, or direct index for width > 0).
template <int D>
__device__ __forceinline__ uint32_t vertex_slot(const uint32_t (&v)[D], uint32_t width, uint32_t mask) {
  uint32_t h = 0, pw = 1u;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    h = width ? h + v[i] * pw : h ^ (v[i] * hash_prime(i));
    pw *= width;
  }
  return h & mask;
}

// Real spherical harmonics of degree 0..3 (l-major, m = -l..l) of a unit vector: the
// orthonormal real basis built from the complex harmonics with the Condon-Shortley phase.
__device__ __forceinline__ void sh16(float x, float y, float z, float (&h)[16]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  h[0] = 0.28209479177387814f;                       // 1/(2 sqrt(pi))
  h[1] = 0.4886025119029199f * y;                    // sqrt(3/(4 pi))
  h[2] = 0.4886025119029199f * z;
  h[3] = 0.4886025119029199f * x;
  h[4] = 1.0925484305920792f * x * y;                // sqrt(15/pi)/2
  h[5] = 1.0925484305920792f * y * z;
  h[6] = 0.31539156525252005f * (3.f * zz - 1.f);    // sqrt(5/pi)/4
  h[7] = 1.0925484305920792f * x * z;
  h[8] = 0.5462742152960396f * (xx - yy);            // sqrt(15/pi)/4
  h[9] = 0.5900435899266435f * y * (3.f * xx - yy);  // sqrt(35/(2 pi))/4
  h[10] = 2.890611442640554f * x * y * z;            // sqrt(105/pi)/2
  h[11] = 0.4570457994644658f * y * (5.f * zz - 1.f);  // sqrt(21/(2 pi))/4
  h[12] = 0.3731763325901154f * z * (5.f * zz - 3.f);  // sqrt(7/pi)/4
  h[13] = 0.4570457994644658f * x * (5.f * zz - 1.f);
  h[14] = 1.445305721320277f * z * (xx - yy);        // sqrt(105/pi)/4
  h[15] = 0.5900435899266435f * x * (xx - 3.f * yy);
}

// Density of the volumetric field from the density network's first output (Instant-NGP's
// exponential activation, argument clamped at 15).
__device__ __forceinline__ float vr_density(float v0) { return expf(fminf(v0, 15.f)); }

}  // namespace sxe
