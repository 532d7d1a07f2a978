// Internal declarations shared by the CUDA translation units of libsimplexenc: the encoder
// handle, error reporting, per-device launch set-up, the launchers of every kernel, the Adam
// helpers and the volumetric field's device helpers.  The lattice arithmetic of the encoding
// (Eq. 2, Sec. 4.2-4.3, Sec. 5 a, Algorithm 1) lives in lattice.cuh.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "simplexenc.h"
#include "lattice.cuh"

struct sxe_encoder {
  sxe_encoding_desc desc;
  int32_t level_res[SXE_MAX_LEVELS];
  uint32_t box_width[SXE_MAX_LEVELS];   // lattice coordinates per axis of [0,1]^d at each level
  sxe::EncParams prm;
  int32_t bwd_aggregate = 0;            // backward: warp-level sum of colliding terms (coherent batches)
  int32_t fwd_order = 0;                // forward work-item order, SXE_FWD_ORDER_*
};

namespace sxe {

// error reporting (defined in api.cu)
sxe_status set_error(sxe_status st, const char* fmt, ...);
sxe_status check_launch(const char* what);
// n_points == 0 in an entry point that overwrites *sq_sum with the batch's sum of squared
// residuals: that sum is zero (nothing is written when sq_sum is NULL)
sxe_status empty_batch_sq_sum(const char* fn, float* sq_sum, void* stream);

// Launch set-up of the current device, cached per device (defined in api.cu): its SM count, and
// for a kernel the resident CTAs per SM at `threads` threads and `smem_bytes` of dynamic shared
// memory, after raising the kernel's dynamic shared-memory limit to `smem_bytes` on that device.
int device_sm_count();
int64_t device_l2_bytes();   // L2 size of the current device (cached per device)
int kernel_ctas_per_sm(const void* kernel, int threads, int smem_bytes);
// 2 / (P n_out), the factor of the L2 loss's gradient dy = 2 (y - t) / (P n_out), rounded on the
// host so that no kernel needs FP64 to form it exactly (P n_out exceeds 2^24).
inline float l2_inv_count(int64_t P, int n_out) { return 2.f / (float)((double)P * n_out); }
// Shape and dtype check of a network description, shared by every network entry point.
sxe_status check_mlp(const char* fn, const sxe_mlp_desc* d);

// launchers (defined in encode.cu / mlp.cu / optim.cu); arguments already validated
sxe_status launch_encode_fwd(const sxe_encoder* enc, const float* x, int64_t P, const void* tables,
                             void* out, cudaStream_t s, int64_t table_stride = 0, uint32_t* touched = nullptr);
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
                               float* dens_out, void* color_in, cudaStream_t s);
sxe_status launch_vr_composite_bwd(const float* sigma, const float* logits, const float* delta, const float* color,
                                   const float* dcolor, int64_t R, int S, float* dsigma, float* dlogits,
                                   cudaStream_t s);
sxe_status launch_vr_field_bwd(const float* dcin, const float* dsigma, const float* sigma, const float* dens,
                               int64_t P, float* dv, cudaStream_t s);
sxe_status launch_vr_composite(const float* sigma, const float* logits, const float* delta, int64_t R, int S,
                               float* color, float* trans, float* weights, cudaStream_t s);

int mlp_grid_blocks(const sxe_mlp_desc* d, int64_t P);
// shared_gpu: the launch runs beside other streams' kernels (the automatic choice then avoids the
// persistent tcgen05 form, whose CTAs each hold a whole SM)
sxe_status launch_mlp_fwd(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out,
                          void* act, cudaStream_t s, bool shared_gpu = false);
sxe_status launch_mlp_bwd(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                          const float* target, float loss_scale, int64_t P, float* din, float* dW,
                          float* sq_sum, float* ws, int grid, cudaStream_t s, int din_group = 0,
                          int64_t loss_count = 0);   // 0: the L2 gradient is normalised by P
sxe_status launch_mlp_bwd_tc(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                             const float* target, float loss_scale, int64_t P, float* din, float* dW,
                             float* sq_sum, float* ws, int grid, cudaStream_t s, int din_group,
                             int64_t loss_count);
sxe_status launch_mlp_bwd_ws(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                             const float* target, float loss_scale, int64_t P, float* din, float* dW,
                             float* sq_sum, float* ws, int grid, cudaStream_t s, int din_group,
                             int64_t loss_count);
sxe_status launch_mlp_bwd_tc3(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                              const float* target, float loss_scale, int64_t P, float* din, float* dW,
                              float* sq_sum, float* ws, int grid, cudaStream_t s, int din_group,
                              int64_t loss_count);
bool mlp_tc2_applies(const sxe_mlp_desc* d, int grid);
bool mlp_tc3_applies(const sxe_mlp_desc* d);
sxe_status launch_selftest_wait(int timeout, int64_t limit_ns, cudaStream_t s);
sxe_status launch_mlp_fwd_tc3(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out,
                              void* act, cudaStream_t s);
sxe_status launch_vr_field_tc3(const sxe_mlp_desc* dd, const void* Wd, const sxe_mlp_desc* dc, const void* Wc,
                               const void* enc, const float* dirs, int64_t R, int S, float* sigma, float* logits,
                               float* dens_out, void* color_in, cudaStream_t s);   // colour n_out <= 8 (render_tc3.cu)
int* tc_error_word();   // device address of the tcgen05 kernels' error word (current device)
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
