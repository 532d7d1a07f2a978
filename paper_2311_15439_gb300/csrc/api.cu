// C ABI of libsimplexenc: argument validation, level constants, dispatch.
// Every entry point checks its arguments on the host, enqueues nothing on error and
// returns a status; the message of the last failure is kept per thread.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "sxe_internal.cuh"

namespace sxe {

static thread_local char g_err[512] = "";

sxe_status set_error(sxe_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

sxe_status check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SXE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return SXE_OK;
}

sxe_status empty_batch_sq_sum(const char* fn, float* sq_sum, void* stream) {
  if (!sq_sum) return SXE_OK;
  const cudaError_t e = cudaMemsetAsync(sq_sum, 0, sizeof(float), (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(SXE_ECUDA, "%s: %s", fn, cudaGetErrorString(e));
  return SXE_OK;
}

// Launch set-up cached per device: a kernel's dynamic shared-memory limit and its occupancy
// belong to the device that is current when they are set or queried, so a second device in the
// same process gets its own set-up instead of inheriting (or missing) the first one's.
static std::mutex g_setup_mu;
static std::map<int, int> g_sms;
static std::map<int, int64_t> g_l2;
static std::map<std::tuple<int, const void*, int, int>, int> g_ctas;
static std::map<std::pair<int, const void*>, int> g_smem_limit;   // dynamic shared-memory limit set per kernel

static int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  return dev;
}

int device_sm_count() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(g_setup_mu);
  auto it = g_sms.find(dev);
  if (it != g_sms.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 148;
  g_sms[dev] = n;
  return n;
}

int64_t device_l2_bytes() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(g_setup_mu);
  auto it = g_l2.find(dev);
  if (it != g_l2.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrL2CacheSize, dev) != cudaSuccess || n < 1) n = 96 << 20;
  g_l2[dev] = n;
  return n;
}

int kernel_ctas_per_sm(const void* kernel, int threads, int smem_bytes) {
  const int dev = current_device();
  const auto key = std::make_tuple(dev, kernel, threads, smem_bytes);
  std::lock_guard<std::mutex> lock(g_setup_mu);
  auto it = g_ctas.find(key);
  if (it != g_ctas.end()) return it->second;
  // the kernel's dynamic shared-memory limit only ever grows, so that a launch set up earlier
  // with a larger size keeps working after a smaller one is set up
  int& limit = g_smem_limit[std::make_pair(dev, kernel)];
  if (smem_bytes > limit) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    limit = smem_bytes;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, (size_t)smem_bytes) != cudaSuccess || n < 1)
    n = 1;
  cudaGetLastError();   // a refused attribute shows up at launch, not here
  g_ctas[key] = n;
  return n;
}

sxe_status check_mlp(const char* fn, const sxe_mlp_desc* d) {
  if (!d) return set_error(SXE_EINVAL, "%s: NULL desc", fn);
  if (d->width != 64) return set_error(SXE_EUNSUPPORTED, "%s: width=%d (only 64 is built)", fn, d->width);
  if (!(d->n_in == 16 || d->n_in == 32 || d->n_in == 64))
    return set_error(SXE_EUNSUPPORTED, "%s: n_in=%d not in {16,32,64}", fn, d->n_in);
  if (d->n_hidden < 1 || d->n_hidden > 3) return set_error(SXE_EUNSUPPORTED, "%s: n_hidden=%d not in 1..3", fn, d->n_hidden);
  if (d->n_out < 1 || d->n_out > 16) return set_error(SXE_EINVAL, "%s: n_out=%d not in 1..16", fn, d->n_out);
  if (d->dtype != SXE_F16 && d->dtype != SXE_BF16) return set_error(SXE_EINVAL, "%s: dtype must be F16 or BF16", fn);
  return SXE_OK;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }
static size_t dtype_size(int32_t dt) { return dt == SXE_F32 ? 4 : 2; }
static bool valid_dtype(int32_t dt) { return dt == SXE_F32 || dt == SXE_F16 || dt == SXE_BF16; }

}  // namespace sxe

using namespace sxe;

extern "C" {

const char* sxe_last_error(void) { return g_err; }

const char* sxe_version(void) { return "simplexenc 0.1 (sm_103a)"; }

sxe_status sxe_encoder_create(const sxe_encoding_desc* d, sxe_encoder** out) {
  g_err[0] = 0;
  if (!d || !out) return set_error(SXE_EINVAL, "encoder_create: NULL argument");
  if (d->d < 1 || d->d > 16) return set_error(SXE_EINVAL, "encoder_create: d=%d out of range", d->d);
  if (d->d < 2 || d->d > 5) return set_error(SXE_EUNSUPPORTED, "encoder_create: d=%d not built (2..5)", d->d);
  if (d->n_levels < 1 || d->n_levels > SXE_MAX_LEVELS)
    return set_error(SXE_EINVAL, "encoder_create: n_levels=%d out of 1..%d", d->n_levels, SXE_MAX_LEVELS);
  if (!(d->n_features == 1 || d->n_features == 2 || d->n_features == 4 || d->n_features == 8))
    return set_error(SXE_EINVAL, "encoder_create: n_features=%d not in {1,2,4,8}", d->n_features);
  if (d->log2_T < 4 || d->log2_T > 26) return set_error(SXE_EINVAL, "encoder_create: log2_T=%d out of 4..26", d->log2_T);
  if (!(d->base_res >= 1.0) || !(d->growth >= 1.0) || !std::isfinite(d->base_res) || !std::isfinite(d->growth))
    return set_error(SXE_EINVAL, "encoder_create: base_res and growth must be finite and >= 1");
  if (d->kind != SXE_SIMPLEX && d->kind != SXE_GRID) return set_error(SXE_EINVAL, "encoder_create: bad kind");
  if (d->res_mode != SXE_RES_RAW && d->res_mode != SXE_RES_EQUAL_MEM)
    return set_error(SXE_EINVAL, "encoder_create: bad res_mode");
  if (d->kind == SXE_GRID && d->res_mode != SXE_RES_RAW)
    return set_error(SXE_EINVAL, "encoder_create: res_mode applies to the simplex encoder only");
  if (!valid_dtype(d->table_dtype) || !valid_dtype(d->out_dtype))
    return set_error(SXE_EINVAL, "encoder_create: bad dtype");
  if (d->index_mode != SXE_INDEX_HASH && d->index_mode != SXE_INDEX_DENSE_COARSE)
    return set_error(SXE_EINVAL, "encoder_create: bad index_mode");
  const int64_t elems = ((int64_t)d->n_levels << d->log2_T) * d->n_features;
  if (elems >= ((int64_t)1 << 34)) return set_error(SXE_EINVAL, "encoder_create: tables too large");

  sxe_encoder* e = new (std::nothrow) sxe_encoder;
  if (!e) return set_error(SXE_ENOMEM, "encoder_create: out of host memory");
  std::memset(e, 0, sizeof(*e));
  e->desc = *d;
  const double n = (double)d->d;
  // Eq. 2: F_n = (sqrt(n+1) - 1) / n.  Sec. 5.1: simplex input multiplier N_l * m / sqrt(n+1),
  // m = 1 or (n+1)^((n-1)/(2n)) (Sec. 5.2); grid multiplier N_l.  FP64, rounded once.
  const double m = d->res_mode == SXE_RES_EQUAL_MEM ? std::pow(n + 1.0, (n - 1.0) / (2.0 * n)) : 1.0;
  for (int l = 0; l < d->n_levels; ++l) {
    const double N = std::floor(d->base_res * std::pow(d->growth, (double)l));
    if (N > 1.0e9) {
      delete e;
      return set_error(SXE_EINVAL, "encoder_create: level %d resolution %.0f too large", l, N);
    }
    e->level_res[l] = (int32_t)N;
    e->prm.scale[l] = d->kind == SXE_SIMPLEX ? (float)(N * m / std::sqrt(n + 1.0)) : (float)N;
    // Directly indexed level: the vertices of [0,1]^n take B = floor(top) + 2 values per axis,
    // top = s_l sqrt(n+1) (simplex, q_i <= s_l (1 + n F_n)) or N_l (grid), with a 2^-20
    // margin for binary32 rounding; used when B^n fits the table.
    const double top = (double)e->prm.scale[l] * (d->kind == SXE_SIMPLEX ? std::sqrt(n + 1.0) : 1.0);
    const double B = std::floor(top * (1.0 + std::ldexp(1.0, -20))) + 2.0;
    e->box_width[l] = B < 4.0e9 ? (uint32_t)B : 0u;
    if (d->index_mode == SXE_INDEX_DENSE_COARSE && std::pow(B, n) <= std::ldexp(1.0, d->log2_T))
      e->prm.width[l] = (uint32_t)B;
  }
  e->prm.n_levels = d->n_levels;
  e->prm.log2_T = d->log2_T;
  e->prm.out_dtype = d->out_dtype;
  e->prm.skew_F = (float)((std::sqrt(n + 1.0) - 1.0) / n);
  *out = e;
  return SXE_OK;
}

sxe_status sxe_encoder_level_index(const sxe_encoder* e, int32_t* width) {
  if (!e || !width) return set_error(SXE_EINVAL, "encoder_level_index: NULL argument");
  for (int l = 0; l < e->desc.n_levels; ++l) width[l] = (int32_t)e->prm.width[l];
  return SXE_OK;
}

sxe_status sxe_encoder_set_bwd_aggregation(sxe_encoder* e, int32_t on) {
  if (!e) return set_error(SXE_EINVAL, "encoder_set_bwd_aggregation: NULL encoder");
  if (on != 0 && on != 1) return set_error(SXE_EINVAL, "encoder_set_bwd_aggregation: on=%d is not 0 or 1", on);
  e->bwd_aggregate = on;
  return SXE_OK;
}

sxe_status sxe_encoder_set_fwd_order(sxe_encoder* e, int32_t order) {
  if (!e) return set_error(SXE_EINVAL, "encoder_set_fwd_order: NULL encoder");
  if (order < SXE_FWD_ORDER_AUTO || order > SXE_FWD_ORDER_LEVEL_MAJOR)
    return set_error(SXE_EINVAL, "encoder_set_fwd_order: order=%d is not 0, 1 or 2", order);
  e->fwd_order = order;
  return SXE_OK;
}

sxe_status sxe_encoder_destroy(sxe_encoder* e) {
  delete e;
  return SXE_OK;
}

sxe_status sxe_encoder_level_params(const sxe_encoder* e, float* scale, int32_t* res) {
  if (!e) return set_error(SXE_EINVAL, "encoder_level_params: NULL encoder");
  for (int l = 0; l < e->desc.n_levels; ++l) {
    if (scale) scale[l] = e->prm.scale[l];
    if (res) res[l] = e->level_res[l];
  }
  return SXE_OK;
}

static sxe_status check_points(const char* fn, const sxe_encoder* e, const float* x, int64_t P) {
  if (!e) return set_error(SXE_EINVAL, "%s: NULL encoder", fn);
  // the encoding kernels run one thread per (point, level): P * L <= 2^38 keeps their grids of
  // P * L / 256 blocks far inside the 2^31 - 1 limit of gridDim.x
  if (P < 0 || P > ((int64_t)1 << 38) / e->desc.n_levels)
    return set_error(SXE_EINVAL, "%s: n_points=%lld out of range (n_points * n_levels <= 2^38)", fn, (long long)P);
  if (P > 0 && !x) return set_error(SXE_EINVAL, "%s: NULL x", fn);
  const size_t xa = e->desc.d == 2 ? 8 : e->desc.d == 4 ? 16 : 4;
  if (!aligned(x, xa)) return set_error(SXE_EINVAL, "%s: x must be %zu-byte aligned for d=%d", fn, xa, e->desc.d);
  return SXE_OK;
}

static sxe_status encode_fwd_common(const char* fn, const sxe_encoder* e, const float* x, int64_t P,
                                    const void* tables, void* out, uint32_t* touched, void* stream) {
  sxe_status st = check_points(fn, e, x, P);
  if (st != SXE_OK) return st;
  if (P == 0) return SXE_OK;
  if (!tables || !out) return set_error(SXE_EINVAL, "%s: NULL tables or out", fn);
  const int F = e->desc.n_features;
  const size_t ta = std::min<size_t>(16, F * dtype_size(e->desc.table_dtype));
  if (!aligned(tables, ta)) return set_error(SXE_EINVAL, "%s: tables must be %zu-byte aligned", fn, ta);
  const size_t oa = F == 2 ? 2 * dtype_size(e->desc.out_dtype) : dtype_size(e->desc.out_dtype);
  if (!aligned(out, oa)) return set_error(SXE_EINVAL, "%s: out must be %zu-byte aligned", fn, oa);
  return launch_encode_fwd(e, x, P, tables, out, (cudaStream_t)stream, 0, touched);
}

sxe_status sxe_encode_fwd(const sxe_encoder* e, const float* x, int64_t P, const void* tables, void* out,
                          void* stream) {
  return encode_fwd_common("encode_fwd", e, x, P, tables, out, nullptr, stream);
}

sxe_status sxe_encode_fwd_marked(const sxe_encoder* e, const float* x, int64_t P, const void* tables, void* out,
                                 uint32_t* touched, void* stream) {
  if (P > 0 && !touched) return set_error(SXE_EINVAL, "encode_fwd_marked: NULL touched");
  if (touched && !aligned(touched, 4)) return set_error(SXE_EINVAL, "encode_fwd_marked: touched misaligned");
  return encode_fwd_common("encode_fwd_marked", e, x, P, tables, out, touched, stream);
}

sxe_status sxe_encode_bwd(const sxe_encoder* e, const float* x, int64_t P, const float* dout, float* grad,
                          int64_t grad_stride, uint32_t* touched, void* stream) {
  if (!e) return set_error(SXE_EINVAL, "encode_bwd: NULL encoder");
  return sxe_encode_bwd_levels(e, x, P, dout, grad, grad_stride, touched, 0, e->desc.n_levels, stream);
}

sxe_status sxe_encode_bwd_levels(const sxe_encoder* e, const float* x, int64_t P, const float* dout, float* grad,
                                 int64_t grad_stride, uint32_t* touched, int32_t level_begin, int32_t level_end,
                                 void* stream) {
  sxe_status st = check_points("encode_bwd", e, x, P);
  if (st != SXE_OK) return st;
  if (P == 0) return SXE_OK;
  if (!dout || !grad) return set_error(SXE_EINVAL, "encode_bwd: NULL dout or grad");
  const int F = e->desc.n_features;
  if (grad_stride < F || grad_stride % F != 0 || grad_stride > (1 << 16))
    return set_error(SXE_EINVAL, "encode_bwd: grad_stride=%lld must be a multiple of F=%d", (long long)grad_stride, F);
  const size_t ga = F == 1 ? 4 : F == 2 ? 8 : 16;
  if (!aligned(grad, ga) || ((grad_stride * 4) % ga) != 0)
    return set_error(SXE_EINVAL, "encode_bwd: gradient entries must be %zu-byte aligned", ga);
  if (!aligned(dout, F == 2 ? 8 : 4)) return set_error(SXE_EINVAL, "encode_bwd: dout misaligned");
  if (touched && !aligned(touched, 4)) return set_error(SXE_EINVAL, "encode_bwd: touched misaligned");
  if (level_begin < 0 || level_end > e->desc.n_levels || level_begin > level_end)
    return set_error(SXE_EINVAL, "encode_bwd: level range [%d, %d) outside [0, %d)", level_begin, level_end,
                     e->desc.n_levels);
  if (level_begin == level_end) return SXE_OK;
  return launch_encode_bwd(e, x, P, dout, grad, grad_stride, touched, (cudaStream_t)stream, level_begin, level_end);
}

int32_t sxe_encode_bwd_kernel_count(const sxe_encoder* e, int64_t P) {
  if (!e || P <= 0) return 0;
  return encode_bwd_launches(e, P);
}

int32_t sxe_encode_bwd_levels_kernel_count(const sxe_encoder* e, int64_t P, int32_t level_begin, int32_t level_end) {
  if (!e || P <= 0 || level_begin < 0 || level_end > e->desc.n_levels || level_begin >= level_end) return 0;
  return encode_bwd_launches(e, P, level_begin, level_end);
}

int32_t sxe_encode_bwd_coarse_levels(const sxe_encoder* e, int64_t P) {
  if (!e || P <= 0) return 0;
  return encode_bwd_coarse_levels(e, P);
}

sxe_status sxe_encode_bwd_input(const sxe_encoder* e, const float* x, int64_t P, const void* tables,
                                const float* dout, float* dx, void* stream) {
  sxe_status st = check_points("encode_bwd_input", e, x, P);
  if (st != SXE_OK) return st;
  if (P == 0) return SXE_OK;
  if (!tables || !dout || !dx) return set_error(SXE_EINVAL, "encode_bwd_input: NULL tables, dout or dx");
  const int F = e->desc.n_features;
  const size_t ta = std::min<size_t>(16, F * dtype_size(e->desc.table_dtype));
  if (!aligned(tables, ta)) return set_error(SXE_EINVAL, "encode_bwd_input: tables must be %zu-byte aligned", ta);
  if (!aligned(dout, 4) || !aligned(dx, 4)) return set_error(SXE_EINVAL, "encode_bwd_input: dout or dx misaligned");
  return launch_encode_bwd_input(e, x, P, tables, dout, dx, (cudaStream_t)stream);
}

static sxe_status check_rays(const char* fn, int64_t R, int32_t S) {
  if (R < 0 || S < 1 || S > (1 << 20) || R > ((int64_t)1 << 36) / S)
    return set_error(SXE_EINVAL, "%s: n_rays=%lld n_samples=%d out of range", fn, (long long)R, S);
  return SXE_OK;
}

sxe_status sxe_vr_samples(const float* origins, const float* dirs, const float* t_near, const float* t_far,
                          int64_t R, int32_t S, float* x, float* delta, void* stream) {
  sxe_status st = check_rays("vr_samples", R, S);
  if (st != SXE_OK || R == 0) return st;
  if (!origins || !dirs || !t_near || !t_far || !x || !delta)
    return set_error(SXE_EINVAL, "vr_samples: NULL buffer");
  if (!aligned(origins, 4) || !aligned(dirs, 4) || !aligned(t_near, 4) || !aligned(t_far, 4) || !aligned(x, 4) ||
      !aligned(delta, 4))
    return set_error(SXE_EINVAL, "vr_samples: misaligned buffer");
  return launch_vr_samples(origins, dirs, t_near, t_far, R, S, x, delta, (cudaStream_t)stream);
}

sxe_status sxe_vr_field(const float* density_out, const float* dirs, int64_t R, int32_t S, int32_t dtype,
                        float* sigma, void* color_in, void* stream) {
  sxe_status st = check_rays("vr_field", R, S);
  if (st != SXE_OK || R == 0) return st;
  if (dtype != SXE_F16 && dtype != SXE_BF16) return set_error(SXE_EINVAL, "vr_field: dtype must be f16 or bf16");
  if (!density_out || !dirs || !sigma || !color_in) return set_error(SXE_EINVAL, "vr_field: NULL buffer");
  if (!aligned(density_out, 16) || !aligned(color_in, 16) || !aligned(dirs, 4) || !aligned(sigma, 4))
    return set_error(SXE_EINVAL, "vr_field: density_out and color_in must be 16-byte aligned");
  return launch_vr_field(density_out, dirs, R, S, dtype, sigma, color_in, (cudaStream_t)stream);
}

sxe_status sxe_vr_composite_bwd(const float* sigma, const float* rgb_logits, const float* delta, const float* color,
                                const float* dcolor, int64_t R, int32_t S, float* dsigma, float* dlogits,
                                void* stream) {
  sxe_status st = check_rays("vr_composite_bwd", R, S);
  if (st != SXE_OK || R == 0) return st;
  if (!sigma || !rgb_logits || !delta || !color || !dcolor || !dsigma || !dlogits)
    return set_error(SXE_EINVAL, "vr_composite_bwd: NULL buffer");
  if (!aligned(sigma, 4) || !aligned(rgb_logits, 4) || !aligned(delta, 4) || !aligned(color, 4) ||
      !aligned(dcolor, 4) || !aligned(dsigma, 4) || !aligned(dlogits, 4))
    return set_error(SXE_EINVAL, "vr_composite_bwd: misaligned buffer");
  return launch_vr_composite_bwd(sigma, rgb_logits, delta, color, dcolor, R, S, dsigma, dlogits,
                                 (cudaStream_t)stream);
}

sxe_status sxe_vr_field_bwd(const float* dcolor_in, const float* dsigma, const float* sigma, const float* density_out,
                            int64_t R, int32_t S, float* dv, void* stream) {
  sxe_status st = check_rays("vr_field_bwd", R, S);
  if (st != SXE_OK || R == 0) return st;
  if (!dcolor_in || !dsigma || !sigma || !density_out || !dv) return set_error(SXE_EINVAL, "vr_field_bwd: NULL buffer");
  if (!aligned(dcolor_in, 16) || !aligned(dv, 16) || !aligned(dsigma, 4) || !aligned(sigma, 4) ||
      !aligned(density_out, 4))
    return set_error(SXE_EINVAL, "vr_field_bwd: dcolor_in and dv must be 16-byte aligned");
  return launch_vr_field_bwd(dcolor_in, dsigma, sigma, density_out, R * S, dv, (cudaStream_t)stream);
}

sxe_status sxe_vr_composite(const float* sigma, const float* rgb_logits, const float* delta, int64_t R, int32_t S,
                            float* color, float* transmittance, float* weights, void* stream) {
  sxe_status st = check_rays("vr_composite", R, S);
  if (st != SXE_OK || R == 0) return st;
  if (!sigma || !rgb_logits || !delta || !color) return set_error(SXE_EINVAL, "vr_composite: NULL buffer");
  if (!aligned(sigma, 4) || !aligned(rgb_logits, 4) || !aligned(delta, 4) || !aligned(color, 4) ||
      !aligned(transmittance, 4) || !aligned(weights, 4))
    return set_error(SXE_EINVAL, "vr_composite: misaligned buffer");
  return launch_vr_composite(sigma, rgb_logits, delta, R, S, color, transmittance, weights, (cudaStream_t)stream);
}

sxe_status sxe_encode_vertices(const sxe_encoder* e, const float* x, int64_t P, uint32_t* slots, float* weights,
                               void* stream) {
  sxe_status st = check_points("encode_vertices", e, x, P);
  if (st != SXE_OK) return st;
  if (P == 0 || (!slots && !weights)) return SXE_OK;
  return launch_encode_vertices(e, x, P, slots, weights, (cudaStream_t)stream);
}

static sxe_status check_plain(const char* fn, const sxe_encoder* e, const float* x, int64_t P, const void* a,
                              const void* b) {
  sxe_status st = check_points(fn, e, x, P);
  if (st != SXE_OK) return st;
  if (e->desc.kind != SXE_SIMPLEX || e->desc.table_dtype != SXE_F32 || e->desc.out_dtype != SXE_F32 ||
      e->desc.index_mode != SXE_INDEX_HASH)
    return set_error(SXE_EUNSUPPORTED, "%s: needs a hashed simplex encoder with binary32 tables and output", fn);
  if (P > 0 && (!a || !b)) return set_error(SXE_EINVAL, "%s: NULL buffer", fn);
  return SXE_OK;
}

sxe_status sxe_encode_plain_fwd(const sxe_encoder* e, const float* x, int64_t P, const float* tables, float* out,
                                void* stream) {
  sxe_status st = check_plain("encode_plain_fwd", e, x, P, tables, out);
  if (st != SXE_OK || P == 0) return st;
  return launch_encode_plain(e, false, x, P, tables, out, (cudaStream_t)stream);
}

sxe_status sxe_encode_plain_bwd(const sxe_encoder* e, const float* x, int64_t P, const float* dout, float* grad,
                                void* stream) {
  sxe_status st = check_plain("encode_plain_bwd", e, x, P, dout, grad);
  if (st != SXE_OK || P == 0) return st;
  return launch_encode_plain(e, true, x, P, dout, grad, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
static sxe_status vr_field_mlp(const char* fn, const sxe_mlp_desc* dd, const void* Wd, const sxe_mlp_desc* dc,
                               const void* Wc, const void* enc, const float* dirs, int64_t R, int32_t S, float* sigma,
                               float* logits, float* dens_out, void* color_in, void* stream) {
  sxe_status st = check_rays(fn, R, S);
  if (st != SXE_OK) return st;
  if (!dd || !dc) return set_error(SXE_EINVAL, "%s: NULL network description", fn);
  if ((st = check_mlp(fn, dd)) != SXE_OK || (st = check_mlp(fn, dc)) != SXE_OK) return st;
  if (dd->n_hidden != 1 || dd->n_out != 16 || dc->n_in != 32 || dc->dtype != dd->dtype)
    return set_error(SXE_EUNSUPPORTED, "%s: needs a density network n_in -> 64 -> 16 and a colour "
                     "network 32 -> ... of the same dtype", fn);
  if (R == 0) return SXE_OK;
  if (!Wd || !Wc || !enc || !dirs || !sigma || !logits) return set_error(SXE_EINVAL, "%s: NULL buffer", fn);
  if (!aligned(enc, 16) || !aligned(Wd, 4) || !aligned(Wc, 4) || !aligned(dirs, 4) || !aligned(sigma, 4) ||
      !aligned(logits, 4))
    return set_error(SXE_EINVAL, "%s: misaligned buffer (encoding rows need 16 bytes)", fn);
  if ((dens_out && !aligned(dens_out, 16)) || (color_in && !aligned(color_in, 16)))
    return set_error(SXE_EINVAL, "%s: density_out and color_in must be 16-byte aligned", fn);
  return launch_vr_field_mlp(dd, Wd, dc, Wc, enc, dirs, R, S, sigma, logits, dens_out, color_in,
                             (cudaStream_t)stream);
}

sxe_status sxe_vr_field_mlp(const sxe_mlp_desc* dd, const void* Wd, const sxe_mlp_desc* dc, const void* Wc,
                            const void* enc, const float* dirs, int64_t R, int32_t S, float* sigma, float* logits,
                            void* stream) {
  return vr_field_mlp("vr_field_mlp", dd, Wd, dc, Wc, enc, dirs, R, S, sigma, logits, nullptr, nullptr, stream);
}

sxe_status sxe_vr_field_mlp_saved(const sxe_mlp_desc* dd, const void* Wd, const sxe_mlp_desc* dc, const void* Wc,
                                  const void* enc, const float* dirs, int64_t R, int32_t S, float* sigma,
                                  float* logits, float* density_out, void* color_in, void* stream) {
  if (R > 0 && (!density_out || !color_in))
    return set_error(SXE_EINVAL, "vr_field_mlp_saved: NULL density_out or color_in");
  return vr_field_mlp("vr_field_mlp_saved", dd, Wd, dc, Wc, enc, dirs, R, S, sigma, logits, density_out, color_in,
                      stream);
}

int64_t sxe_mlp_n_params(const sxe_mlp_desc* d) {
  if (!d) return 0;
  return (int64_t)d->width * d->n_in + (int64_t)(d->n_hidden - 1) * d->width * d->width + (int64_t)d->n_out * d->width;
}

sxe_status sxe_mlp_fwd(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out, void* act,
                       void* stream) {
  sxe_status st = check_mlp("mlp_fwd", d);
  if (st != SXE_OK) return st;
  if (P < 0) return set_error(SXE_EINVAL, "mlp_fwd: n_points < 0");
  if (P == 0) return SXE_OK;
  if (!W || !in || !out) return set_error(SXE_EINVAL, "mlp_fwd: NULL weights, in or out");
  if (!aligned(in, 16) || !aligned(W, 4) || (act && !aligned(act, 4)))
    return set_error(SXE_EINVAL, "mlp_fwd: in must be 16-byte aligned, weights/act 4-byte aligned");
  return launch_mlp_fwd(d, W, in, P, out, act, (cudaStream_t)stream);
}

int64_t sxe_mlp_bwd_workspace_bytes(const sxe_mlp_desc* d, int64_t P) {
  if (!d || P <= 0) return 0;
  return (int64_t)mlp_grid_blocks(d, P) * (sxe_mlp_n_params(d) + 1) * (int64_t)sizeof(float);
}

static sxe_status mlp_bwd_common(const char* fn, const sxe_mlp_desc* d, const void* W, const void* in,
                                 const float* dout, const float* target, float loss_scale, int64_t P, float* din,
                                 float* dW, float* sq_sum, void* ws, int64_t ws_bytes, void* stream,
                                 int64_t loss_count = 0) {
  sxe_status st = check_mlp(fn, d);
  if (st != SXE_OK) return st;
  if (P < 0) return set_error(SXE_EINVAL, "%s: n_points < 0", fn);
  if (P == 0) return empty_batch_sq_sum(fn, sq_sum, stream);
  if (!W || !in || !dW || !ws) return set_error(SXE_EINVAL, "%s: NULL weights, in, dweights or workspace", fn);
  if (!(loss_scale > 0.f) || !std::isfinite(loss_scale)) return set_error(SXE_EINVAL, "%s: loss_scale must be > 0", fn);
  if (!aligned(in, 16) || !aligned(W, 4) || !aligned(ws, 4) || (din && !aligned(din, 8)))
    return set_error(SXE_EINVAL, "%s: misaligned buffer", fn);
  const int64_t need = sxe_mlp_bwd_workspace_bytes(d, P);
  if (ws_bytes < need) return set_error(SXE_ENOMEM, "%s: workspace %lld < %lld bytes", fn, (long long)ws_bytes, (long long)need);
  return launch_mlp_bwd(d, W, in, dout, target, loss_scale, P, din, dW, sq_sum, (float*)ws, mlp_grid_blocks(d, P),
                        (cudaStream_t)stream, 0, loss_count);
}

sxe_status sxe_mlp_bwd(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout, float loss_scale,
                       int64_t P, float* din, float* dW, void* ws, int64_t ws_bytes, void* stream) {
  if (P > 0 && !dout) return set_error(SXE_EINVAL, "mlp_bwd: NULL dout");
  return mlp_bwd_common("mlp_bwd", d, W, in, dout, nullptr, loss_scale, P, din, dW, nullptr, ws, ws_bytes, stream);
}

sxe_status sxe_mlp_train_l2(const sxe_mlp_desc* d, const void* W, const void* in, const float* target,
                            float loss_scale, int64_t P, float* din, float* dW, float* sq_sum, void* ws,
                            int64_t ws_bytes, void* stream) {
  if (P > 0 && (!target || !sq_sum)) return set_error(SXE_EINVAL, "mlp_train_l2: NULL target or sq_sum");
  return mlp_bwd_common("mlp_train_l2", d, W, in, nullptr, target, loss_scale, P, din, dW, sq_sum, ws, ws_bytes,
                        stream);
}

sxe_status sxe_mlp_train_l2_part(const sxe_mlp_desc* d, const void* W, const void* in, const float* target,
                                 float loss_scale, int64_t P, int64_t batch_points, float* din, float* dW,
                                 float* sq_sum, void* ws, int64_t ws_bytes, void* stream) {
  if (P > 0 && (!target || !sq_sum)) return set_error(SXE_EINVAL, "mlp_train_l2_part: NULL target or sq_sum");
  if (P > 0 && batch_points < P)
    return set_error(SXE_EINVAL, "mlp_train_l2_part: batch_points=%lld must be >= n_points=%lld",
                     (long long)batch_points, (long long)P);
  return mlp_bwd_common("mlp_train_l2_part", d, W, in, nullptr, target, loss_scale, P, din, dW, sq_sum, ws, ws_bytes,
                        stream, batch_points);
}

sxe_status sxe_mlp_train_l2_grouped(const sxe_mlp_desc* d, const void* W, const void* in, const float* target,
                                    float loss_scale, int64_t P, float* din, int32_t din_group, float* dW,
                                    float* sq_sum, void* ws, int64_t ws_bytes, void* stream) {
  if (!d) return set_error(SXE_EINVAL, "mlp_train_l2_grouped: NULL desc");
  if (!(din_group == 1 || din_group == 2 || din_group == 4 || din_group == 8) || d->n_in % din_group != 0)
    return set_error(SXE_EINVAL, "mlp_train_l2_grouped: din_group=%d must be 1, 2, 4 or 8 and divide n_in", din_group);
  if (P > 0 && (!target || !sq_sum || !din)) return set_error(SXE_EINVAL, "mlp_train_l2_grouped: NULL target, sq_sum or din");
  sxe_status st = check_mlp("mlp_train_l2_grouped", d);
  if (st != SXE_OK) return st;
  if (P < 0) return set_error(SXE_EINVAL, "mlp_train_l2_grouped: n_points < 0");
  if (P == 0) return empty_batch_sq_sum("mlp_train_l2_grouped", sq_sum, stream);
  if (!W || !in || !dW || !ws) return set_error(SXE_EINVAL, "mlp_train_l2_grouped: NULL weights, in, dweights or workspace");
  if (!(loss_scale > 0.f) || !std::isfinite(loss_scale)) return set_error(SXE_EINVAL, "mlp_train_l2_grouped: loss_scale must be > 0");
  if (!aligned(in, 16) || !aligned(W, 4) || !aligned(ws, 4) || !aligned(din, 8))
    return set_error(SXE_EINVAL, "mlp_train_l2_grouped: misaligned buffer");
  const int64_t need = sxe_mlp_bwd_workspace_bytes(d, P);
  if (ws_bytes < need) return set_error(SXE_ENOMEM, "mlp_train_l2_grouped: workspace %lld < %lld bytes", (long long)ws_bytes, (long long)need);
  return launch_mlp_bwd(d, W, in, nullptr, target, loss_scale, P, din, dW, sq_sum, (float*)ws, mlp_grid_blocks(d, P),
                        (cudaStream_t)stream, din_group);
}

sxe_status sxe_mlp_set_kernel(int32_t k) {
  if (k != SXE_MLP_KERNEL_AUTO && k != SXE_MLP_KERNEL_MMA_SYNC && k != SXE_MLP_KERNEL_TCGEN05 &&
      k != SXE_MLP_KERNEL_TCGEN05_PIPELINED && k != SXE_MLP_KERNEL_TCGEN05_3TILE)
    return set_error(SXE_EINVAL, "mlp_set_kernel: unknown kernel %d", k);
  g_mlp_kernel = k;
  return SXE_OK;
}

int32_t sxe_mlp_get_kernel(void) { return g_mlp_kernel; }

sxe_status sxe_selftest_wait(int32_t expect_timeout, int64_t limit_ns, void* stream) {
  if (!(limit_ns > 0 && limit_ns <= 2000000000ll))
    return set_error(SXE_EINVAL, "selftest_wait: limit_ns=%lld outside (0, 2e9]", (long long)limit_ns);
  return launch_selftest_wait(expect_timeout != 0, limit_ns, (cudaStream_t)stream);
}

sxe_status sxe_device_error(int32_t* flag, int32_t clear) {
  if (!flag) return set_error(SXE_EINVAL, "device_error: NULL flag");
  return read_tc_error(flag, clear != 0);
}

sxe_status sxe_loss_l2(const float* y, const float* target, int64_t P, int32_t n_out, float* dy, float* sq_sum,
                       void* stream) {
  if (P < 0 || n_out < 1) return set_error(SXE_EINVAL, "loss_l2: bad sizes");
  if (P == 0) return SXE_OK;
  if (!y || !target || !dy || !sq_sum) return set_error(SXE_EINVAL, "loss_l2: NULL argument");
  return launch_loss_l2(y, target, P, n_out, dy, sq_sum, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
static sxe_status check_adam(const char* fn, const sxe_adam_desc* a, int64_t t) {
  if (!a) return set_error(SXE_EINVAL, "%s: NULL desc", fn);
  if (t < 1) return set_error(SXE_EINVAL, "%s: step t must be >= 1", fn);
  if (!(a->lr >= 0.f) || !(a->beta1 >= 0.f && a->beta1 < 1.f) || !(a->beta2 >= 0.f && a->beta2 < 1.f) ||
      !(a->eps >= 0.f))
    return set_error(SXE_EINVAL, "%s: bad hyper-parameters", fn);
  return SXE_OK;
}

sxe_status sxe_step(const sxe_adam_desc* a, int64_t t, int64_t n, float* p, float* m, float* v, float* g,
                    void* lowp, int32_t lowp_dtype, void* stream) {
  sxe_status st = check_adam("step", a, t);
  if (st != SXE_OK) return st;
  if (n < 0) return set_error(SXE_EINVAL, "step: n < 0");
  if (n == 0) return SXE_OK;
  if (!p || !m || !v || !g) return set_error(SXE_EINVAL, "step: NULL param, m, v or grad");
  if (lowp && !valid_dtype(lowp_dtype)) return set_error(SXE_EINVAL, "step: bad lowp dtype");
  return launch_adam_dense(a, t, n, p, m, v, g, lowp, lowp_dtype, (cudaStream_t)stream);
}

sxe_status sxe_step_touched(const sxe_adam_desc* a, int64_t t, int64_t n_entries, int32_t F, float* state,
                            uint32_t* touched, void* lowp, int32_t lowp_dtype, void* stream) {
  sxe_status st = check_adam("step_touched", a, t);
  if (st != SXE_OK) return st;
  if (n_entries < 0) return set_error(SXE_EINVAL, "step_touched: n_entries < 0");
  if (!(F == 1 || F == 2 || F == 4 || F == 8)) return set_error(SXE_EINVAL, "step_touched: F=%d", F);
  if (n_entries == 0) return SXE_OK;
  if (!state || !touched || !lowp) return set_error(SXE_EINVAL, "step_touched: NULL state, touched or table");
  if (!valid_dtype(lowp_dtype)) return set_error(SXE_EINVAL, "step_touched: bad lowp dtype");
  if (!aligned(state, 16) || !aligned(touched, 4) || !aligned(lowp, F == 2 ? 2 * dtype_size(lowp_dtype) : 1))
    return set_error(SXE_EINVAL, "step_touched: misaligned buffer");
  return launch_adam_touched(a, t, n_entries, F, state, touched, lowp, lowp_dtype, (cudaStream_t)stream);
}

sxe_status sxe_adam_advance(const sxe_adam_desc* a, int64_t* t, float* corrections, void* stream) {
  sxe_status st = check_adam("adam_advance", a, 1);
  if (st != SXE_OK) return st;
  if (!t || !corrections || !aligned(t, 8) || !aligned(corrections, 4))
    return set_error(SXE_EINVAL, "adam_advance: NULL or misaligned step counter or corrections");
  return launch_adam_advance(a, t, corrections, (cudaStream_t)stream);
}

sxe_status sxe_step_dev(const sxe_adam_desc* a, const float* corrections, int64_t n, float* p, float* m, float* v,
                        float* g, void* lowp, int32_t lowp_dtype, void* stream) {
  if (!corrections || !aligned(corrections, 4)) return set_error(SXE_EINVAL, "step_dev: NULL or misaligned corrections");
  sxe_status st = check_adam("step_dev", a, 1);
  if (st != SXE_OK) return st;
  if (n < 0) return set_error(SXE_EINVAL, "step_dev: n < 0");
  if (n == 0) return SXE_OK;
  if (!p || !m || !v || !g) return set_error(SXE_EINVAL, "step_dev: NULL buffer");
  if (lowp && !valid_dtype(lowp_dtype)) return set_error(SXE_EINVAL, "step_dev: bad lowp dtype");
  return launch_adam_dense(a, 1, n, p, m, v, g, lowp, lowp_dtype, (cudaStream_t)stream, corrections);
}

sxe_status sxe_step_touched_dev(const sxe_adam_desc* a, const float* corrections, int64_t n_entries, int32_t F,
                                float* state, uint32_t* touched, void* lowp, int32_t lowp_dtype, void* stream) {
  if (!corrections || !aligned(corrections, 4))
    return set_error(SXE_EINVAL, "step_touched_dev: NULL or misaligned corrections");
  sxe_status st = check_adam("step_touched_dev", a, 1);
  if (st != SXE_OK) return st;
  if (n_entries < 0) return set_error(SXE_EINVAL, "step_touched_dev: n_entries < 0");
  if (!(F == 1 || F == 2 || F == 4 || F == 8)) return set_error(SXE_EINVAL, "step_touched_dev: F=%d", F);
  if (n_entries == 0) return SXE_OK;
  if (!state || !touched || !lowp) return set_error(SXE_EINVAL, "step_touched_dev: NULL state, touched or table");
  if (!valid_dtype(lowp_dtype)) return set_error(SXE_EINVAL, "step_touched_dev: bad lowp dtype");
  if (!aligned(state, 16) || !aligned(touched, 4) || !aligned(lowp, F == 2 ? 2 * dtype_size(lowp_dtype) : 1))
    return set_error(SXE_EINVAL, "step_touched_dev: misaligned buffer");
  return launch_adam_touched(a, 1, n_entries, F, state, touched, lowp, lowp_dtype, (cudaStream_t)stream, corrections);
}

}  // extern "C"
