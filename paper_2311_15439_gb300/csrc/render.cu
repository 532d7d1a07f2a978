// Volumetric rendering with the encodings (Sec. 6.2, Eq. 5): ray samples, the field head
// between the density and colour networks, and the front-to-back compositing of a ray.
//
// Sampling: S samples per ray at the midpoints of S equal segments of [t_near, t_far],
// delta = (t_far - t_near) / S, t_i = t_near + (i + 1/2) delta, x_i = o + t_i d, each
// operation rounded once in this order.  Quadrature of Eq. 5 for a field constant on each
// segment: T_i = exp(-sum_{j<i} sigma_j delta), alpha_i = 1 - exp(-sigma_i delta),
// C = sum_i T_i alpha_i c_i.  The transmittance is a running product, but it is the exp of a
// prefix sum, so a warp computes 32 samples at a time with a shuffle scan and carries the sum.
#include "sxe_internal.cuh"

namespace sxe {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
vr_samples_kernel(const float* __restrict__ o, const float* __restrict__ d, const float* __restrict__ tn,
                  const float* __restrict__ tf, int64_t R, int S, float* __restrict__ x, float* __restrict__ delta) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= R * S) return;
  const int64_t r = i / S;
  const int k = (int)(i - r * S);
  const float t0 = __ldg(tn + r);
  const float dl = __fdiv_rn(__fsub_rn(__ldg(tf + r), t0), (float)S);
  const float t = __fadd_rn(t0, __fmul_rn((float)k + 0.5f, dl));
#pragma unroll
  for (int c = 0; c < 3; ++c) x[i * 3 + c] = __fadd_rn(__ldg(o + r * 3 + c), __fmul_rn(t, __ldg(d + r * 3 + c)));
  if (k == 0) delta[r] = dl;
}

// Field head: sigma = exp(min(v_0, 15)) from the density network's 16 outputs v, and the
// colour network's input row [v_0..v_15, SH(d)] in the network dtype.
template <typename T>
__global__ void __launch_bounds__(kThreads)
vr_field_kernel(const float* __restrict__ dens, const float* __restrict__ dirs, int64_t P, int S,
                float* __restrict__ sigma, T* __restrict__ cin) {
  const int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= P) return;
  float v[16];
  const float4* src = reinterpret_cast<const float4*>(dens + p * 16);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float4 a = __ldg(src + j);
    v[4 * j] = a.x; v[4 * j + 1] = a.y; v[4 * j + 2] = a.z; v[4 * j + 3] = a.w;
  }
  sigma[p] = vr_density(v[0]);
  const int64_t r = p / S;
  float h[16];
  sh16(__ldg(dirs + r * 3), __ldg(dirs + r * 3 + 1), __ldg(dirs + r * 3 + 2), h);
  // 32 values of 2 bytes = 64 bytes per row: four 16-byte stores
  union { uint4 q[4]; T t[32]; } u;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    u.t[j] = from_f32<T>(v[j]);
    u.t[16 + j] = from_f32<T>(h[j]);
  }
  uint4* dst = reinterpret_cast<uint4*>(cin + p * 32);
#pragma unroll
  for (int j = 0; j < 4; ++j) dst[j] = u.q[j];
}

// One warp per ray; lanes take 32 consecutive samples at a time.
__global__ void __launch_bounds__(kThreads)
vr_composite_kernel(const float* __restrict__ sigma, const float* __restrict__ logits,
                    const float* __restrict__ delta, int64_t R, int S, float* __restrict__ color,
                    float* __restrict__ trans, float* __restrict__ weights) {
  const int64_t r = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (r >= R) return;                                   // whole warps leave together
  const int lane = threadIdx.x & 31;
  const float dl = __ldg(delta + r);
  float carry = 0.f;                                    // sum of sigma delta over earlier chunks
  float c0 = 0.f, c1 = 0.f, c2 = 0.f;
  for (int base = 0; base < S; base += 32) {
    const int k = base + lane;
    const int64_t i = r * S + k;
    float s = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f;
    if (k < S) {
      s = __ldg(sigma + i) * dl;
      l0 = __ldg(logits + i * 3);
      l1 = __ldg(logits + i * 3 + 1);
      l2 = __ldg(logits + i * 3 + 2);
    }
    float incl = s;                                     // inclusive prefix sum within the chunk
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    float excl = __shfl_up_sync(0xffffffffu, incl, 1);  // exclusive prefix, no cancellation
    if (lane == 0) excl = 0.f;
    const float tau = carry + excl;                     // sum over all earlier samples
    const float w = expf(-tau) * -expm1f(-s);           // T_i alpha_i
    if (k < S) {
      c0 += w / (1.f + expf(-l0));
      c1 += w / (1.f + expf(-l1));
      c2 += w / (1.f + expf(-l2));
      if (weights) weights[i] = w;
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c0 += __shfl_xor_sync(0xffffffffu, c0, o);
    c1 += __shfl_xor_sync(0xffffffffu, c1, o);
    c2 += __shfl_xor_sync(0xffffffffu, c2, o);
  }
  if (lane == 0) {
    color[r * 3] = c0;
    color[r * 3 + 1] = c1;
    color[r * 3 + 2] = c2;
    if (trans) trans[r] = expf(-carry);
  }
}

// Backward of the compositing for upstream colour gradients dC [R][3], one warp per ray.
// With w_k = T_k alpha_k and P_k = sum_{i<=k} w_i c_i (the colour accumulated up to sample k):
//   dL/dsigma_k = delta sum_c dC_c (T_{k+1} c_k,c - (C_c - P_k,c)),
//   dL/dlogit_k,c = dC_c w_k c_k,c (1 - c_k,c)  (1 - c taken as the sigmoid of -logit),
// where T_{k+1} = T_k (1 - alpha_k) and C is the forward pass's colour.  The same prefix scans
// as the forward pass, plus one of w c per channel.
__global__ void __launch_bounds__(kThreads)
vr_composite_bwd_kernel(const float* __restrict__ sigma, const float* __restrict__ logits,
                        const float* __restrict__ delta, const float* __restrict__ color,
                        const float* __restrict__ dcolor, int64_t R, int S, float* __restrict__ dsigma,
                        float* __restrict__ dlogits) {
  const int64_t r = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (r >= R) return;                                   // whole warps leave together
  const int lane = threadIdx.x & 31;
  const float dl = __ldg(delta + r);
  float Cc[3], dC[3], pc[3] = {0.f, 0.f, 0.f};          // colour, its gradient, P_{k-1} carried
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cc[c] = __ldg(color + r * 3 + c);
    dC[c] = __ldg(dcolor + r * 3 + c);
  }
  float carry = 0.f;
  for (int base = 0; base < S; base += 32) {
    const int k = base + lane;
    const int64_t i = r * S + k;
    float s = 0.f, col[3] = {0.f, 0.f, 0.f}, ncol[3] = {0.f, 0.f, 0.f};
    if (k < S) {
      s = __ldg(sigma + i) * dl;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float x = __ldg(logits + i * 3 + c);
        col[c] = 1.f / (1.f + expf(-x));
        ncol[c] = 1.f / (1.f + expf(x));                // 1 - c without cancellation near c = 1
      }
    }
    float incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    float excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.f;
    const float w = expf(-(carry + excl)) * -expm1f(-s);
    const float t_next = expf(-(carry + incl));         // T_{k+1}
    float wc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      wc[c] = w * col[c];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(0xffffffffu, wc[c], o);
        if (lane >= o) wc[c] += t;
      }
    }
    if (k < S) {
      float g = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float Pk = pc[c] + wc[c];                 // P_k, inclusive
        g = fmaf(dC[c], t_next * col[c] - (Cc[c] - Pk), g);
        dlogits[i * 3 + c] = dC[c] * w * col[c] * ncol[c];
      }
      dsigma[i] = dl * g;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) pc[c] += __shfl_sync(0xffffffffu, wc[c], 31);
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// Gradient of the density network's 16 outputs: the colour network's input gradient of the
// first 16 columns, plus dL/dsigma * sigma on output 0 below the clamp (sigma = exp(min(v_0, 15))).
__global__ void __launch_bounds__(kThreads)
vr_field_bwd_kernel(const float* __restrict__ dcin, const float* __restrict__ dsigma,
                    const float* __restrict__ sigma, const float* __restrict__ dens, int64_t P,
                    float* __restrict__ dv) {
  const int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= P) return;
  const float4* src = reinterpret_cast<const float4*>(dcin + p * 32);
  float4* dst = reinterpret_cast<float4*>(dv + p * 16);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float4 a = __ldg(src + j);
    if (j == 0 && __ldg(dens + p * 16) < 15.f) a.x = fmaf(__ldg(dsigma + p), __ldg(sigma + p), a.x);
    dst[j] = a;
  }
}

unsigned blocks(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

sxe_status launch_vr_samples(const float* o, const float* d, const float* tn, const float* tf, int64_t R, int S,
                             float* x, float* delta, cudaStream_t s) {
  vr_samples_kernel<<<blocks(R * S, kThreads), kThreads, 0, s>>>(o, d, tn, tf, R, S, x, delta);
  return check_launch("vr_samples");
}

sxe_status launch_vr_field(const float* dens, const float* dirs, int64_t R, int S, int dtype, float* sigma,
                           void* cin, cudaStream_t s) {
  const int64_t P = R * S;
  if (dtype == SXE_F16)
    vr_field_kernel<__half><<<blocks(P, kThreads), kThreads, 0, s>>>(dens, dirs, P, S, sigma, (__half*)cin);
  else
    vr_field_kernel<__nv_bfloat16><<<blocks(P, kThreads), kThreads, 0, s>>>(dens, dirs, P, S, sigma,
                                                                            (__nv_bfloat16*)cin);
  return check_launch("vr_field");
}

sxe_status launch_vr_composite(const float* sigma, const float* logits, const float* delta, int64_t R, int S,
                               float* color, float* trans, float* weights, cudaStream_t s) {
  vr_composite_kernel<<<blocks(R, kThreads / 32), kThreads, 0, s>>>(sigma, logits, delta, R, S, color, trans, weights);
  return check_launch("vr_composite");
}

sxe_status launch_vr_composite_bwd(const float* sigma, const float* logits, const float* delta, const float* color,
                                   const float* dcolor, int64_t R, int S, float* dsigma, float* dlogits,
                                   cudaStream_t s) {
  vr_composite_bwd_kernel<<<blocks(R, kThreads / 32), kThreads, 0, s>>>(sigma, logits, delta, color, dcolor, R, S,
                                                                         dsigma, dlogits);
  return check_launch("vr_composite_bwd");
}

sxe_status launch_vr_field_bwd(const float* dcin, const float* dsigma, const float* sigma, const float* dens,
                               int64_t P, float* dv, cudaStream_t s) {
  vr_field_bwd_kernel<<<blocks(P, kThreads), kThreads, 0, s>>>(dcin, dsigma, sigma, dens, P, dv);
  return check_launch("vr_field_bwd");
}

}  // namespace sxe
