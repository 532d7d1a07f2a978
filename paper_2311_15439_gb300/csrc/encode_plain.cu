// Plain binary32 simplex encoding: the straightforward GPU form of the method that the
// optimised kernels are measured against.  One thread per point loops over the levels;
// the fractional parts are ordered with the bubble sort the paper uses (Sec. 4.2
// footnote: n is small), the vertices are walked one axis at a time (Remark 2), every
// feature is a separate scalar load, every gradient term a separate scalar atomic.
// Same lattice arithmetic and the same results as the optimised kernels.
#include "sxe_internal.cuh"

namespace sxe {
namespace {

template <int D>
__device__ __forceinline__ uint32_t hash_of(const uint32_t (&v)[D], uint32_t mask) {
  uint32_t h = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) h ^= v[i] * hash_prime(i);
  return h & mask;
}

// Vertices and weights of one level, walk order (base vertex first).
template <int D>
__device__ void plain_level(const float* xp, float s, float skewF, uint32_t mask, uint32_t* slot, float* w) {
  float p[D], f[D];
  uint32_t c[D];
  int idx[D];
  float sigma = 0.f;
  for (int i = 0; i < D; ++i) {
    p[i] = __fmul_rn(xp[i], s);
    sigma = i == 0 ? p[0] : __fadd_rn(sigma, p[i]);
  }
  const float t = __fmul_rn(skewF, sigma);
  for (int i = 0; i < D; ++i) {
    const float q = __fadd_rn(p[i], t);
    const float fl = floorf(q);
    f[i] = __fsub_rn(q, fl);
    c[i] = (uint32_t)__float2int_rz(fl);
    idx[i] = i;
  }
  // bubble sort of the axes by fractional part, decreasing; equal values keep axis order
  for (int a = 0; a < D - 1; ++a)
    for (int b = 0; b < D - 1 - a; ++b)
      if (f[idx[b]] < f[idx[b + 1]]) {
        const int tmp = idx[b];
        idx[b] = idx[b + 1];
        idx[b + 1] = tmp;
      }
  slot[0] = hash_of<D>(c, mask);
  w[0] = __fsub_rn(1.f, f[idx[0]]);
  for (int k = 1; k <= D; ++k) {
    c[idx[k - 1]] += 1u;
    slot[k] = hash_of<D>(c, mask);
    w[k] = k < D ? __fsub_rn(f[idx[k - 1]], f[idx[k]]) : f[idx[D - 1]];
  }
}

template <int D>
__global__ void encode_plain_fwd_kernel(const float* __restrict__ x, int64_t P, const float* __restrict__ tables,
                                        float* __restrict__ out, int F, const EncParams prm) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const uint32_t mask = (1u << prm.log2_T) - 1u;
  const int L = prm.n_levels;
  for (int l = 0; l < L; ++l) {
    uint32_t slot[D + 1];
    float w[D + 1];
    plain_level<D>(x + p * D, prm.scale[l], prm.skew_F, mask, slot, w);
    const float* tab = tables + ((int64_t)l << prm.log2_T) * F;
    for (int f = 0; f < F; ++f) {
      float acc = 0.f;
      for (int k = 0; k <= D; ++k) acc = fmaf(w[k], tab[(int64_t)slot[k] * F + f], acc);
      out[(p * L + l) * F + f] = acc;
    }
  }
}

template <int D>
__global__ void encode_plain_bwd_kernel(const float* __restrict__ x, int64_t P, const float* __restrict__ dout,
                                        float* __restrict__ grad, int F, const EncParams prm) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const uint32_t mask = (1u << prm.log2_T) - 1u;
  const int L = prm.n_levels;
  for (int l = 0; l < L; ++l) {
    uint32_t slot[D + 1];
    float w[D + 1];
    plain_level<D>(x + p * D, prm.scale[l], prm.skew_F, mask, slot, w);
    float* g = grad + ((int64_t)l << prm.log2_T) * F;
    for (int k = 0; k <= D; ++k)
      for (int f = 0; f < F; ++f) atomicAdd(g + (int64_t)slot[k] * F + f, w[k] * dout[(p * L + l) * F + f]);
  }
}

}  // namespace

sxe_status launch_encode_plain(const sxe_encoder* e, bool backward, const float* x, int64_t P, const float* a,
                               float* b, cudaStream_t s) {
  const unsigned g = (unsigned)((P + 127) / 128);
  const int F = e->desc.n_features;
#define SXE_PLAIN(DD)                                                                           \
  case DD:                                                                                      \
    if (backward) encode_plain_bwd_kernel<DD><<<g, 128, 0, s>>>(x, P, a, b, F, e->prm);         \
    else encode_plain_fwd_kernel<DD><<<g, 128, 0, s>>>(x, P, a, b, F, e->prm);                  \
    break;
  switch (e->desc.d) {
    SXE_PLAIN(2)
    SXE_PLAIN(3)
    SXE_PLAIN(4)
    SXE_PLAIN(5)
  }
#undef SXE_PLAIN
  return check_launch(backward ? "encode_plain_bwd" : "encode_plain_fwd");
}

}  // namespace sxe
