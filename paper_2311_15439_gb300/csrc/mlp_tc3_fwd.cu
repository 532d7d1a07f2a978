// Forward-only form of the three-tile tcgen05 network kernel (inference: sxe_mlp_fwd for networks
// with n_out <= 16): the tile's forward chain on tcgen05, the output layer on mma.sync, the
// outputs (and optionally the hidden activations) written to global memory.
#include "mlp_tc3.cuh"

namespace sxe {

sxe_status launch_mlp_fwd_tc3(const sxe_mlp_desc* d, const void* W, const void* in, int64_t P, float* out,
                              void* act, cudaStream_t s) {
  if (d->n_out > 16) return set_error(SXE_EUNSUPPORTED, "mlp_fwd_tc3: n_out=%d > 16", d->n_out);
  if (d->n_out <= 8)
    return d->dtype == SXE_F16 ? tc3_fwd_in<__half, 1>(d, W, in, P, out, act, s)
                               : tc3_fwd_in<__nv_bfloat16, 1>(d, W, in, P, out, act, s);
  return d->dtype == SXE_F16 ? tc3_fwd_in<__half, 2>(d, W, in, P, out, act, s)
                             : tc3_fwd_in<__nv_bfloat16, 2>(d, W, in, P, out, act, s);
}

}  // namespace sxe
