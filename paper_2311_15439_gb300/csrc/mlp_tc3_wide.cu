// Three-tile network training pass for 8 < n_out <= 16: the output layer's weights read from
// shared memory with ldmatrix, two 8-wide tiles of outputs.
#include "mlp_tc3.cuh"

namespace sxe {

sxe_status launch_mlp_bwd_tc3_wide(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                                   const float* target, float loss_scale, int64_t P, float* din, float* dW,
                                   float* sq_sum, float* ws, int grid, cudaStream_t s, int din_group, int64_t lc) {
  return d->dtype == SXE_F16
             ? tc3_in<__half, 2>(d, W, in, dout, target, loss_scale, P, din, din_group, dW, sq_sum, ws, grid, s, lc)
             : tc3_in<__nv_bfloat16, 2>(d, W, in, dout, target, loss_scale, P, din, din_group, dW, sq_sum, ws, grid,
                                        s, lc);
}

}  // namespace sxe
