// Three-tile network training pass for n_out <= 8 (the output layer's weights in registers), the
// dispatch by output width, and the per-device address of the tensor-core error word.
#include <mutex>

#include "mlp_tc3.cuh"

namespace sxe {

namespace {
std::mutex g_err_mu;
int* g_err_ptr[64];
bool g_err_known[64];
}  // namespace

// the device address of the tensor-core error word (per device, looked up once)
int* tc3_error_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_err_mu);
  if (!g_err_known[dev]) {
    g_err_ptr[dev] = tc_error_word();
    g_err_known[dev] = true;
  }
  return g_err_ptr[dev];
}

namespace {

// One bounded wait on a fresh mbarrier: with `timeout` set nobody arrives, so the wait runs out
__global__ void selftest_wait_kernel(int timeout, uint64_t limit_ns, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar, 1);
    if (!timeout) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(&mbar)) : "memory");
    const bool ok = tc::mbar_wait_sleep(&mbar, 0, 20000u, limit_ns, 1u << 20);
    if (!ok && err) atomicExch(err, 1);
  }
}

}  // namespace

sxe_status launch_selftest_wait(int timeout, int64_t limit_ns, cudaStream_t s) {
  int* err = tc3_error_word();
  if (!err) return set_error(SXE_ECUDA, "selftest_wait: no device error word");
  selftest_wait_kernel<<<1, 32, 0, s>>>(timeout, (uint64_t)limit_ns, err);
  return check_launch("selftest_wait");
}

bool mlp_tc3_applies(const sxe_mlp_desc* d) { return d->n_out <= 16; }

sxe_status launch_mlp_bwd_tc3(const sxe_mlp_desc* d, const void* W, const void* in, const float* dout,
                              const float* target, float loss_scale, int64_t P, float* din, float* dW, float* sq_sum,
                              float* ws, int grid, cudaStream_t s, int din_group, int64_t lc) {
  if (!mlp_tc3_applies(d)) return set_error(SXE_EUNSUPPORTED, "mlp_train_tc3: n_out=%d > 16", d->n_out);
  if (d->n_out > 8)
    return launch_mlp_bwd_tc3_wide(d, W, in, dout, target, loss_scale, P, din, dW, sq_sum, ws, grid, s, din_group, lc);
  return d->dtype == SXE_F16
             ? tc3_in<__half, 1>(d, W, in, dout, target, loss_scale, P, din, din_group, dW, sq_sum, ws, grid, s, lc)
             : tc3_in<__nv_bfloat16, 1>(d, W, in, dout, target, loss_scale, P, din, din_group, dW, sq_sum, ws, grid,
                                        s, lc);
}

}  // namespace sxe
