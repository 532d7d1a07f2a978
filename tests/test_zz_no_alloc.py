"""The allocation-free network step sxe_mlp_train_l2_static, called through the C ABI.

Some callers cannot allocate device memory (they run under another framework's allocator,
in a real-time loop, or while a stream is captured), so this entry point keeps its scratch
in a fixed array inside the library instead of a caller workspace.  It must give what
sxe_mlp_train_l2 gives with a workspace, on consecutive calls that reuse the array.  This
file is collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest
import torch

from paper_2311_15439_gb300 import synth

pytestmark = pytest.mark.gpu


def test_static_scratch_matches_workspace_entry(cuda_lib):
    from paper_2311_15439_gb300.api import Mlp
    from test_gpu_mlp import _dens, _round, within
    P, n_out = 50001, 3
    mlp = Mlp(32, n_out, n_hidden=2, dtype="f16")
    W_t, W = _round(mlp.init_weights(7), "f16")
    x_t, x = _round(synth.rng(8).uniform(-1, 1, size=(P, 32)), "f16")
    Wd, xd = W_t.cuda(), x_t.cuda()
    tgt = torch.from_numpy(synth.rng(9).random((P, n_out)).astype(np.float32)).cuda()
    ls = 2.0 ** 16
    ref_dW = torch.zeros((mlp.n_params,), device="cuda")
    ref_din = torch.empty((P, 32), device="cuda")
    ref_sq = torch.zeros((1,), device="cuda")
    mlp.mlp_train_l2(Wd, xd, tgt, ref_dW, ref_sq, din=ref_din, loss_scale=ls)
    # the same tolerance as the network parity tests: (2 NH + 2) u against magnitude bounds
    u = 2.0 ** -11
    tol = 6 * u
    Ws = mlp.split(W)
    yden = _dens(Ws, x, np.zeros((P, n_out)))[0]
    dy_bound = 2.0 * (yden + 1.0) / (P * n_out)                  # |y - t| <= |y| + 1 with t in [0, 1)
    _, dW_den, _ = _dens(Ws, x, dy_bound)
    for call in range(2):                         # two calls in a row share the static scratch
        dW = torch.zeros((mlp.n_params,), device="cuda")
        din = torch.empty((P, 32), device="cuda")
        sq = torch.full((1,), -1.0, device="cuda")
        mlp.mlp_train_l2_static(Wd, xd, tgt, dW, sq, din=din, loss_scale=ls)
        torch.cuda.synchronize()
        got, ref = mlp.split(dW.cpu().numpy()), mlp.split(ref_dW.cpu().numpy())
        for i in range(len(Ws)):
            assert within(got[i], ref[i], dW_den[i], tol) <= 1.0, "call %d layer %d" % (call, i)
        assert torch.equal(din, ref_din)          # the input gradient does not depend on the grid
        assert abs(sq.item() - ref_sq.item()) <= 1e-5 * ref_sq.item()


@pytest.mark.parametrize("kernel", ["mma_sync", "tcgen05", "tcgen05_pipelined", "tcgen05_3tile"])
def test_static_scratch_cuts_the_grid(cuda_lib, kernel):
    """A network large enough that the fixed array holds fewer per-CTA partial rows than the
    persistent grid the workspace entry point launches (the first of the candidates below for which
    that holds on this GPU; 2^21 / (weights + 1) rows fit): the static entry point then runs on the
    smaller grid, and its gradients still match the workspace entry point's (same products; only
    the summation order of the partials differs), on two calls in a row, under both network
    kernels."""
    import ctypes
    from paper_2311_15439_gb300 import _lib as L
    from paper_2311_15439_gb300.api import Mlp
    from test_gpu_mlp import _dens, _round, within
    code = {"mma_sync": L.SXE_MLP_KERNEL_MMA_SYNC, "tcgen05": L.SXE_MLP_KERNEL_TCGEN05,
            "tcgen05_pipelined": L.SXE_MLP_KERNEL_TCGEN05_PIPELINED, "tcgen05_3tile": L.SXE_MLP_KERNEL_TCGEN05_3TILE}[kernel]
    prev = L.lib().sxe_mlp_get_kernel()
    assert L.lib().sxe_mlp_set_kernel(code) == 0
    try:
        P = 1 << 18
        chosen = None
        for n_in, nh, n_out in ((32, 3, 16), (16, 3, 16), (32, 2, 16), (64, 2, 16), (64, 3, 16)):
            mlp = Mlp(n_in, n_out, n_hidden=nh, dtype="f16")
            capacity = (1 << 21) // (mlp.n_params + 1)
            grid = mlp.workspace_bytes(P) // (4 * (mlp.n_params + 1))
            if capacity < grid:
                chosen = (n_in, nh, n_out)
                break
        assert chosen is not None, "no candidate network has a grid above the array's capacity"
        n_in, nh, n_out = chosen
        W_t, W = _round(mlp.init_weights(11), "f16")
        x_t, x = _round(synth.rng(12).uniform(-1, 1, size=(P, n_in)), "f16")
        Wd, xd = W_t.cuda(), x_t.cuda()
        tgt = torch.from_numpy(synth.rng(13).random((P, n_out)).astype(np.float32)).cuda()
        ls = 2.0 ** 16
        ref_dW = torch.zeros((mlp.n_params,), device="cuda")
        ref_din = torch.empty((P, n_in), device="cuda")
        ref_sq = torch.zeros((1,), device="cuda")
        mlp.mlp_train_l2(Wd, xd, tgt, ref_dW, ref_sq, din=ref_din, loss_scale=ls)
        u = 2.0 ** -11
        tol = (2 * nh + 2) * u
        Ws = mlp.split(W)
        yden = _dens(Ws, x, np.zeros((P, n_out)))[0]
        _, dW_den, _ = _dens(Ws, x, 2.0 * (yden + 1.0) / (P * n_out))
        for call in range(2):
            dW = torch.zeros((mlp.n_params,), device="cuda")
            din = torch.empty((P, n_in), device="cuda")
            sq = torch.full((1,), -1.0, device="cuda")
            mlp.mlp_train_l2_static(Wd, xd, tgt, dW, sq, din=din, loss_scale=ls)
            torch.cuda.synchronize()
            got, ref = mlp.split(dW.cpu().numpy()), mlp.split(ref_dW.cpu().numpy())
            for i in range(len(Ws)):
                assert within(got[i], ref[i], dW_den[i], tol) <= 1.0, "%s %s call %d layer %d" % (kernel, chosen,
                                                                                                 call, i)
            assert torch.equal(din, ref_din)
            assert abs(sq.item() - ref_sq.item()) <= 1e-5 * ref_sq.item()
        flag = ctypes.c_int32(0)
        assert L.lib().sxe_device_error(ctypes.byref(flag), 1) == 0 and flag.value == 0
    finally:
        L.lib().sxe_mlp_set_kernel(prev)
