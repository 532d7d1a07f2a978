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
