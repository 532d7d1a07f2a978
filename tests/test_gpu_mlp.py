"""GPU parity of the tensor-core network, its backward pass, the L2 loss and Adam.

Network results are compared with the FP64 oracle run on the same fp16/bf16 weights and
inputs, against an upper bound of the magnitudes involved (absolute weights and
activations propagated through the network, no ReLU masking).  The kernel rounds each
hidden activation and each delta to the operand type once, so a chain of at most
2*NH + 2 roundings of unit roundoff u (2^-11 fp16, 2^-8 bf16) bounds the relative error:
tolerance = (2*NH + 2) * u."""
import math

import numpy as np
import pytest
import torch

from conftest import record_error, rel_err
from oracle import adam as OA
from oracle import mlp as OM
from paper_2311_15439_gb300 import synth

pytestmark = pytest.mark.gpu

U = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
NP = {"f16": np.float16}


def _round(a, dt):
    t = torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.float16 if dt == "f16" else torch.bfloat16)
    return t, t.float().numpy().astype(np.float64)


def _dens(Ws, x, dy):
    """Magnitude bounds: forward |y| <= |W_L| ... |W_1| |x|; backward likewise."""
    h = [np.abs(x)]
    for W in Ws:
        h.append(h[-1] @ np.abs(W).T)
    d = np.abs(dy)
    dW = [None] * len(Ws)
    for i in reversed(range(len(Ws))):
        dW[i] = d.T @ h[i]
        d = d @ np.abs(Ws[i])
    return h[-1], dW, d


def flip_slack(Ws, x, dy, u, x_err=0.0):
    """Extra error the backward pass may show where a ReLU decision is ambiguous at the
    kernel's precision.  The kernel feeds each layer the previous activations rounded once
    to the operand type (unit roundoff u; exact inputs for the first layer), so a
    pre-activation z can differ from the oracle's by up to 2 u sum_i |h_i W_ji| (+ binary32
    accumulation); if |z| is inside that band the unit's mask may differ, which changes its
    delta by at most the full unmasked term |d_pre_j|.  ``x_err`` bounds how far the kernel's
    inputs may differ from ``x`` (zero when both read the same values).  Returns (dW slack
    list, din slack), propagated through |W| like the magnitude bounds; rows with no ambiguous
    unit get zero."""
    h = np.asarray(x, dtype=np.float64)
    habs = [np.abs(h)]
    amb = []
    for i, W in enumerate(Ws[:-1]):
        z = h @ W.T
        band = ((2.0 * u if i > 0 else 0.0) + 64 * 2.0 ** -24) * (np.abs(h) @ np.abs(W).T)
        if i == 0:
            band = band + np.broadcast_to(np.asarray(x_err, dtype=np.float64), h.shape) @ np.abs(W).T
        amb.append(np.abs(z) <= band)
        h = np.maximum(z, 0.0)
        habs.append(habs[-1] @ np.abs(W).T)
    d = np.abs(dy)
    slack = np.zeros_like(d)
    dW_slack = [None] * len(Ws)
    for i in reversed(range(len(Ws))):
        dW_slack[i] = slack.T @ habs[i]
        d_pre = d @ np.abs(Ws[i])
        s_pre = slack @ np.abs(Ws[i])
        if i > 0:
            slack = s_pre + d_pre * amb[i - 1]
            d = d_pre
        else:
            return dW_slack, s_pre


def _adam_err(name, got, want):
    """Record the Adam result's error as a fraction of 2e-6 |want| + 1e-7 (the binary32 bound)."""
    got, want = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    r = float(np.max(np.abs(got - want) / (2e-6 * np.abs(want) + 1e-7))) if got.size else 0.0
    record_error(name, r, 1.0, "2e-6 |value| + 1e-7")


def within(got, want, den, tol, slack=0.0):
    """max |got - want| / (tol den + slack); <= 1 means inside the bound everywhere."""
    bound = tol * np.asarray(den, dtype=np.float64) + slack
    err = np.abs(np.asarray(got, dtype=np.float64) - np.asarray(want, dtype=np.float64))
    return float(np.max(err / np.maximum(bound, 1e-300)))


@pytest.fixture(params=["mma_sync", "tcgen05", "tcgen05_pipelined", "tcgen05_3tile"])
def mlp_kernel(request, cuda_lib):
    """Run the test with the network's training pass on each kernel; afterwards no bounded
    device wait may have given up."""
    import ctypes
    L = cuda_lib
    code = {"mma_sync": L.SXE_MLP_KERNEL_MMA_SYNC, "tcgen05": L.SXE_MLP_KERNEL_TCGEN05,
            "tcgen05_pipelined": L.SXE_MLP_KERNEL_TCGEN05_PIPELINED,
            "tcgen05_3tile": L.SXE_MLP_KERNEL_TCGEN05_3TILE}[request.param]
    prev = L.lib().sxe_mlp_get_kernel()
    assert L.lib().sxe_mlp_set_kernel(code) == 0
    try:
        yield request.param
        torch.cuda.synchronize()
        flag = ctypes.c_int32(0)
        assert L.lib().sxe_device_error(ctypes.byref(flag), 1) == 0
        assert flag.value == 0
    finally:
        L.lib().sxe_mlp_set_kernel(prev)


# (n_in, n_hidden, n_out, dtype, P)
NETS = [(32, 2, 3, "f16", 4099), (32, 2, 3, "bf16", 2000), (32, 1, 1, "bf16", 3333), (16, 3, 16, "f16", 1000),
        (64, 1, 5, "f16", 257), (32, 2, 3, "f16", 1 << 16), (16, 2, 3, "f16", 3001), (64, 3, 8, "bf16", 1500),
        (32, 1, 16, "bf16", 2500)]
# the image workload's network at its full batch, in the launch configuration the benchmark times
FULL = (32, 2, 3, "f16", 1 << 18)


def _setup(net, seed=0):
    from paper_2311_15439_gb300.api import Mlp
    n_in, nh, n_out, dt, P = net
    mlp = Mlp(n_in, n_out, n_hidden=nh, dtype=dt)
    W_t, W = _round(mlp.init_weights(seed), dt)
    x_t, x = _round(synth.rng(seed + 1).uniform(-1, 1, size=(P, n_in)), dt)
    return mlp, W_t.cuda(), mlp.split(W), x_t.cuda(), x


@pytest.mark.parametrize("net", NETS, ids=lambda n: "in%d_h%d_out%d_%s_P%d" % n)
def test_forward(cuda_lib, net, mlp_kernel):
    """The forward pass and its hidden activations against the oracle (mma.sync under the
    mma_sync / tcgen05 / pipelined settings, the three-tile tcgen05 kernel's forward form under
    tcgen05_3tile)."""
    mlp, Wd, Ws, xd, x = _setup(net)
    nh, dt = net[1], net[3]
    act = torch.empty((nh, x.shape[0], 64), dtype=Wd.dtype, device="cuda")
    y = mlp.mlp_fwd(Wd, xd, act=act).cpu().numpy()
    ref, acts = OM.mlp_forward(Ws, x)
    yden, _, _ = _dens(Ws, x, np.zeros_like(ref))
    tol = (2 * nh + 2) * U[dt]
    assert record_error("mlp_fwd output, %s network (%s)" % (dt, mlp_kernel), rel_err(y, ref, yden), tol,
                        "magnitude bound |W|...|x| (+ fp16-ambiguous ReLU slack)") <= tol
    h = [np.abs(x)]
    for W in Ws[:-1]:
        h.append(h[-1] @ np.abs(W).T)
    for i in range(nh):
        assert rel_err(act[i].float().cpu().numpy(), acts[i + 1], h[i + 1]) <= tol


@pytest.mark.parametrize("net", NETS, ids=lambda n: "in%d_h%d_out%d_%s_P%d" % n)
def test_backward(cuda_lib, net, mlp_kernel):
    mlp, Wd, Ws, xd, x = _setup(net, seed=5)
    nh, dt = net[1], net[3]
    dy = synth.normal_grads(x.shape[0], net[2], 9).astype(np.float64)
    dW = torch.zeros((mlp.n_params,), device="cuda")
    din = torch.empty((x.shape[0], net[0]), device="cuda")
    mlp.mlp_bwd(Wd, xd, torch.from_numpy(dy.astype(np.float32)).cuda(), dW, din=din, loss_scale=1.0)
    _, acts = OM.mlp_forward(Ws, x)
    dW_ref, din_ref = OM.mlp_backward(Ws, acts, dy)
    _, dW_den, din_den = _dens(Ws, x, dy)
    dW_sl, din_sl = flip_slack(Ws, x, dy, U[dt])
    tol = (2 * nh + 2) * U[dt]
    got = mlp.split(dW.cpu().numpy())
    for i in range(len(Ws)):
        r = within(got[i], dW_ref[i], dW_den[i], tol, dW_sl[i])
        record_error("mlp_bwd weight gradient, %s network (%s)" % (dt, mlp_kernel), r * tol, tol, "magnitude bound |W|...|x| (+ fp16-ambiguous ReLU slack)")
        assert r <= 1.0, "layer %d" % i
    r = within(din.cpu().numpy(), din_ref, din_den, tol, din_sl)
    record_error("mlp_bwd input gradient, %s network (%s)" % (dt, mlp_kernel), r * tol, tol, "magnitude bound |W|...|x| (+ fp16-ambiguous ReLU slack)")
    assert r <= 1.0


def test_backward_accumulates_and_is_deterministic(cuda_lib, mlp_kernel):
    mlp, Wd, Ws, xd, x = _setup((32, 2, 3, "f16", 5000), seed=3)
    dy = torch.from_numpy(synth.normal_grads(5000, 3, 4)).cuda()
    a = torch.zeros((mlp.n_params,), device="cuda")
    b = torch.zeros((mlp.n_params,), device="cuda")
    mlp.mlp_bwd(Wd, xd, dy, a)
    mlp.mlp_bwd(Wd, xd, dy, b)
    assert torch.equal(a, b)                       # fixed-order reduction: bitwise repeatable
    mlp.mlp_bwd(Wd, xd, dy, a)
    torch.testing.assert_close(a, 2 * b, rtol=1e-6, atol=0)


@pytest.mark.parametrize("net", [NETS[0], NETS[2], NETS[5], NETS[6], NETS[7], NETS[8], FULL],
                         ids=lambda n: "in%d_h%d_out%d_%s_P%d" % n)
def test_train_l2(cuda_lib, net, mlp_kernel):
    """Fused forward + L2 loss + backward equals the oracle's loss and gradients, with the
    gradient scaled by a power of two before the fp16 rounding and unscaled after."""
    from paper_2311_15439_gb300.trainer import default_loss_scale
    mlp, Wd, Ws, xd, x = _setup(net, seed=21)
    n_in, nh, n_out, dt, P = net
    tgt = synth.rng(22).random((P, n_out)).astype(np.float32)
    dW = torch.zeros((mlp.n_params,), device="cuda")
    din = torch.empty((P, n_in), device="cuda")
    sq = torch.full((1,), 123.0, device="cuda")     # overwritten, not accumulated
    ls = default_loss_scale(P, n_out)
    mlp.mlp_train_l2(Wd, xd, torch.from_numpy(tgt).cuda(), dW, sq, din=din, loss_scale=ls)
    y, acts = OM.mlp_forward(Ws, x)
    loss, dy = OM.l2_loss(y, tgt)
    dW_ref, din_ref = OM.mlp_backward(Ws, acts, dy)
    tol = (2 * nh + 2) * U[dt]
    yden = _dens(Ws, x, dy)[0]
    # |dy| is bounded by 2 (|y| + |t|) / (P n_out); the squared residual's error by 3 tol (|y| + |t|)^2
    dy_bound = 2.0 * (yden + np.abs(tgt)) / dy.size
    _, dW_den, din_den = _dens(Ws, x, dy_bound)
    dW_sl, din_sl = flip_slack(Ws, x, dy_bound, U[dt])
    assert abs(sq.item() / (P * n_out) - loss) <= 3 * tol * np.mean((yden + np.abs(tgt)) ** 2)
    got = mlp.split(dW.cpu().numpy())
    for i in range(len(Ws)):
        r = within(got[i], dW_ref[i], dW_den[i], tol, dW_sl[i])
        record_error("mlp_train_l2 weight gradient, %s network (%s)" % (dt, mlp_kernel), r * tol, tol, "magnitude bound |W|...|x| (+ fp16-ambiguous ReLU slack)")
        assert r <= 1.0, "layer %d" % i
    r = within(din.cpu().numpy(), din_ref, din_den, tol, din_sl)
    record_error("mlp_train_l2 input gradient, %s network (%s)" % (dt, mlp_kernel), r * tol, tol, "magnitude bound |W|...|x| (+ fp16-ambiguous ReLU slack)")
    assert r <= 1.0


def test_loss_kernel(cuda_lib):
    from paper_2311_15439_gb300.api import loss_l2
    g = synth.rng(3)
    y = g.standard_normal((1000, 3)).astype(np.float32)
    t = g.random((1000, 3)).astype(np.float32)
    dy = torch.empty((1000, 3), device="cuda")
    sq = torch.zeros((1,), device="cuda")
    loss_l2(torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda(), dy, sq)
    ref_loss, ref_dy = OM.l2_loss(y, t)
    assert sq.item() / 3000 == pytest.approx(ref_loss, rel=1e-5)
    np.testing.assert_allclose(dy.cpu().numpy(), ref_dy, rtol=1e-6, atol=1e-12)


def _hp32():
    # the kernel works with the binary32 values of the hyper-parameters
    return dict(lr=float(np.float32(1e-2)), beta1=float(np.float32(0.9)), beta2=float(np.float32(0.99)),
                eps=float(np.float32(1e-15)))


@pytest.mark.parametrize("n,low_dt", [(10007, torch.float16), (10008, torch.float16), (10008, torch.bfloat16),
                                      (10008, torch.float32)])      # n % 4 == 0: the 16-byte-access kernel
@pytest.mark.parametrize("skip", [False, True])
def test_adam_dense(cuda_lib, skip, n, low_dt):
    from paper_2311_15439_gb300.api import Adam
    g = synth.rng(4)
    p = g.standard_normal(n).astype(np.float32)
    m = (g.standard_normal(n) * 0.1).astype(np.float32)
    v = (g.random(n) * 0.01).astype(np.float32)
    gr = (g.standard_normal(n) * (g.random(n) < 0.8)).astype(np.float32)
    dev = [torch.from_numpy(a.copy()).cuda() for a in (p, m, v, gr)]
    low = torch.empty(n, dtype=low_dt, device="cuda")
    Adam(1e-2, 0.9, 0.99, 1e-15, skip_zero_grad=skip).step(3, *dev, lowp=low)
    rp, rm, rv = OA.adam_step(p, gr, m, v, 3, skip_zero_grad=skip, **_hp32())
    for got, want in zip(dev[:3], (rp, rm, rv)):
        _adam_err("adam dense step (binary32 master)", got.cpu().numpy(), want)
        np.testing.assert_allclose(got.cpu().numpy(), want, rtol=2e-6, atol=1e-7)
    assert torch.equal(low, dev[0].to(low_dt))
    if skip:
        assert torch.all(dev[3] == 0)


@pytest.mark.parametrize("F,dt", [(2, "f16"), (2, "bf16"), (1, "f32"), (4, "f16"), (8, "f32")])
def test_adam_touched(cuda_lib, F, dt):
    """The bitmap-driven table step equals dense Adam with the zero-gradient skip rule."""
    from paper_2311_15439_gb300.api import Adam
    g = synth.rng(5 + F)
    n_entries = 4096 + 17
    marked = g.random(n_entries) < 0.3
    p = g.standard_normal((n_entries, F)).astype(np.float32)
    m = (g.standard_normal((n_entries, F)) * 0.1).astype(np.float32)
    v = (g.random((n_entries, F)) * 0.01).astype(np.float32)
    gr = (g.standard_normal((n_entries, F)) * marked[:, None]).astype(np.float32)
    gr[::7] = 0.0                                   # marked entries whose gradient is exactly zero
    state = torch.from_numpy(np.concatenate([p, m, v, gr], axis=1).copy()).cuda()
    words = np.zeros((n_entries + 31) // 32, dtype=np.uint32)
    for e in np.nonzero(marked)[0]:
        words[e >> 5] |= np.uint32(1 << (e & 31))
    touched = torch.from_numpy(words.view(np.int32).copy()).cuda()
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16, "f32": torch.float32}[dt]
    table = torch.from_numpy(p.copy()).to(tdt).cuda()
    Adam(1e-2, 0.9, 0.99, 1e-15).step_touched(5, state, touched, table, F)
    rp, rm, rv = OA.adam_step(p, gr, m, v, 5, skip_zero_grad=True, **_hp32())
    s = state.cpu().numpy()
    for got, want in ((s[:, :F], rp), (s[:, F:2 * F], rm), (s[:, 2 * F:3 * F], rv)):
        _adam_err("adam table step over marked entries (binary32 records)", got, want)
    np.testing.assert_allclose(s[:, :F], rp, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(s[:, F:2 * F], rm, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(s[:, 2 * F:3 * F], rv, rtol=2e-6, atol=1e-9)
    assert np.all(s[:, 3 * F:] == 0)
    assert torch.all(touched == 0)
    assert torch.equal(table[torch.from_numpy(marked).cuda()], state[:, :F][torch.from_numpy(marked).cuda()].to(tdt))


@pytest.mark.parametrize("net", [NETS[0], NETS[1], NETS[3], NETS[4], NETS[6], NETS[7], NETS[8]],
                         ids=lambda n: "in%d_h%d_out%d_%s_P%d" % n)
def test_tcgen05_and_mma_sync_agree(cuda_lib, net):
    """The two kernels compute the same products in the same precision: their gradients
    differ only by binary32 accumulation order (and the rare ReLU decision at a rounding tie)."""
    import ctypes
    L = cuda_lib
    mlp, Wd, Ws, xd, x = _setup(net, seed=31)
    dy = torch.from_numpy(synth.normal_grads(x.shape[0], net[2], 32)).cuda()
    outs = {}
    prev = L.lib().sxe_mlp_get_kernel()
    try:
        for k in (L.SXE_MLP_KERNEL_MMA_SYNC, L.SXE_MLP_KERNEL_TCGEN05, L.SXE_MLP_KERNEL_TCGEN05_PIPELINED,
                  L.SXE_MLP_KERNEL_TCGEN05_3TILE):
            assert L.lib().sxe_mlp_set_kernel(k) == 0
            dW = torch.zeros((mlp.n_params,), device="cuda")
            din = torch.empty((x.shape[0], net[0]), device="cuda")
            mlp.mlp_bwd(Wd, xd, dy, dW, din=din)
            outs[k] = (dW.cpu().numpy(), din.cpu().numpy())
    finally:
        L.lib().sxe_mlp_set_kernel(prev)
    flag = ctypes.c_int32(0)
    assert L.lib().sxe_device_error(ctypes.byref(flag), 1) == 0 and flag.value == 0
    _, dW_den, din_den = _dens(Ws, x, dy.cpu().numpy().astype(np.float64))
    dW_sl, din_sl = flip_slack(Ws, x, dy.cpu().numpy().astype(np.float64), U[net[3]])
    tol = (2 * net[1] + 2) * U[net[3]]
    a = outs[L.SXE_MLP_KERNEL_MMA_SYNC]
    for k in (L.SXE_MLP_KERNEL_TCGEN05, L.SXE_MLP_KERNEL_TCGEN05_PIPELINED, L.SXE_MLP_KERNEL_TCGEN05_3TILE):
        b = outs[k]
        for i, (ga, gb) in enumerate(zip(mlp.split(a[0]), mlp.split(b[0]))):
            assert within(gb, ga, dW_den[i], tol, 2 * dW_sl[i]) <= 1.0, "kernel %d layer %d" % (k, i)
        assert within(b[1], a[1], din_den, tol, 2 * din_sl) <= 1.0


def test_adam_touched_full_size_table(cuda_lib):
    """The bitmap-driven table step at the image workload's full table (L = 16, T = 2^22, F = 2:
    67 M entries, 2 GiB of state records, fp16 table), in the launch configuration the benchmark
    times: a seeded sample of 200 K entries (marked and unmarked) against the oracle's Adam."""
    from paper_2311_15439_gb300.api import Adam
    n, F = 16 << 22, 2
    gen = torch.Generator(device="cuda").manual_seed(123)
    state = torch.empty((n, 4 * F), device="cuda")
    state[:, :F].normal_(generator=gen)
    state[:, F:2 * F].normal_(generator=gen).mul_(0.1)
    state[:, 2 * F:3 * F].uniform_(0.0, 0.01, generator=gen)
    marked = torch.rand(n, device="cuda", generator=gen) < 0.1
    state[:, 3 * F:].normal_(generator=gen).mul_(marked[:, None])
    state[::11, 3 * F:] = 0.0                        # some marked entries with an exactly zero gradient
    words = (marked.view(-1, 32).to(torch.int64) << torch.arange(32, device="cuda")).sum(dim=1)
    touched = (words - ((words >= (1 << 31)).to(torch.int64) << 32)).to(torch.int32)   # same 32 bits
    table = state[:, :F].to(torch.float16)
    idx = torch.from_numpy(synth.rng(124).choice(n, 200_000, replace=False)).cuda()
    before = state[idx].cpu().numpy()
    was_marked = marked[idx].cpu().numpy()
    Adam(1e-2, 0.9, 0.99, 1e-15).step_touched(5, state, touched, table, F)
    torch.cuda.synchronize()
    after = state[idx].cpu().numpy()
    p, m, v, g = (before[:, k * F:(k + 1) * F].astype(np.float64) for k in range(4))
    rp, rm, rv = OA.adam_step(p, g, m, v, 5, skip_zero_grad=True, **_hp32())
    np.testing.assert_allclose(after[:, :F], rp, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(after[:, F:2 * F], rm, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(after[:, 2 * F:3 * F], rv, rtol=2e-6, atol=1e-9)
    assert np.all(after[:, 3 * F:] == 0)
    assert int((touched != 0).sum().item()) == 0
    tab = table[idx].cpu().numpy()
    np.testing.assert_array_equal(tab[was_marked], after[was_marked, :F].astype(np.float16))
    assert was_marked.sum() > 15_000 and (~was_marked).sum() > 150_000


def test_bounded_wait_gives_up_and_the_context_stays_usable(cuda_lib):
    """The bounded mbarrier wait every tcgen05 kernel uses, on a barrier nothing arrives at: it
    gives up after its limit (50 ms here) and raises the device error word instead of hanging; the
    word clears, a wait whose phase completes leaves it clear, and the network's training pass
    still runs and matches its own earlier result afterwards."""
    import ctypes
    import time
    L = cuda_lib
    lib = L.lib()
    mlp, Wd, Ws, xd, x = _setup(NETS[0], seed=41)
    dy = torch.from_numpy(synth.normal_grads(x.shape[0], NETS[0][2], 42)).cuda()
    before = torch.zeros((mlp.n_params,), device="cuda")
    mlp.mlp_bwd(Wd, xd, dy, before)
    torch.cuda.synchronize()
    flag = ctypes.c_int32(0)
    assert lib.sxe_device_error(ctypes.byref(flag), 1) == 0 and flag.value == 0
    t0 = time.perf_counter()
    assert lib.sxe_selftest_wait(1, 50_000_000, None) == 0
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 >= 0.045                      # it waited out its limit
    assert lib.sxe_device_error(ctypes.byref(flag), 1) == 0 and flag.value == 1
    assert lib.sxe_device_error(ctypes.byref(flag), 0) == 0 and flag.value == 0   # cleared
    assert lib.sxe_selftest_wait(0, 50_000_000, None) == 0
    torch.cuda.synchronize()
    assert lib.sxe_device_error(ctypes.byref(flag), 1) == 0 and flag.value == 0
    after = torch.zeros((mlp.n_params,), device="cuda")
    mlp.mlp_bwd(Wd, xd, dy, after)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    assert lib.sxe_device_error(ctypes.byref(flag), 1) == 0 and flag.value == 0


@pytest.mark.parametrize("net", [NETS[0], NETS[3], NETS[5], NETS[8]], ids=lambda n: "in%d_h%d_out%d_%s_P%d" % n)
def test_forward_kernels_agree(cuda_lib, net):
    """The three-tile tcgen05 forward and the mma.sync forward compute the same products in the
    same precision: outputs and hidden activations within the accumulation-order bound of their
    depth against the magnitude bound |W|...|x|."""
    L = cuda_lib
    mlp, Wd, Ws, xd, x = _setup(net, seed=77)
    nh = net[1]
    outs = {}
    prev = L.lib().sxe_mlp_get_kernel()
    try:
        for k in (L.SXE_MLP_KERNEL_MMA_SYNC, L.SXE_MLP_KERNEL_TCGEN05_3TILE):
            assert L.lib().sxe_mlp_set_kernel(k) == 0
            act = torch.empty((nh, x.shape[0], 64), dtype=Wd.dtype, device="cuda")
            y = mlp.mlp_fwd(Wd, xd, act=act)
            outs[k] = (y.cpu().numpy(), act.float().cpu().numpy())
    finally:
        L.lib().sxe_mlp_set_kernel(prev)
    (ya, aa), (yb, ab) = outs[L.SXE_MLP_KERNEL_MMA_SYNC], outs[L.SXE_MLP_KERNEL_TCGEN05_3TILE]
    yden, _, _ = _dens(Ws, x, np.zeros_like(ya, dtype=np.float64))
    u = U[net[3]]
    assert np.all(np.abs(yb - ya) <= (2 * nh + 2) * u * yden + 1e-30)
    h = [np.abs(x)]
    for W in Ws[:-1]:
        h.append(h[-1] @ np.abs(W).T)
    for i in range(nh):                              # hidden layer i: within the bound of its depth
        assert np.all(np.abs(ab[i] - aa[i]) <= (2 * i + 4) * u * h[i + 1] + 2.0 ** -24), "layer %d" % i


def test_empty_batch(cuda_lib, mlp_kernel):
    """No points: every L2 entry point sets the squared-residual sum to zero (the sum over an empty
    batch) and leaves the accumulated weight gradient as it was; the forward returns no rows; the
    bare backward writes nothing."""
    import ctypes
    from paper_2311_15439_gb300 import _lib as L
    net = (32, 2, 3, "f16", 0)
    mlp, Wd, Ws, xd, x = _setup(net, seed=63)
    tgt = torch.zeros((0, 3), device="cuda")
    din = torch.empty((0, 32), device="cuda")
    ws = mlp.workspace(1, "cuda")
    dW = torch.full((mlp.n_params,), 7.0, device="cuda")
    sq = torch.full((1,), -1.0, device="cuda")
    mlp.mlp_train_l2(Wd, xd, tgt, dW, sq, din=din, workspace=ws)
    torch.cuda.synchronize()
    assert sq.item() == 0.0 and bool((dW == 7.0).all())
    sq.fill_(-1.0)
    mlp.mlp_train_l2_static(Wd, xd, tgt, dW, sq, din=din)
    torch.cuda.synchronize()
    assert sq.item() == 0.0 and bool((dW == 7.0).all())
    sq.fill_(-1.0)
    mlp.mlp_train_l2_part(Wd, xd, tgt, dW, sq, 1024, din=din, workspace=ws)
    torch.cuda.synchronize()
    assert sq.item() == 0.0 and bool((dW == 7.0).all())
    sq.fill_(-1.0)
    st = L.lib().sxe_mlp_train_l2_grouped(ctypes.byref(mlp.desc), Wd.data_ptr(), xd.data_ptr(), None, 1.0, 0, None,
                                          2, dW.data_ptr(), sq.data_ptr(), ws.data_ptr(), ws.numel() * 4, None)
    torch.cuda.synchronize()
    assert st == 0 and sq.item() == 0.0 and bool((dW == 7.0).all())
    assert mlp.mlp_fwd(Wd, xd).shape == (0, 3)
    mlp.mlp_bwd(Wd, xd, torch.zeros((0, 3), device="cuda"), dW, din=din, workspace=ws)
    torch.cuda.synchronize()
    assert bool((dW == 7.0).all())


@pytest.mark.parametrize("P", [1, 127, 129, 383])
def test_tiny_batches(cuda_lib, P, mlp_kernel):
    """Batches of one point, just under and over one 128-point tile, and a few tiles with a ragged
    tail: the training pass and the forward match the oracle under every kernel setting (groups
    and CTAs without a tile contribute nothing)."""
    from paper_2311_15439_gb300.trainer import default_loss_scale
    net = (32, 2, 3, "f16", P)
    mlp, Wd, Ws, xd, x = _setup(net, seed=61)
    tgt = synth.rng(62).random((P, 3)).astype(np.float32)
    dW = torch.zeros((mlp.n_params,), device="cuda")
    din = torch.empty((P, 32), device="cuda")
    sq = torch.zeros((1,), device="cuda")
    mlp.mlp_train_l2(Wd, xd, torch.from_numpy(tgt).cuda(), dW, sq, din=din, loss_scale=default_loss_scale(P, 3))
    y, acts = OM.mlp_forward(Ws, x)
    loss, dy = OM.l2_loss(y, tgt)
    dW_ref, din_ref = OM.mlp_backward(Ws, acts, dy)
    tol = 6 * U["f16"]
    yden = _dens(Ws, x, dy)[0]
    dy_bound = 2.0 * (yden + np.abs(tgt)) / dy.size
    _, dW_den, din_den = _dens(Ws, x, dy_bound)
    dW_sl, din_sl = flip_slack(Ws, x, dy_bound, U["f16"])
    got = mlp.split(dW.cpu().numpy())
    for i in range(len(Ws)):
        assert within(got[i], dW_ref[i], dW_den[i], tol, dW_sl[i]) <= 1.0, "layer %d" % i
    assert within(din.cpu().numpy(), din_ref, din_den, tol, din_sl) <= 1.0
    assert abs(sq.item() / (P * 3) - loss) <= 3 * tol * np.mean((yden + np.abs(tgt)) ** 2)
    yf = mlp.mlp_fwd(Wd, xd).cpu().numpy()
    assert rel_err(yf, y, yden) <= tol
