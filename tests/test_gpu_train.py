"""GPU parity of the full training step (encode -> network + L2 -> encode backward -> Adam)
and of the autograd wrappers."""
import numpy as np
import pytest
import torch

from conftest import record_error, rel_err
from oracle import adam as OA
from oracle import encoding as OE
from oracle import mlp as OM
from paper_2311_15439_gb300 import synth

pytestmark = pytest.mark.gpu

CFG = dict(d=2, n_levels=8, n_features=2, log2_T=12, base_res=16.0, growth=1.5)


def _make(P=4096, seed=0, table_dtype="f16", layout="auto", cfg=None):
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import Trainer
    enc = Encoder(**(cfg or CFG), table_dtype=table_dtype)
    mlp = Mlp(16, 3, n_hidden=2, dtype="f16")
    return Trainer(enc, mlp, P, seed=seed, table_layout=layout)


@pytest.mark.parametrize("layout", ["records", "dense"])
def test_one_step_matches_oracle(layout):
    """Gradients of one step against the oracle pipeline: encode (FP64, rounded to the fp16
    encoding the network consumes), network + L2 loss and backward (FP64), scatter-add of
    dL/d(encoding) into the tables (FP64); then the Adam step of every table entry whose
    gradient sign is unambiguous, and of every network weight likewise; for both table layouts
    (interleaved records + touched bitmap, dense arrays).  2^15 points on levels up to resolution
    2048 (growth 2.0) and T = 2^17, so that most entries receive the terms of few points and over
    5000 updated entries are compared (a point with an fp16-ambiguous ReLU decision, about a
    third of them, makes every entry it touches ambiguous)."""
    from paper_2311_15439_gb300.build import build
    build()
    P = 1 << 15
    cfg = dict(d=2, n_levels=8, n_features=2, log2_T=17, base_res=16.0, growth=2.0)
    tr = _make(P, layout=layout, cfg=cfg)
    assert tr.tab.layout == layout
    x = synth.uniform_points(P, 2, 5)
    tgt = synth.ProceduralImage(6, size=4096, n_waves=16).sample(x)
    F, L, log2_T, growth = 2, 8, 17, 2.0
    T = 1 << log2_T
    # the oracle regenerates the seeded initial values on the host and rounds them itself
    p_tab0 = synth.uniform_tables(L, T, F, 0, dtype="f32", scale=1e-4)[0].reshape(L * T, F).astype(np.float64)
    tables = p_tab0.astype(np.float16).astype(np.float64).reshape(L, T, F)
    W0 = tr.mlp.init_weights(1).astype(np.float64)
    W = [w.astype(np.float16).astype(np.float64) for w in tr.mlp.split(W0)]

    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda()
    # run the first three stages of the step and stop before the optimiser
    tr.tab.forward(xd, tr.enc_out)
    tr.mlp.mlp_train_l2(tr.W_lowp, tr.enc_out, td, tr.dW, tr.sq_sum, din=tr.d_enc, loss_scale=tr.loss_scale,
                        workspace=tr.ws)
    tr.tab.backward(xd, tr.d_enc)
    g_tab = tr.table_grads().reshape(L * T, F).cpu().numpy().copy()
    g_W = tr.dW.cpu().numpy().copy()
    loss_gpu = tr.loss()

    enc = OE.simplex_encode(x, tables, base_res=16.0, growth=growth)
    enc16 = enc.astype(np.float16).astype(np.float64)          # the encoding dtype the network reads
    y, acts = OM.mlp_forward(W, enc16)
    loss, dy = OM.l2_loss(y, tgt)
    dW_ref, denc = OM.mlp_backward(W, acts, dy)
    g_ref, g_den = OE.simplex_encode_bwd(x, denc, n_levels=L, log2_T=log2_T, n_features=F, base_res=16.0,
                                         growth=growth, with_denominator=True)
    # magnitude bound of dL/d(encoding): |dy| through |W|
    d = 2 * (np.abs(y) + np.abs(tgt)) / dy.size
    for Wi in reversed(W):
        d = d @ np.abs(Wi)
    _, den_bound = OE.simplex_encode_bwd(x, d, n_levels=L, log2_T=log2_T, n_features=F, base_res=16.0,
                                         growth=growth, with_denominator=True)
    tol = 6 * 2.0 ** -11
    assert abs(loss_gpu - loss) <= 3 * tol * loss + 1e-6
    # ReLU decisions that are ambiguous at fp16 widen the bound of the entries they feed
    from test_gpu_mlp import flip_slack, within
    # the kernel's fp16 encoding may differ from the oracle's rounded one by one fp16 rounding
    # (relative 2^-11, or 2^-25 absolute in the subnormal range these small tables produce)
    enc_err = 2.0 ** -11 * np.abs(enc16) + 2.0 ** -25
    _, denc_slack = flip_slack(W, enc16, 2 * (np.abs(y) + np.abs(tgt)) / dy.size, 2.0 ** -11, x_err=enc_err)
    _, slack = OE.simplex_encode_bwd(x, denc_slack, n_levels=L, log2_T=log2_T, n_features=F, base_res=16.0,
                                     growth=growth, with_denominator=True)
    assert np.all(np.isfinite(g_tab))
    for l in range(L):
        r = within(g_tab[l * T:(l + 1) * T], g_ref[l], den_bound[l], tol, slack[l])
        record_error("training step: table gradient through encode + network (%s)" % layout, r * tol, tol,
                     "magnitude bound of dL/d(encoding) scattered (+ ReLU slack)")
        assert r <= 1.0, "level %d" % l
    shaky = np.concatenate([slack[l] for l in range(L)]) > 0

    # optimiser: Adam at t = 1 moves each parameter by -lr * g / (|g| + eps); compare where the
    # sign of the gradient is unambiguous (|g_ref| well above the tolerance)
    tr.adam_tables.advance(tr.t_dev, tr.corrections)                 # t = 1 on the device
    tr.tab.adam(tr.adam_tables, tr.corrections)
    tr.adam_mlp.step(1, tr.W, tr.mW, tr.vW, tr.dW, lowp=tr.W_lowp)
    hp = dict(lr=float(np.float32(1e-2)), beta1=float(np.float32(0.9)), beta2=float(np.float32(0.99)),
              eps=float(np.float32(1e-15)))
    g_all = np.concatenate([g_ref[l] for l in range(L)])
    den_all = np.concatenate([den_bound[l] for l in range(L)])
    p_ref, _, _ = OA.adam_step(p_tab0, g_all, np.zeros_like(g_all), np.zeros_like(g_all), 1, skip_zero_grad=True, **hp)
    clear = ((np.abs(g_all) > 4 * tol * den_all) | (den_all == 0)) & ~shaky
    p_gpu = tr.table_params().reshape(L * T, F).cpu().numpy()
    record_error("training step: Adam table update at t = 1 (%s)" % layout,
                 np.max(np.abs(p_gpu[clear] - p_ref[clear])), 2e-6, "absolute")
    np.testing.assert_allclose(p_gpu[clear], p_ref[clear], rtol=0, atol=2e-6)
    assert (clear & (den_all > 0)).sum() > 5000          # the comparison covers many updated entries
    gW_ref = np.concatenate([a.ravel() for a in dW_ref])
    W_ref, _, _ = OA.adam_step(W0, gW_ref, np.zeros_like(W0), np.zeros_like(W0), 1, skip_zero_grad=False, **hp)
    clearW = np.abs(gW_ref) > 1e-2 * np.abs(gW_ref).max()
    record_error("training step: Adam network update at t = 1", np.max(np.abs(tr.W.cpu().numpy()[clearW] -
                                                                        W_ref[clearW])), 1e-5, "absolute")
    np.testing.assert_allclose(tr.W.cpu().numpy()[clearW], W_ref[clearW], rtol=0, atol=1e-5)
    assert np.abs(g_W - gW_ref).max() <= tol * np.abs(gW_ref).max() * 4


@pytest.mark.parametrize("kind,d", [("simplex", 2), ("simplex", 3), ("grid", 2), ("grid", 3)])
def test_forward_marks_the_entries_the_backward_marks(kind, d):
    """``sxe_encode_fwd_marked`` sets exactly the touched bits that the backward of the same points
    sets (every vertex slot of every level), and its encoding equals the unmarked forward's bit
    for bit; marking into a bitmap that already holds bits only adds the missing ones."""
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.build import build
    build()
    cfg = dict(CFG, d=d, n_levels=6, log2_T=13)
    enc = Encoder(kind=kind, **cfg, table_dtype="f16")
    L, T, F = 6, 1 << 13, 2
    P = 3000 + 17                                            # several blocks and a ragged tail
    tables = torch.from_numpy(synth.uniform_tables(L, T, F, 3, dtype="f32", scale=1e-1)[0]).half().cuda()
    x = torch.from_numpy(synth.uniform_points(P, d, 41)).cuda()
    words = (L * T + 31) // 32
    t_fwd = torch.zeros((words,), dtype=torch.int32, device="cuda")
    t_bwd = torch.zeros_like(t_fwd)
    out_plain = enc.encode_fwd(x, tables)
    out_marked = enc.encode_fwd(x, tables, touched=t_fwd)
    assert torch.equal(out_plain, out_marked)
    state = torch.zeros((L * T, 4 * F), dtype=torch.float32, device="cuda")
    dout = torch.ones((P, L * F), dtype=torch.float32, device="cuda")
    enc.encode_bwd(x, dout, state, grad_stride=4 * F, grad_offset=3 * F, touched=t_bwd)
    torch.cuda.synchronize()
    assert torch.equal(t_fwd, t_bwd)
    n_set = int(sum(bin(w & 0xFFFFFFFF).count("1") for w in t_fwd.cpu().tolist()))
    assert 0 < n_set < L * T
    # a second pass over other points adds their bits to those already set
    x2 = torch.from_numpy(synth.uniform_points(500, d, 42)).cuda()
    enc.encode_fwd(x2, tables, touched=t_fwd)
    enc.encode_bwd(x2, dout[:500], state, grad_stride=4 * F, grad_offset=3 * F, touched=t_bwd)
    torch.cuda.synchronize()
    assert torch.equal(t_fwd, t_bwd)
    # an empty batch marks nothing
    before = t_fwd.clone()
    enc.encode_fwd(x[:0], tables, touched=t_fwd)
    torch.cuda.synchronize()
    assert torch.equal(before, t_fwd)


def test_marking_in_forward_trains_like_marking_in_backward():
    """The records-layout step with the touched entries marked in the forward trains like the step
    that marks them in the backward (parameters equal up to the order of the binary32 atomics);
    Adam clears every bit either way."""
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import Trainer
    P = 4096
    mk = lambda mark: Trainer(Encoder(**CFG, table_dtype="f16"), Mlp(16, 3, n_hidden=2, dtype="f16"), P, seed=21,
                              table_layout="records", mark_touched_in_forward=mark)
    a, b = mk(True), mk(False)
    assert a.tab.mark_in_forward and not b.tab.mark_in_forward
    img = synth.ProceduralImage(4, size=1024, n_waves=4)
    for i in range(4):
        x = synth.uniform_points(P, 2, 120 + i)
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(img.sample(x)).cuda()
        a.step(xd, td)
        b.step(xd, td)
    torch.cuda.synchronize()
    assert int(a.touched.abs().sum().item()) == 0 and int(b.touched.abs().sum().item()) == 0
    _close_up_to_atomics(a.W, b.W, steps=4, atol=1e-5)
    _close_up_to_atomics(a.state, b.state, steps=4)
    a.set_table_chunks(3)                                    # level ranges mark in their backward
    assert not a.tab.mark_in_forward
    a.set_table_chunks(1)
    assert a.tab.mark_in_forward


def test_training_reduces_loss():
    """Fitting the procedural image with the full step drives the L2 loss down."""
    P = 1 << 14
    tr = _make(P, seed=3)
    img = synth.ProceduralImage(7, size=2048, n_waves=8)
    losses = []
    for it in range(60):
        x = synth.uniform_points(P, 2, 100 + it)
        tr.step(torch.from_numpy(x).cuda(), torch.from_numpy(img.sample(x)).cuda())
        if it in (0, 59):
            losses.append(tr.loss())
    assert losses[1] < 0.5 * losses[0]


def test_step_is_repeatable():
    """Two trainers with the same seed and batches end bitwise identical (forward has no
    atomics; the table gradient atomics may reorder, so compare the parameters within the
    Adam step's sensitivity and the loss exactly for the first step)."""
    P = 2048
    a, b = _make(P, seed=9), _make(P, seed=9)
    x = synth.uniform_points(P, 2, 1)
    tgt = synth.ProceduralImage(2, size=1024, n_waves=4).sample(x)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda()
    a.step(xd, td)
    b.step(xd, td)
    assert a.loss() == b.loss()
    assert torch.equal(a.W, b.W)


def test_autograd_encoding_matches_oracle_and_fd():
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.autograd import encode
    enc = Encoder(3, 6, 2, 12, 8.0, 1.5, table_dtype="f32")
    vals = synth.uniform_tables(6, 1 << 12, 2, 4, scale=1.0)[0]
    H = torch.from_numpy(vals).cuda().requires_grad_(True)
    x = synth.uniform_points(1500, 3, 5)
    D = synth.normal_grads(1500, 12, 6)
    out = encode(torch.from_numpy(x).cuda(), H, enc)
    (out * torch.from_numpy(D).cuda()).sum().backward()
    g = H.grad.cpu().numpy()
    ref, den = OE.simplex_encode_bwd(x, D, n_levels=6, log2_T=12, n_features=2, base_res=8.0, growth=1.5,
                                     with_denominator=True)
    for l in range(6):
        assert rel_err(g[l], ref[l], den[l]) <= 1e-5
    # finite differences of the CUDA forward in binary32 (exact up to rounding: linear in H)
    rng = synth.rng(7)
    Dt = torch.from_numpy(D).cuda()
    xd = torch.from_numpy(x).cuda()
    for _ in range(10):
        l, s, f = int(rng.integers(6)), int(ref[0].shape[0] * 0 + rng.integers(1 << 12)), int(rng.integers(2))
        if den[l][s, f] == 0:
            continue
        Hp, Hm = H.detach().clone(), H.detach().clone()
        Hp[l, s, f] += 0.5
        Hm[l, s, f] -= 0.5
        fd = ((enc.encode_fwd(xd, Hp) * Dt).double().sum() - (enc.encode_fwd(xd, Hm) * Dt).double().sum()).item()
        assert abs(fd - g[l, s, f]) <= 1e-4 * max(1.0, den[l][s, f])
    # FP64 finite differences of the oracle's forward (exact up to FP64 rounding: the encoding is
    # linear in the tables): the library's table gradient within 1e-4 of the sum of |w D| per entry
    n_fd = 0
    for _ in range(12):
        l, s, f = int(rng.integers(6)), int(rng.integers(1 << 12)), int(rng.integers(2))
        if den[l][s, f] == 0:
            continue
        Hp, Hm = vals.astype(np.float64), vals.astype(np.float64)
        Hp[l, s, f] += 0.5
        Hm[l, s, f] -= 0.5
        fd64 = (np.sum(OE.simplex_encode(x, Hp, base_res=8.0, growth=1.5) * D)
                - np.sum(OE.simplex_encode(x, Hm, base_res=8.0, growth=1.5) * D))
        e = abs(fd64 - g[l, s, f]) / den[l][s, f]
        record_error("encode_bwd table gradient against FP64 finite differences", e, 1e-4, "sum_k |w_k dout| per entry")
        assert e <= 1e-4
        n_fd += 1
    assert n_fd >= 3


@pytest.mark.parametrize("kind", ["simplex", "grid"])
def test_autograd_input_gradient(kind):
    """x.grad through the autograd Function equals the oracle's input gradient and the
    central difference of the CUDA forward (points whose cells stay the same at x +- h)."""
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.autograd import encode
    enc = Encoder(3, 6, 2, 12, 8.0, 1.5, kind=kind, table_dtype="f32")
    vals = synth.uniform_tables(6, 1 << 12, 2, 40, scale=1.0)[0]
    H = torch.from_numpy(vals).cuda()
    x = np.clip(synth.uniform_points(1500, 3, 41), 0.01, 0.99).astype(np.float32)
    D = synth.normal_grads(1500, 12, 42)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    Dt = torch.from_numpy(D).cuda()
    (encode(xt, H, enc) * Dt).sum().backward()
    g = xt.grad.cpu().numpy()
    f = OE.simplex_encode_dx if kind == "simplex" else OE.grid_encode_dx
    ref, den = f(x, vals, D, base_res=8.0, growth=1.5, with_denominator=True)
    assert np.all(np.abs(g - ref) <= 1e-5 * den + 1e-30)
    h = 2.0 ** -12
    slots0 = enc.encode_vertices(torch.from_numpy(x).cuda())[0].sort(dim=-1).values
    n_checked = 0
    for j in range(3):
        xp, xm = x.copy(), x.copy()
        xp[:, j] += h
        xm[:, j] -= h
        same = torch.ones(len(x), dtype=torch.bool, device="cuda")
        outs = []
        for xx in (xp, xm):
            xd = torch.from_numpy(xx).cuda()
            s1 = enc.encode_vertices(xd)[0].sort(dim=-1).values
            same &= (s1 == slots0).flatten(1).all(dim=1)
            outs.append((enc.encode_fwd(xd, H).double() * Dt.double()).sum(dim=1))
        fd = ((outs[0] - outs[1]) / (2 * h)).cpu().numpy()
        ok = same.cpu().numpy()
        assert np.all(np.abs(fd - g[:, j])[ok] <= 2e-3 * den[ok, j] + 1e-12)
        n_checked += ok.sum()
    assert n_checked > 1000
    # FP64 central differences of the oracle's FP64 forward (scale and skew in FP64, exactly
    # piecewise linear in x) for points whose FP64 cells stay the same at x +- h
    fwd64 = OE.simplex_encode_fp64 if kind == "simplex" else OE.grid_encode_fp64
    x64, h64 = x.astype(np.float64), 1e-7
    from test_oracle_encoding import _fp64_cells, _same_cells
    cells = _fp64_cells(kind, x64, 3, 6, 8.0, 1.5, 12)
    same32 = np.ones(len(x), dtype=bool)              # the binary32 coordinate picks the same cell
    for c32, c64 in zip(_same_cells(kind, x, 3, 6, 8.0, 1.5, 12), cells):
        same32 &= np.all(c32 == c64, axis=1)
    n_fd = 0
    for j in range(3):
        xp, xm = x64.copy(), x64.copy()
        xp[:, j] += h64
        xm[:, j] -= h64
        ok = same32.copy()
        for xx in (xp, xm):
            for c0, c1 in zip(cells, _fp64_cells(kind, xx, 3, 6, 8.0, 1.5, 12)):
                ok &= np.all(c0 == c1, axis=1)
        fd64 = ((fwd64(xp, vals, base_res=8.0, growth=1.5) - fwd64(xm, vals, base_res=8.0, growth=1.5)) * D).sum(1) / (2 * h64)
        e = np.max(np.abs(fd64 - g[:, j])[ok] / (den[ok, j] + 1e-30))
        record_error("encode_bwd_input dL/dx against FP64 finite differences (%s)" % kind, e, 1e-4,
                     "sum of |terms| of each dL/dx_i")
        assert e <= 1e-4
        n_fd += ok.sum()
    assert n_fd > 1000


def test_autograd_mlp_matches_oracle():
    from paper_2311_15439_gb300.api import Mlp
    from paper_2311_15439_gb300.autograd import mlp_apply
    mlp = Mlp(32, 3, n_hidden=2, dtype="f16")
    W = torch.from_numpy(mlp.init_weights(1)).half().cuda().requires_grad_(True)
    x = torch.from_numpy(synth.rng(2).uniform(-1, 1, (600, 32)).astype(np.float32)).half().cuda().requires_grad_(True)
    y = mlp_apply(x, W, mlp)
    dy = torch.from_numpy(synth.normal_grads(600, 3, 3)).cuda()
    (y * dy).sum().backward()
    Ws = [w.astype(np.float64) for w in mlp.split(W.detach().float().cpu().numpy())]
    _, acts = OM.mlp_forward(Ws, x.detach().float().cpu().numpy().astype(np.float64))
    dW_ref, din_ref = OM.mlp_backward(Ws, acts, dy.cpu().numpy().astype(np.float64))
    # the Function returns exactly what the C ABI computes, cast to the parameter dtypes
    dW_direct = torch.zeros((mlp.n_params,), device="cuda")
    din_direct = torch.empty((600, 32), device="cuda")
    mlp.mlp_bwd(W.detach(), x.detach(), dy, dW_direct, din=din_direct)
    assert torch.equal(W.grad, dW_direct.half())
    assert torch.equal(x.grad, din_direct.half())
    # and agrees with the oracle within the network tolerance plus the final fp16 rounding
    from test_gpu_mlp import _dens, flip_slack, within
    xs = x.detach().float().cpu().numpy().astype(np.float64)
    dyn = dy.cpu().numpy().astype(np.float64)
    _, dW_den, din_den = _dens(Ws, xs, dyn)
    dW_sl, din_sl = flip_slack(Ws, xs, dyn, 2.0 ** -11)
    tol = 6 * 2.0 ** -11 + 2.0 ** -11
    for a, b, den, sl in zip(mlp.split(W.grad.float().cpu().numpy()), dW_ref, dW_den, dW_sl):
        assert within(a, b, den, tol, sl) <= 1.0
    assert within(x.grad.float().cpu().numpy(), din_ref, din_den, tol, din_sl) <= 1.0


def test_grouped_input_gradient_is_the_transpose():
    """dL/din written grouped ([n_in/g][P][g]) equals the row-major result rearranged, bit for bit."""
    from paper_2311_15439_gb300.api import Mlp
    mlp = Mlp(32, 3, n_hidden=2, dtype="f16")
    W = torch.from_numpy(mlp.init_weights(2)).half().cuda()
    P = 3001
    x = torch.from_numpy(synth.rng(3).uniform(-1, 1, (P, 32)).astype(np.float32)).half().cuda()
    tgt = torch.from_numpy(synth.rng(4).random((P, 3)).astype(np.float32)).cuda()
    d_rows = torch.empty((P, 32), device="cuda")
    mlp.mlp_train_l2(W, x, tgt, torch.zeros(mlp.n_params, device="cuda"), torch.zeros(1, device="cuda"), din=d_rows)
    for g in (1, 2, 4, 8):
        d_g = torch.empty((32 // g, P, g), device="cuda")
        mlp.mlp_train_l2_grouped(W, x, tgt, torch.zeros(mlp.n_params, device="cuda"), torch.zeros(1, device="cuda"),
                                 d_g, g)
        assert torch.equal(d_g.permute(1, 0, 2).reshape(P, 32), d_rows)


def test_sdf_training_reduces_loss():
    """SDF-style workload (d = 3, bf16 tables and network, one hidden layer, one output):
    fitting the signed distance of a union of spheres and tori drives the L2 loss down."""
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import Trainer
    P = 1 << 15
    enc = Encoder(3, 16, 2, 16, 16.0, 1.38, table_dtype="bf16")
    tr = Trainer(enc, Mlp(32, 1, n_hidden=1, dtype="bf16"), P, seed=4)
    scene = synth.SphereTorusScene(5)
    losses = []
    for it in range(80):
        x = synth.sdf_points(P, 200 + it)
        tr.step(torch.from_numpy(x).cuda(), torch.from_numpy(scene.sdf(x)).cuda())
        if it in (0, 79):
            losses.append(tr.loss())
    assert np.isfinite(losses).all() and losses[1] < 0.5 * losses[0]


def _close_up_to_atomics(a, b, steps, lr=1e-2, rtol=1e-3, atol=1e-6, max_frac=1e-3):
    """Two trainers whose table gradients were summed by binary32 atomics in different orders:
    an entry whose gradient nearly cancels can take a different Adam update (m / (sqrt(v) + eps)
    normalises the rounding noise), so every element lies within 2 lr per step of the other run
    and all but a small fraction within the tight tolerance."""
    diff = (a - b).abs()
    assert float(diff.max()) <= 2 * lr * steps
    loose = diff > atol + rtol * b.abs()
    assert float(loose.float().mean()) <= max_frac, int(loose.sum())


def test_graph_replay_equals_eager_steps():
    """A step recorded into a CUDA graph and replayed on new batch contents (the step count and
    the Adam bias corrections advance on the device) gives the eager steps' parameters."""
    P = 4096
    a, b = _make(P, seed=11), _make(P, seed=11)
    img = synth.ProceduralImage(3, size=1024, n_waves=4)
    batches = []
    for i in range(5):
        x = synth.uniform_points(P, 2, 40 + i)
        batches.append((torch.from_numpy(x).cuda(), torch.from_numpy(img.sample(x)).cuda()))
    bx, bt = torch.empty_like(batches[0][0]), torch.empty_like(batches[0][1])
    bx.copy_(batches[0][0]); bt.copy_(batches[0][1])
    b.capture(bx, bt, warmup=2)                      # two eager steps on batch 0
    a.step(*batches[0]); a.step(*batches[0])
    for x, t in batches[1:]:
        a.step(x, t)
        bx.copy_(x); bt.copy_(t)
        b.replay()
    torch.cuda.synchronize()
    assert a.t == b.t == 6 and int(b.t_dev.item()) == 6
    # equal up to the order of the binary32 atomics of the table backward (which then feeds the
    # next steps' encodings and network gradients)
    _close_up_to_atomics(a.W, b.W, steps=6, atol=1e-5)
    _close_up_to_atomics(a.table_params(), b.table_params(), steps=6)
    assert a.loss() == pytest.approx(b.loss(), rel=1e-3)


def test_full_size_image_step_replayed_equals_eager():
    """The image workload at full size (d = 2, L = 16, F = 2, T = 2^22 fp16 tables, 2 GiB of state
    records, network 32-64-64-3, 2^18 points per step), trained the way the benchmark times it:
    one recording of the step per resident batch, replayed.  Three replayed steps give the
    parameters of three eager steps (up to the order of the table backward's atomics), over every
    table entry either run moved and every network weight."""
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import Trainer
    P = 1 << 18
    cfg = dict(d=2, n_levels=16, n_features=2, log2_T=22, base_res=16.0, growth=2.0)
    img = synth.ProceduralImage(3, size=16384, n_waves=64)
    xs = [torch.from_numpy(synth.uniform_points(P, 2, 80 + i)).cuda() for i in range(3)]
    ts = [torch.from_numpy(img.sample(x.cpu().numpy())).cuda() for x in xs]

    def make():
        enc = Encoder(**cfg, table_dtype="f16")
        return Trainer(enc, Mlp(32, 3, n_hidden=2, dtype="f16"), P, seed=3, table_layout="records")

    a = make()
    init = a.table_params().clone()
    for x, t in zip(xs, ts):
        a.step(x, t)
    pa, Wa = a.table_params().clone(), a.W.clone()
    del a
    torch.cuda.empty_cache()
    b = make()
    graphs = []
    for x, t in zip(xs, ts):
        b.capture(x, t, warmup=0)
        graphs.append(b.graph)
    for g in graphs:
        b.t += 1
        g.replay()
    torch.cuda.synchronize()
    assert b.t == 3 and int(b.t_dev.item()) == 3
    pb = b.table_params()
    moved = (pa != init) | (pb != init)
    assert int(moved.sum()) > 1_000_000                  # millions of touched entries compared
    # (the fraction is taken over the moved entries only, not diluted by the untouched majority;
    # a replay on the wrong batch or step count moves most of them differently)
    _close_up_to_atomics(pa[moved], pb[moved], steps=3, max_frac=1e-2)
    _close_up_to_atomics(Wa, b.W, steps=3, atol=1e-5)


@pytest.mark.parametrize("split", [1, 2])
def test_stage_events_inside_recordings(split):
    """Timing events marked while a step is recorded are nodes of that graph: after replays of two
    distinct recordings each recording's stage events are complete, ordered and inside the span of
    the replays, and the replays train like eager steps."""
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import Trainer
    try:
        torch.cuda.Event(enable_timing=True, external=True)
    except TypeError:
        pytest.skip("this PyTorch records no timing events inside graphs")
    P = 8192
    enc = Encoder(**CFG, table_dtype="f16")
    mlp = Mlp(16, 3, n_hidden=2, dtype="f16")
    a = Trainer(enc, mlp, P, seed=5, table_layout="records", split_batch=split)
    b = Trainer(enc, mlp, P, seed=5, table_layout="records", split_batch=split)
    img = synth.ProceduralImage(3, size=1024, n_waves=4)
    xs = [torch.from_numpy(synth.uniform_points(P, 2, 70 + i)).cuda() for i in range(2)]
    ts = [torch.from_numpy(img.sample(x.cpu().numpy())).cuda() for x in xs]
    recs = []
    for i in range(2):
        b.stage_events = {}
        b.capture(xs[i], ts[i], warmup=0)
        recs.append((b.graph, b.stage_events))
    b.stage_events = None
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for g, _ in recs:
        b.t += 1
        g.replay()
    e.record()
    for i in range(2):
        a.step(xs[i], ts[i])
    torch.cuda.synchronize()
    span = s.elapsed_time(e)
    order = ["encode_fwd", "encode_fwd_end", "mlp_train_l2", "mlp_train_l2_end", "adam_tables",
             "adam_tables_end", "adam_mlp_end"]
    for _, ev in recs:
        assert set(order) | {"encode_bwd", "encode_bwd_end"} <= set(ev)
        for n in ev:
            assert all(x.query() for x in ev[n]), n
        t = [s.elapsed_time(ev[n][0]) for n in order]
        assert all(0.0 <= u <= span for u in t), t
        assert t == sorted(t), t
        for x, y in zip(ev["encode_bwd"], ev["encode_bwd_end"]):
            assert 0.0 < x.elapsed_time(y) <= span
    assert a.t == b.t == 2
    _close_up_to_atomics(a.W, b.W, steps=2, atol=1e-5)
    _close_up_to_atomics(a.table_params(), b.table_params(), steps=2)
    # a recording that marks one stage only
    b.stage_events, b.stage_only = {}, {"encode_bwd"}
    b.capture(xs[0], ts[0], warmup=0)
    ev, b.stage_events, b.stage_only = b.stage_events, None, None
    assert set(ev) == {"encode_bwd", "encode_bwd_end"} and len(ev["encode_bwd"]) == split
    b.t += 1
    b.graph.replay()
    torch.cuda.synchronize()
    assert all(0.0 < x.elapsed_time(y) for x, y in zip(ev["encode_bwd"], ev["encode_bwd_end"]))


@pytest.mark.parametrize("k", [2, 3, 5])
def test_overlapped_table_step_equals_plain_step(k):
    """The table backward and Adam in k level ranges, Adam of one range on a second stream while
    the backward of the next runs, gives the plain two-pass step's parameters (equal up to the
    order of the binary32 atomics), eagerly and replayed from a CUDA graph."""
    P = 4096
    a, b = _make(P, seed=12, layout="records"), _make(P, seed=12, layout="records")
    b.set_table_chunks(k)
    assert len(b.chunks) == k and b.chunks[0][0] == 0 and b.chunks[-1][1] == CFG["n_levels"]
    assert all(c[1] == n[0] for c, n in zip(b.chunks, b.chunks[1:]))
    img = synth.ProceduralImage(4, size=1024, n_waves=4)
    batches = []
    for i in range(5):
        x = synth.uniform_points(P, 2, 60 + i)
        batches.append((torch.from_numpy(x).cuda(), torch.from_numpy(img.sample(x)).cuda()))
    for x, t in batches[:3]:
        a.step(x, t)
        b.step(x, t)
    torch.cuda.synchronize()
    _close_up_to_atomics(a.state, b.state, steps=3)
    assert int(b.touched.abs().sum().item()) == 0                 # every range cleared its bits
    bx, bt = torch.empty_like(batches[0][0]), torch.empty_like(batches[0][1])
    bx.copy_(batches[3][0]); bt.copy_(batches[3][1])
    b.capture(bx, bt, warmup=1)                                    # one eager step on batch 3
    a.step(*batches[3])
    a.step(*batches[4])
    bx.copy_(batches[4][0]); bt.copy_(batches[4][1])
    b.replay()
    torch.cuda.synchronize()
    assert a.t == b.t == 5
    _close_up_to_atomics(a.W, b.W, steps=5, atol=1e-5)
    _close_up_to_atomics(a.state, b.state, steps=5)
    _close_up_to_atomics(a.tables.float(), b.tables.float(), steps=5)


@pytest.mark.parametrize("layout", ["records", "dense"])
def test_split_batch_step_equals_plain_step(layout):
    """The step in two parts (each part's network pass normalised by the whole batch, each part's
    table backward on a second stream beside the next part's network pass) trains like the plain
    step: the same loss, and parameters equal up to the order of the binary32 atomics and of the
    network gradient's partial sums, eagerly and replayed from a CUDA graph; the end-to-end feed
    reads both parts' losses."""
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import HostFeed, Trainer
    P = 4096 + 128
    mk = lambda split: Trainer(Encoder(**CFG, table_dtype="f16"), Mlp(16, 3, n_hidden=2, dtype="f16"), P, seed=14,
                               table_layout=layout, split_batch=split)
    a, b = mk(1), mk(2)
    assert b.parts() == [(0, P // 2), (P // 2, P)]
    img = synth.ProceduralImage(4, size=1024, n_waves=4)
    batches = []
    for i in range(6):
        x = synth.uniform_points(P, 2, 90 + i)
        batches.append((torch.from_numpy(x).cuda(), torch.from_numpy(img.sample(x)).cuda()))
    for x, t in batches[:3]:
        a.step(x, t)
        b.step(x, t)
        assert abs(a.loss() - b.loss()) <= 1e-5 * a.loss()
    torch.cuda.synchronize()
    _close_up_to_atomics(a.W, b.W, steps=3, atol=1e-5)
    _close_up_to_atomics(a.table_params(), b.table_params(), steps=3)
    bx, bt = torch.empty_like(batches[0][0]), torch.empty_like(batches[0][1])
    bx.copy_(batches[3][0]); bt.copy_(batches[3][1])
    b.capture(bx, bt, warmup=1)
    a.step(*batches[3])
    a.step(*batches[4])
    bx.copy_(batches[4][0]); bt.copy_(batches[4][1])
    b.replay()
    torch.cuda.synchronize()
    assert a.t == b.t == 5
    assert abs(a.loss() - b.loss()) <= 1e-5 * a.loss()
    _close_up_to_atomics(a.W, b.W, steps=5, atol=1e-5)
    _close_up_to_atomics(a.table_params(), b.table_params(), steps=5)
    feed = HostFeed(b, (batches[5][0].cpu().pin_memory(), batches[5][1].cpu().pin_memory()), warmup=0)
    assert feed.step(batches[5][0].cpu().pin_memory(), batches[5][1].cpu().pin_memory()) is None
    last = feed.finish()
    assert np.isfinite(last) and last > 0


@pytest.mark.parametrize("layout", ["records", "dense"])
def test_coarse_levels_on_a_second_stream_equal_plain_step(layout):
    """The backward of the levels summed in shared memory on a second stream, concurrently with
    the other levels, gives the one-stream step's parameters (equal up to the order of the
    binary32 atomics), eagerly and replayed from a CUDA graph."""
    P = 4096
    a, b = _make(P, seed=13, layout=layout), _make(P, seed=13, layout=layout)
    a.tab.set_split_coarse(False)
    b.tab.set_split_coarse(True)
    assert a.tab.split_coarse is False and b.tab.split_coarse is True
    lc = b.enc.bwd_coarse_levels(P)
    assert 0 < lc < CFG["n_levels"]
    assert b.enc.bwd_kernel_count(P, levels=(0, lc)) == 1 and b.enc.bwd_kernel_count(P, levels=(lc, 8)) == 1
    img = synth.ProceduralImage(5, size=1024, n_waves=4)
    batches = []
    for i in range(5):
        x = synth.uniform_points(P, 2, 70 + i)
        batches.append((torch.from_numpy(x).cuda(), torch.from_numpy(img.sample(x)).cuda()))
    for x, t in batches[:3]:
        a.step(x, t)
        b.step(x, t)
    torch.cuda.synchronize()
    _close_up_to_atomics(a.table_params(), b.table_params(), steps=3)
    bx, bt = torch.empty_like(batches[0][0]), torch.empty_like(batches[0][1])
    bx.copy_(batches[3][0]); bt.copy_(batches[3][1])
    b.capture(bx, bt, warmup=1)                                    # one eager step on batch 3
    a.step(*batches[3])
    a.step(*batches[4])
    bx.copy_(batches[4][0]); bt.copy_(batches[4][1])
    b.replay()
    torch.cuda.synchronize()
    assert a.t == b.t == 5
    _close_up_to_atomics(a.W, b.W, steps=5, atol=1e-5)
    _close_up_to_atomics(a.table_params(), b.table_params(), steps=5)
    _close_up_to_atomics(a.tables.float(), b.tables.float(), steps=5)
    if layout == "records":
        assert int(b.touched.abs().sum().item()) == 0


def _bias_corrections(b1, b2, k):
    """1 / (1 - beta^k) for the descriptor's binary32 betas, exactly rounded to binary32 (FP64 on
    the host; beta^k through exact rationals where FP64 could lose the last bit)."""
    from fractions import Fraction
    out = []
    for b in (b1, b2):
        bb = Fraction(float(np.float32(b)))
        pk = bb ** k if k <= 4096 else Fraction(float(np.float64(np.float32(b))) ** k)
        out.append(np.float32(float(1 / (1 - pk))))
    return np.array(out, dtype=np.float32)


def test_device_step_counter_and_bias_corrections():
    """sxe_adam_advance: t counts up on the device and the corrections are 1 / (1 - beta^t), formed
    in double-word binary32 arithmetic (no FP64 on the device) and rounded once: at most one
    binary32 ulp from the exactly rounded value, for every t up to 4097 checked, and for t far out
    (10^6, 2^31) where beta^t has underflowed."""
    from paper_2311_15439_gb300.api import Adam
    a = Adam(1e-2, 0.9, 0.99, 1e-15, skip_zero_grad=True)
    t = torch.zeros((1,), dtype=torch.int64, device="cuda")
    c = torch.zeros((2,), dtype=torch.float32, device="cuda")
    checks = {1, 2, 3, 4, 5, 7, 10, 16, 33, 64, 100, 229, 459, 1000, 2048, 4097}
    for k in range(1, 4098):
        a.advance(t, c)
        if k in checks:
            got = c.cpu().numpy()
            want32 = _bias_corrections(0.9, 0.99, k)
            assert int(t.item()) == k
            assert np.all(np.abs(got.astype(np.float64) - want32) <= np.spacing(want32)), (k, got, want32)
    for k in (10 ** 6, 1 << 31):
        t.fill_(k - 1)
        a.advance(t, c)
        assert int(t.item()) == k
        assert np.array_equal(c.cpu().numpy(), np.ones(2, dtype=np.float32)), (k, c.cpu().numpy())
    # other betas, including the 0.999 of Kingma & Ba (amplification 1 / (1 - beta) = 1000)
    a2 = Adam(1e-3, 0.5, 0.999, 1e-8)
    t.zero_()
    for k in range(1, 3001):
        a2.advance(t, c)
        if k in checks or k % 500 == 0:
            got = c.cpu().numpy()
            want32 = _bias_corrections(0.5, 0.999, k)
            assert np.all(np.abs(got.astype(np.float64) - want32) <= np.spacing(want32)), (k, got, want32)


def test_host_feed_equals_eager_steps():
    """HostFeed (pinned host batches, double-buffered copies on a copy stream, a recorded step per
    buffer pair, the loss returned one step late) trains like eager steps on device copies of the
    same batches and reports each step's loss."""
    from paper_2311_15439_gb300.trainer import HostFeed
    P = 4096
    a, b = _make(P, seed=13), _make(P, seed=13)
    img = synth.ProceduralImage(5, size=1024, n_waves=4)
    batches = []
    for i in range(7):
        x = synth.uniform_points(P, 2, 80 + i)
        batches.append((torch.from_numpy(x).pin_memory(), torch.from_numpy(img.sample(x)).pin_memory()))
    feed = HostFeed(b, batches[0], warmup=2)            # two eager steps on batch 0, then two recordings
    for _ in range(2):
        a.step(batches[0][0].cuda(), batches[0][1].cuda())
    want = []
    for x, t in batches[1:]:
        a.step(x.cuda(), t.cuda())
        want.append(a.loss())
    got = [feed.step(x, t) for x, t in batches[1:]]
    last = feed.finish()
    assert got[0] is None
    got = got[1:] + [last]
    assert a.t == b.t == 8
    assert got == pytest.approx(want, rel=1e-3)
    _close_up_to_atomics(a.W, b.W, steps=8, atol=1e-5)
    _close_up_to_atomics(a.table_params(), b.table_params(), steps=8)


def test_table_layouts_train_alike():
    """The interleaved-record layout (touched bitmap, sweep over the touched records) and the dense
    layout (dense gradient array, dense Adam skipping zero gradients) take the same steps."""
    P = 4096
    a, b = _make(P, seed=14, layout="records"), _make(P, seed=14, layout="dense")
    img = synth.ProceduralImage(6, size=1024, n_waves=4)
    for i in range(4):
        x = synth.uniform_points(P, 2, 90 + i)
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(img.sample(x)).cuda()
        a.step(xd, td)
        b.step(xd, td)
        if i == 0:
            assert a.loss() == b.loss()                  # same first forward pass
    torch.cuda.synchronize()
    _close_up_to_atomics(a.W, b.W, steps=4, atol=1e-5)
    _close_up_to_atomics(a.table_params(), b.table_params(), steps=4)
    _close_up_to_atomics(a.tables.float(), b.tables.float(), steps=4)
    assert int(a.touched.abs().sum().item()) == 0 and float(b.tab.grad.abs().max()) == 0.0


def test_data_parallel_shards_average_to_the_union_step():
    """The data-parallel step on the library's kernels, two ranks emulated one after the other on
    one GPU (no collective: their gradient buffers are averaged in place of the all-reduce): the
    average equals the gradients and loss of one step on the union of the two batches, and Adam on
    it moves the parameters like the union step."""
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.data_parallel import DataParallelTrainer, shard
    from paper_2311_15439_gb300.trainer import Trainer
    cfg = dict(d=3, n_levels=8, n_features=2, log2_T=15, base_res=16.0, growth=1.5)
    P = 1 << 14
    dp = DataParallelTrainer(Encoder(**cfg, table_dtype="f16"), Mlp(16, 1, n_hidden=1, dtype="f16"), P, seed=3)
    un = Trainer(Encoder(**cfg, table_dtype="f16"), Mlp(16, 1, n_hidden=1, dtype="f16"), 2 * P, seed=3,
                 table_layout="dense")
    scene = synth.SphereTorusScene(5)
    x = scene.sample(2 * P, 77)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(scene.sdf(x)).cuda()
    un.t += 1
    un.adam_tables.advance(un.t_dev, un.corrections)
    un.tab.forward(xd, un.enc_out)
    un.mlp.mlp_train_l2(un.W_lowp, un.enc_out, td, un.dW, un.sq_sum, din=un.d_enc, loss_scale=un.loss_scale,
                        workspace=un.ws)
    un.tab.backward(xd, un.d_enc)
    g_un, dW_un, loss_un = un.table_grads().cpu().numpy().copy(), un.dW.cpu().numpy().copy(), un.loss()
    dp.tr.t += 1
    dp.tr.adam_tables.advance(dp.tr.t_dev, dp.tr.corrections)
    flats = []
    for r in range(2):
        s = shard(2 * P, r, 2)
        dp.flat.zero_()
        dp.local_grads(xd[s].contiguous(), td[s].contiguous())
        flats.append(dp.flat.clone())
    dp.flat.copy_((flats[0] + flats[1]) * 0.5)          # what the all-reduce (mean over 2 ranks) gives
    g_dp, dW_dp = dp.tr.table_grads().cpu().numpy(), dp.tr.dW.cpu().numpy()
    assert abs(dp.loss() - loss_un) <= 1e-5 * loss_un
    gmax = np.abs(g_un).max()
    assert gmax > 0 and np.abs(g_dp - g_un).max() <= 1e-5 * gmax
    assert np.array_equal(g_dp == 0, g_un == 0)
    assert np.abs(dW_dp - dW_un).max() <= 1e-5 * np.abs(dW_un).max()
    dp.apply()
    un.tab.adam(un.adam_tables, un.corrections)
    un.adam_mlp.step_dev(un.corrections, un.W, un.mW, un.vW, un.dW, lowp=un.W_lowp)
    clear = np.abs(g_un) > 1e-3 * gmax                 # entries whose step direction is unambiguous
    assert clear.sum() > 1000
    p_dp, p_un = dp.tr.table_params().cpu().numpy(), un.table_params().cpu().numpy()
    np.testing.assert_allclose(p_dp[clear], p_un[clear], rtol=0, atol=1e-6)
    assert np.array_equal(p_dp[g_un == 0], p_un[g_un == 0])
    assert torch.all(dp.flat[:-1] == 0)                 # Adam left the gradient parts zero
