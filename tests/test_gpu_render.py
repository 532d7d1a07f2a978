"""GPU parity of the volumetric rendering kernels (Sec. 6.2, Eq. 5) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from conftest import record_error

from oracle import render as OR
from paper_2311_15439_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _rays(R, seed):
    return [torch.from_numpy(a).cuda() for a in synth.camera_rays(R, seed)]


@pytest.mark.parametrize("S", [1, 3, 32, 33, 257])
def test_samples_bit_exact(cuda_lib, S):
    from paper_2311_15439_gb300.render import vr_samples
    o, d, tn, tf = synth.camera_rays(500, 1)
    x, delta = vr_samples(*[torch.from_numpy(a).cuda() for a in (o, d, tn, tf)], S)
    xr, dr = OR.ray_samples_fp32(o, d, tn, tf, S)
    assert np.array_equal(x.cpu().numpy().view(np.uint32), xr.view(np.uint32))
    assert np.array_equal(delta.cpu().numpy().view(np.uint32), dr.view(np.uint32))


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_field_head_matches_oracle(cuda_lib, dtype):
    from paper_2311_15439_gb300.render import vr_field
    R, S = 300, 7
    g = synth.rng(2)
    dens = (4.0 * g.standard_normal((R * S, 16))).astype(np.float32)
    dens[::11, 0] = g.uniform(15.0, 40.0, size=dens[::11, 0].shape)          # clamped logits
    _, d, _, _ = synth.camera_rays(R, 3)
    sigma, cin = vr_field(torch.from_numpy(dens).cuda(), torch.from_numpy(d).cuda(), S, dtype)
    sigma = sigma.cpu().numpy()
    want = OR.density_from_logit(dens[:, 0])
    assert np.all(np.abs(sigma - want) <= 8 * U32 * want)
    c = cin.float().cpu().numpy()
    if dtype == "f16":
        lowp = dens.astype(np.float16).astype(np.float32)
        ulp = 2.0 ** -11
    else:
        lowp = synth.bf16_bits_to_fp32(synth.fp32_to_bf16_bits(dens))
        ulp = 2.0 ** -8
    assert np.array_equal(c[:, :16], lowp)                                   # rounded once, to nearest even
    sh = np.repeat(OR.sh_basis(d.astype(np.float64)), S, axis=0)
    assert np.all(np.abs(c[:, 16:] - sh) <= ulp * np.abs(sh) + 1e-6)          # binary32 polynomial, one rounding


@pytest.mark.parametrize("R,S", [(257, 1), (257, 5), (257, 32), (257, 33), (257, 100), (257, 1024),
                                 (1 << 16, 64)])                  # the last: the volumetric workload's size
def test_composite_matches_oracle(cuda_lib, R, S):
    from paper_2311_15439_gb300.render import vr_composite
    g = synth.rng(10 + S)
    scale = g.choice([0.0, 0.1, 3.0, 50.0, 1e4], size=(R, 1))
    sigma = (g.exponential(1.0, size=(R, S)) * scale).astype(np.float32)
    logits = (3.0 * g.standard_normal((R * S, 3))).astype(np.float32)
    delta = g.uniform(1e-3, 2.0 / S, size=R).astype(np.float32)
    color, trans, w = vr_composite(torch.from_numpy(sigma.reshape(-1)).cuda(), torch.from_numpy(logits).cuda(),
                                   torch.from_numpy(delta).cuda(), S, with_weights=True)
    rgb = OR.sigmoid(logits).reshape(R, S, 3)
    C, T, W = OR.composite(sigma, rgb, delta)
    # binary32 error: the scan of sigma*delta (at most 5 + S/32 additions deep), exp/expm1, products
    tau = np.concatenate([np.zeros((R, 1)), np.cumsum(sigma.astype(np.float64) * delta[:, None], axis=1)[:, :-1]], 1)
    depth = 5 + (S + 31) // 32
    werr = W * ((depth + 2) * tau + 12) * U32 + 1e-30
    assert np.all(np.abs(w.cpu().numpy().reshape(R, S) - W) <= werr)
    cerr = (werr[:, :, None] * rgb).sum(axis=1) + W.sum(axis=1, keepdims=True) * (depth + 8) * U32 + 1e-7
    record_error("vr_composite colour (Eq. 5 quadrature)", np.max(np.abs(color.cpu().numpy() - C) / cerr), 1.0,
                 "binary32 bound of the transmittance scan")
    assert np.all(np.abs(color.cpu().numpy() - C) <= cerr)
    tot = tau[:, -1] + sigma[:, -1].astype(np.float64) * delta
    assert np.all(np.abs(trans.cpu().numpy() - T) <= T * ((depth + 2) * tot + 4) * U32 + 1e-30)


def _renderer(kind, R, S, L=8, log2_T=14, seed=0):
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.render import Renderer
    enc = Encoder(3, L, 2, log2_T, 16.0, 1.5, kind=kind, table_dtype="f16")
    rr = Renderer(enc, R, S, dtype="f16")
    vals, store = synth.uniform_tables(L, 1 << log2_T, 2, seed + 1, dtype="f16", scale=1.0)
    Wd, Wc = rr.init_weights(seed + 2)
    return enc, rr, vals, torch.from_numpy(store).cuda(), Wd, Wc


def _oracle_render(rays, n, S, vals, Wd, Wc, rr, kind):
    o, d, tn, tf = [a[:n] for a in rays]
    Wd_ = [w.astype(np.float64) for w in rr.density.split(Wd.float().cpu().numpy())]
    Wc_ = [w.astype(np.float64) for w in rr.color.split(Wc.float().cpu().numpy())]
    return OR.render(o, d, tn, tf, S, vals, Wd_, Wc_, kind=kind, base_res=16.0, growth=1.5)


@pytest.mark.parametrize("kind", ["simplex", "grid"])
def test_render_end_to_end(cuda_lib, kind):
    """Six launches against the FP64 pipeline (fp16 encoding and networks on the GPU): colours
    within 0.03, and the weights plus the remaining transmittance sum to 1."""
    R, S = 96, 24
    enc, rr, vals, t, Wd, Wc = _renderer(kind, R, S)
    rays = synth.camera_rays(R, 20)
    trans = torch.empty((R,), device="cuda")
    w = torch.empty((R * S,), device="cuda")
    C = rr.render(*[torch.from_numpy(a).cuda() for a in rays], t, Wd, Wc, transmittance=trans, weights=w)
    Cref, Tref, _ = _oracle_render(rays, R, S, vals, Wd, Wc, rr, kind)
    err = np.abs(C.cpu().numpy() - Cref)
    assert err.max() <= 0.03 and np.median(err) <= 3e-3
    np.testing.assert_allclose(w.view(R, S).sum(1).cpu().numpy() + trans.cpu().numpy(), 1.0, atol=2e-5)


def test_render_full_size(cuda_lib):
    """2^16 rays x 1024 samples (2^26 encoded points, T = 2^19 fp16, L = 16), one render as the
    benchmark times it: 8 sampled rays against the oracle, invariants on every ray."""
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.render import Renderer
    R, S, L = 1 << 16, 1024, 16
    enc = Encoder(3, L, 2, 19, 16.0, 1.38, table_dtype="f16")
    rr = Renderer(enc, R, S, dtype="f16")
    vals, store = synth.uniform_tables(L, 1 << 19, 2, 30, dtype="f16", scale=1.0)
    t = torch.from_numpy(store).cuda()
    Wd, Wc = rr.init_weights(31)
    rays = synth.camera_rays(R, 32)
    trans = torch.empty((R,), device="cuda")
    C = rr.render(*[torch.from_numpy(a).cuda() for a in rays], t, Wd, Wc, transmittance=trans).cpu().numpy()
    T = trans.cpu().numpy()
    assert np.isfinite(C).all() and C.min() >= 0 and np.all(C <= 1 - T[:, None] + 1e-5)
    assert T.min() >= 0 and T.max() <= 1
    idx = synth.rng(33).choice(R, 8, replace=False)
    sub = [a[idx] for a in rays]
    Wd_ = [w.astype(np.float64) for w in rr.density.split(Wd.float().cpu().numpy())]
    Wc_ = [w.astype(np.float64) for w in rr.color.split(Wc.float().cpu().numpy())]
    Cref, _, _ = OR.render(*sub, S, vals, Wd_, Wc_, kind="simplex", base_res=16.0, growth=1.38)
    assert np.abs(C[idx] - Cref).max() <= 0.03


@pytest.mark.parametrize("kind,dtype,L", [("simplex", "f16", 16), ("grid", "bf16", 8), ("simplex", "f16", 32)])
def test_fused_field_equals_three_launches(cuda_lib, kind, dtype, L):
    """The one-kernel field (density network, field head, colour network) gives the same sigma,
    colour logits and colours, bit for bit, as the three separate launches; ragged last tile."""
    from paper_2311_15439_gb300.api import Encoder, torch_dtype
    from paper_2311_15439_gb300.render import Renderer
    R, S = 333, 7
    F = 2 if L <= 16 else 1
    enc = Encoder(3, L, F, 14, 16.0, 1.4, kind=kind, table_dtype=dtype)
    _, store = synth.uniform_tables(L, 1 << 14, F, 40, dtype=dtype, scale=1.0)
    t = torch.from_numpy(store.astype(np.int16) if dtype == "bf16" else store).cuda()
    if dtype == "bf16":
        t = t.view(torch.bfloat16)
    rays = [torch.from_numpy(a).cuda() for a in synth.camera_rays(R, 41)]
    out = []
    for fused in (False, True):
        rr = Renderer(enc, R, S, dtype=dtype, fused=fused)
        Wd, Wc = rr.init_weights(42)
        tr = torch.empty((R,), device="cuda")
        C = rr.render(*rays, t, Wd, Wc, transmittance=tr)
        out.append((C.clone(), tr.clone(), rr.sigma[:R * S].clone(), rr.logits[:R * S].clone()))
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("kernel", ["auto", "mma_sync"])
@pytest.mark.parametrize("kind,dtype,L", [("simplex", "f16", 16), ("grid", "bf16", 8)])
def test_fused_field_with_saved_intermediates(cuda_lib, kernel, kind, dtype, L):
    """sxe_vr_field_mlp_saved: sigma, colour logits and colours as the one-kernel field, and the
    density outputs and colour input it keeps for the backward equal those the three separate
    launches write, bit for bit (the tcgen05 kernel under the automatic choice; the three launches
    themselves under mma.sync); ragged last tile."""
    from paper_2311_15439_gb300 import _lib as Lb
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.render import Renderer
    R, S = 333, 7
    enc = Encoder(3, L, 2, 14, 16.0, 1.4, kind=kind, table_dtype=dtype)
    _, store = synth.uniform_tables(L, 1 << 14, 2, 43, dtype=dtype, scale=1.0)
    t = torch.from_numpy(store.astype(np.int16) if dtype == "bf16" else store).cuda()
    if dtype == "bf16":
        t = t.view(torch.bfloat16)
    rays = [torch.from_numpy(a).cuda() for a in synth.camera_rays(R, 44)]
    prev = Lb.lib().sxe_mlp_get_kernel()
    code = {"auto": Lb.SXE_MLP_KERNEL_AUTO, "mma_sync": Lb.SXE_MLP_KERNEL_MMA_SYNC}[kernel]
    assert Lb.lib().sxe_mlp_set_kernel(code) == 0
    try:
        out = []
        for fused, keep in ((False, False), (True, True)):
            rr = Renderer(enc, R, S, dtype=dtype, fused=fused, keep_intermediates=keep)
            Wd, Wc = rr.init_weights(45)
            rr.dens_out.fill_(float("nan"))
            rr.color_in.fill_(float("nan"))
            C = rr.render(*rays, t, Wd, Wc)
            P = R * S
            out.append((C.clone(), rr.sigma[:P].clone(), rr.logits[:P].clone(), rr.dens_out[:P].clone(),
                        rr.color_in[:P].clone()))
        torch.cuda.synchronize()
    finally:
        Lb.lib().sxe_mlp_set_kernel(prev)
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("R,S", [(129, 1), (129, 33), (129, 100), (129, 1024), (1 << 16, 64)])
def test_composite_bwd_matches_oracle(cuda_lib, R, S):
    """dL/dsigma and dL/dlogits of the compositing against the FP64 chain rule, within a bound
    built from the binary32 scans (transmittance and accumulated colour) the kernel runs."""
    from paper_2311_15439_gb300 import _lib as L
    from paper_2311_15439_gb300.render import vr_composite
    g = synth.rng(30 + S)
    scale = g.choice([0.0, 0.1, 3.0, 50.0], size=(R, 1))
    sigma = (g.exponential(1.0, size=(R, S)) * scale).astype(np.float32)
    logits = (2.0 * g.standard_normal((R * S, 3))).astype(np.float32)
    delta = g.uniform(1e-3, 2.0 / S, size=R).astype(np.float32)
    dC = g.standard_normal((R, 3)).astype(np.float32)
    sd, ld, dd = [torch.from_numpy(a).cuda() for a in (sigma.reshape(-1), logits, delta)]
    color, _, _ = vr_composite(sd, ld, dd, S)
    dsig = torch.empty((R * S,), device="cuda")
    dlog = torch.empty((R * S, 3), device="cuda")
    assert L.lib().sxe_vr_composite_bwd(sd.data_ptr(), ld.data_ptr(), dd.data_ptr(), color.data_ptr(),
                                        torch.from_numpy(dC).cuda().data_ptr(), R, S, dsig.data_ptr(),
                                        dlog.data_ptr(), None) == 0
    torch.cuda.synchronize()
    rgb = OR.sigmoid(logits).reshape(R, S, 3)
    ds_ref, dr_ref = OR.composite_bwd(sigma, rgb, delta, dC)
    dl_ref = dr_ref.reshape(-1, 3) * rgb.reshape(-1, 3) * (1 - rgb.reshape(-1, 3))
    C, _, W = OR.composite(sigma, rgb, delta)
    tau = np.cumsum(sigma.astype(np.float64) * delta[:, None], axis=1)          # T_{k+1} = exp(-tau_k)
    depth = 5 + (S + 31) // 32
    P = np.cumsum(W[:, :, None] * rgb, axis=1)
    # T_{k+1} c: the scan depth times tau plus exp, sigmoid and product roundings; C - P_k: two
    # binary32 accumulations of w c (forward and backward kernels round the sigmoid differently)
    t_err = (np.exp(-tau) * ((depth + 2) * tau + 32))[:, :, None] * rgb
    sum_err = 4 * (depth + 12) * (C[:, None, :] + P)
    bound = (delta[:, None] * (np.abs(dC)[:, None, :] * (t_err + sum_err)).sum(axis=2)) * U32 + 1e-30
    got = dsig.cpu().numpy().reshape(R, S)
    record_error("vr_composite_bwd dL/dsigma", np.max(np.abs(got - ds_ref) / bound), 1.0,
                 "binary32 bound of the two scans")
    bad = np.argwhere(np.abs(got - ds_ref) > bound)
    assert len(bad) == 0, [(tuple(i), float(got[tuple(i)]), float(ds_ref[tuple(i)]), float(bound[tuple(i)]),
                            float(sigma[tuple(i)]), float(delta[i[0]])) for i in bad[:5]]
    lbound = np.abs(dl_ref) * ((depth + 2) * np.repeat(tau.reshape(-1), 3).reshape(-1, 3) + 16) * U32 + 1e-30
    gl = dlog.cpu().numpy()
    record_error("vr_composite_bwd dL/dlogits", np.max(np.abs(gl - dl_ref) / lbound), 1.0,
                 "binary32 bound of the scan and sigmoid")
    badl = np.argwhere(np.abs(gl - dl_ref) > lbound)
    assert len(badl) == 0, [(tuple(i), float(gl[tuple(i)]), float(dl_ref[tuple(i)]), float(lbound[tuple(i)]))
                            for i in badl[:5]]


def test_field_bwd_matches_oracle(cuda_lib):
    from paper_2311_15439_gb300 import _lib as L
    R, S = 50, 9
    P = R * S
    g = synth.rng(40)
    dcin = g.standard_normal((P, 32)).astype(np.float32)
    dsig = g.standard_normal(P).astype(np.float32)
    dens = (6.0 * g.standard_normal((P, 16))).astype(np.float32)
    dens[::5, 0] = 15.0 + g.random(len(dens[::5, 0])).astype(np.float32)         # clamped: no sigma term
    sig = OR.density_from_logit(dens[:, 0]).astype(np.float32)
    t = [torch.from_numpy(a).cuda() for a in (dcin, dsig, sig, dens)]
    dv = torch.empty((P, 16), device="cuda")
    assert L.lib().sxe_vr_field_bwd(t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), t[3].data_ptr(), R, S,
                                    dv.data_ptr(), None) == 0
    want = dcin[:, :16].astype(np.float64)
    want[:, 0] += np.where(dens[:, 0] < 15.0, dsig.astype(np.float64) * sig, 0.0)
    got = dv.cpu().numpy()
    assert np.all(np.abs(got - want) <= 2 * U32 * (np.abs(want) + np.abs(dsig.astype(np.float64) * sig)[:, None]))


@pytest.mark.parametrize("layout", ["records", "dense"])
def test_volume_gradients_match_oracle(cuda_lib, layout):
    """Every gradient of one volumetric training step (tables, density and colour networks)
    against the FP64 chain rule on the same fp16 weights and tables: relative L2 error within
    5 %, direction within 0.99 cosine (fp16 networks, ReLU decisions near zero can flip); both
    table layouts."""
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.render import VolumeTrainer
    R, S, L, log2_T = 128, 16, 8, 12
    enc = Encoder(3, L, 2, log2_T, 8.0, 1.5, table_dtype="f16")
    vt = VolumeTrainer(enc, R, S, seed=3, table_init=0.5, table_layout=layout)
    assert vt.tab.layout == layout
    rays = synth.camera_rays(R, 44)
    target = synth.rng(45).random((R, 3)).astype(np.float32)
    vt.gradients(*[torch.from_numpy(a).cuda() for a in rays], torch.from_numpy(target).cuda())
    torch.cuda.synchronize()
    tab = vt.tables.float().cpu().numpy().astype(np.float64)
    Ws = [[w.astype(np.float64) for w in n["mlp"].split(n["W_lowp"].float().cpu().numpy())] for n in vt.nets]
    loss, gt, dWd, dWc, _ = OR.render_l2_grads(*rays, S, tab, Ws[0], Ws[1], target, kind="simplex", base_res=8.0,
                                                growth=1.5)
    assert vt.loss() == pytest.approx(loss, rel=2e-2)

    def close(a, b):
        a, b = np.ravel(a), np.ravel(b)
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        return rel <= 0.05 and cos >= 0.99

    g_tab = vt.table_grads().cpu().numpy()
    assert close(g_tab, np.stack([gt[l] for l in range(L)]))
    assert close(vt.nets[0]["dW"].cpu().numpy(), np.concatenate([w.ravel() for w in dWd]))
    assert close(vt.nets[1]["dW"].cpu().numpy(), np.concatenate([w.ravel() for w in dWc]))


def test_volume_training_reduces_loss(cuda_lib):
    """Fitting ray colours of a Gaussian-blob scene (targets by the FP64 quadrature of the analytic
    field at the same samples) drives the colour error down."""
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.render import VolumeTrainer
    R, S = 2048, 32
    scene = synth.BlobScene(5)
    batches = []
    for b in range(4):
        o, d, tn, tf = synth.camera_rays(R, 300 + b)
        x, delta = OR.ray_samples_fp32(o, d, tn, tf, S)
        sig, rgb = scene.field(x)
        C, _, _ = OR.composite(sig.reshape(R, S), rgb.reshape(R, S, 3), delta)
        batches.append([torch.from_numpy(a).cuda() for a in (o, d, tn, tf, C.astype(np.float32))])
    enc = Encoder(3, 16, 2, 16, 16.0, 1.38, table_dtype="f16")
    vt = VolumeTrainer(enc, R, S, seed=6)
    losses = []
    for it in range(150):
        vt.step(*batches[it % 4])
        if it in (0, 149):
            losses.append(vt.loss())
    assert np.isfinite(losses).all() and losses[1] < 0.3 * losses[0]
