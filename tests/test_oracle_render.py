"""Pins of the oracle's volumetric rendering (Eq. 5 quadrature, sampling, spherical harmonics)."""
import math

import numpy as np
import pytest
import scipy.special

from oracle import render
from paper_2311_15439_gb300 import synth


def test_composite_equals_eq5_for_homogeneous_media():
    """Constant sigma and colour along [t_n, t_f]: Eq. 5 integrates to c (1 - exp(-sigma (t_f - t_n)))."""
    g = synth.rng(1)
    R, S = 50, 37
    sigma = np.repeat(g.uniform(0.0, 20.0, size=(R, 1)), S, axis=1)
    c = g.random((R, 3))
    rgb = np.repeat(c[:, None, :], S, axis=1)
    length = g.uniform(0.1, 2.0, size=R)
    C, T, w = render.composite(sigma, rgb, length / S)
    want = c * (1.0 - np.exp(-sigma[:, :1] * length[:, None]))
    np.testing.assert_allclose(C, want, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(T, np.exp(-sigma[:, 0] * length), rtol=1e-12)


def test_composite_piecewise_constant_media():
    """Segments of different constant density: the remaining transmittance is exp(-sum sigma delta),
    the weights sum to 1 - T, and a single-colour field gives C = c (1 - T)."""
    g = synth.rng(2)
    R, S = 40, 64
    sigma = g.exponential(3.0, size=(R, S))
    delta = g.uniform(0.001, 0.05, size=R)
    c = g.random(3)
    C, T, w = render.composite(sigma, np.broadcast_to(c, (R, S, 3)), delta)
    np.testing.assert_allclose(T, np.exp(-sigma.sum(axis=1) * delta), rtol=1e-12)
    np.testing.assert_allclose(w.sum(axis=1), 1.0 - T, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(C, (1.0 - T)[:, None] * c[None, :], rtol=1e-12, atol=1e-15)


def test_composite_keeps_tiny_transmittance():
    """A nearly opaque segment: T = exp(-sigma delta) to full relative precision, not 1 - (1 - e^-x)."""
    sigma = np.array([[80.0], [700.0], [1e-20]])
    C, T, w = render.composite(sigma, np.ones((3, 1, 3)), np.ones(3))
    np.testing.assert_allclose(T, np.exp(-sigma[:, 0]), rtol=1e-15)
    np.testing.assert_allclose(w[:, 0], -np.expm1(-sigma[:, 0]), rtol=1e-15)


def test_composite_opaque_and_empty():
    S = 16
    rgb = synth.rng(3).random((1, S, 3))
    C, T, w = render.composite(np.zeros((1, S)), rgb, np.array([0.1]))
    assert np.all(C == 0) and T[0] == 1.0
    sigma = np.zeros((1, S))
    sigma[0, 5] = 1e6                                   # an opaque wall at sample 5
    C, T, w = render.composite(sigma, rgb, np.array([0.1]))
    np.testing.assert_allclose(C[0], rgb[0, 5], rtol=1e-12)
    assert np.all(w[0, 6:] == 0) and T[0] == 0.0


def _unit(n, seed):
    v = synth.rng(seed).standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_sh_equals_scipy_real_basis():
    d = _unit(500, 4)
    polar = np.arccos(np.clip(d[:, 2], -1, 1))
    azim = np.arctan2(d[:, 1], d[:, 0])
    got = render.sh_basis(d)
    j = 0
    for l in range(4):
        for m in range(-l, l + 1):
            Y = scipy.special.sph_harm_y(l, abs(m), polar, azim)
            if m < 0:
                want = math.sqrt(2.0) * (-1) ** m * Y.imag
            elif m == 0:
                want = Y.real
            else:
                want = math.sqrt(2.0) * (-1) ** m * Y.real
            np.testing.assert_allclose(got[:, j], want, rtol=0, atol=1e-12, err_msg="l=%d m=%d" % (l, m))
            j += 1


def test_sh_orthonormal_on_the_sphere():
    """Gauss-Legendre in cos(polar) x uniform azimuth integrates degree <= 6 products exactly."""
    u, wu = np.polynomial.legendre.leggauss(12)
    phi = np.arange(24) * (2 * np.pi / 24)
    U, PHI = np.meshgrid(u, phi, indexing="ij")
    s = np.sqrt(1 - U ** 2)
    d = np.stack([s * np.cos(PHI), s * np.sin(PHI), U], -1).reshape(-1, 3)
    wt = (wu[:, None] * np.full(24, 2 * np.pi / 24)[None, :]).reshape(-1)
    Y = render.sh_basis(d)
    G = (Y * wt[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_samples_lie_on_their_rays_in_order():
    g = synth.rng(5)
    R, S = 30, 100
    o = g.uniform(-1, 2, (R, 3)).astype(np.float32)
    d = _unit(R, 6).astype(np.float32)
    tn = g.uniform(0.0, 1.0, R).astype(np.float32)
    tf = (tn + g.uniform(0.1, 2.0, R)).astype(np.float32)
    x, delta = render.ray_samples_fp32(o, d, tn, tf, S)
    x = x.reshape(R, S, 3).astype(np.float64)
    t = tn[:, None] + (np.arange(S) + 0.5)[None, :] * ((tf - tn) / S)[:, None]
    np.testing.assert_allclose(x, o[:, None, :] + t[:, :, None] * d[:, None, :].astype(np.float64), atol=1e-5)
    np.testing.assert_allclose(delta * S, tf - tn, rtol=1e-6)
    proj = np.einsum("rsk,rk->rs", x - o[:, None, :], d.astype(np.float64))
    assert np.all(np.diff(proj, axis=1) > 0)
    assert np.all(proj > tn[:, None] - 1e-5) and np.all(proj < tf[:, None] + 1e-5)


def test_composite_bwd_matches_central_differences():
    g = synth.rng(20)
    R, S = 4, 9
    sigma = g.exponential(2.0, (R, S))
    rgb = g.random((R, S, 3))
    delta = g.uniform(0.05, 0.3, R)
    dC = g.standard_normal((R, 3))
    ds, dr = render.composite_bwd(sigma, rgb, delta, dC)
    h = 1e-6
    for r in range(R):
        for k in range(S):
            sp, sm = sigma.copy(), sigma.copy()
            sp[r, k] += h
            sm[r, k] -= h
            fd = ((render.composite(sp, rgb, delta)[0] - render.composite(sm, rgb, delta)[0]) * dC).sum() / (2 * h)
            assert abs(fd - ds[r, k]) <= 1e-8 * (1 + abs(fd))
            for c in range(3):
                rp, rm = rgb.copy(), rgb.copy()
                rp[r, k, c] += h
                rm[r, k, c] -= h
                fd = ((render.composite(sigma, rp, delta)[0] - render.composite(sigma, rm, delta)[0]) * dC).sum() / (2 * h)
                assert abs(fd - dr[r, k, c]) <= 1e-8 * (1 + abs(fd))


def test_composite_bwd_homogeneous_closed_form():
    """Raising the density of every sample of a homogeneous segment of length l: d/d sigma of
    c (1 - exp(-sigma l)) = c l exp(-sigma l), the sum of the per-sample derivatives."""
    R, S = 3, 40
    sig = np.array([0.5, 3.0, 10.0])
    length = np.array([0.7, 0.2, 1.3])
    c = synth.rng(21).random((R, 3))
    sigma = np.repeat(sig[:, None], S, axis=1)
    ds, _ = render.composite_bwd(sigma, np.repeat(c[:, None, :], S, axis=1), length / S, np.ones((R, 3)))
    want = c.sum(axis=1) * length * np.exp(-sig * length)
    np.testing.assert_allclose(ds.sum(axis=1), want, rtol=1e-10)


def test_render_l2_grads_match_central_differences():
    """The chain rule of the render loss against central differences of the whole oracle render
    (a few table entries and weights of each network, where two step sizes agree)."""
    from oracle import mlp as OM
    g = synth.rng(22)
    R, S, L, log2_T = 6, 8, 3, 8
    o, d, tn, tf = synth.camera_rays(R, 23)
    tables = g.uniform(-1, 1, (L, 1 << log2_T, 2))
    Wd = [g.standard_normal((64, 6)) * 0.4, g.standard_normal((16, 64)) * 0.2]
    Wc = [g.standard_normal((64, 32)) * 0.3, g.standard_normal((64, 64)) * 0.2, g.standard_normal((3, 64)) * 0.2]
    target = g.random((R, 3))
    kw = dict(kind="simplex", base_res=4.0, growth=1.5)
    loss, gt, dWd, dWc, _ = render.render_l2_grads(o, d, tn, tf, S, tables, Wd, Wc, target, **kw)

    def L_of(tab=tables, wd=Wd, wc=Wc):
        C, _, _ = render.render(o, d, tn, tf, S, tab, wd, wc, **kw)
        return np.mean((C - target) ** 2)

    checked = 0
    for l in range(L):
        nz = np.nonzero(np.abs(gt[l]).sum(axis=1))[0][:3]
        for s in nz:
            fds = []
            for h in (1e-4, 1e-5):
                tp, tm = tables.copy(), tables.copy()
                tp[l, s, 0] += h
                tm[l, s, 0] -= h
                fds.append((L_of(tab=tp) - L_of(tab=tm)) / (2 * h))
            if abs(fds[0] - fds[1]) <= 1e-6 * (abs(fds[1]) + 1e-9):
                assert abs(fds[1] - gt[l][s, 0]) <= 1e-5 * (abs(fds[1]) + 1e-9)
                checked += 1
    for W, dW, name in ((Wd, dWd, "d"), (Wc, dWc, "c")):
        for li in range(len(W)):
            i, j = g.integers(W[li].shape[0]), g.integers(W[li].shape[1])
            fds = []
            for h in (1e-4, 1e-5):
                Wp = [w.copy() for w in W]
                Wm = [w.copy() for w in W]
                Wp[li][i, j] += h
                Wm[li][i, j] -= h
                args_p = dict(wd=Wp) if name == "d" else dict(wc=Wp)
                args_m = dict(wd=Wm) if name == "d" else dict(wc=Wm)
                fds.append((L_of(**args_p) - L_of(**args_m)) / (2 * h))
            if abs(fds[0] - fds[1]) <= 1e-6 * (abs(fds[1]) + 1e-9):
                assert abs(fds[1] - dW[li][i, j]) <= 1e-5 * (abs(fds[1]) + 1e-9)
                checked += 1
    assert checked >= 8
