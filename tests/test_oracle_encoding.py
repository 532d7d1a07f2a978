"""Pins of the oracle's encodings, network, loss and optimiser (CPU only)."""
import itertools
import math

import numpy as np
import pytest

from oracle import adam, encoding, lattice, mlp
from paper_2311_15439_gb300 import synth


def _collision_free_tables(kind, n, L, base, growth, log2_T, fn, fp32_scale=True):
    """Tables whose entry at each vertex of every level's lattice box holds fn(position in
    the original unit-cube coordinates, through the binary32 level multiplier, or the FP64 one
    with fp32_scale=False); asserts no two box vertices share a slot."""
    T = 1 << log2_T
    tables = np.zeros((L, T, 1))
    if kind == "simplex":
        scales = lattice.simplex_level_scales_fp64(n, L, base, growth)
    else:
        scales = [float(N) for N in lattice.level_resolutions(L, base, growth)]
    for l in range(L):
        N = lattice.level_resolutions(L, base, growth)[l]
        box = np.stack(np.meshgrid(*([np.arange(0, N + 2)] * n), indexing="ij"), -1).reshape(-1, n)
        slots = lattice.hash_slot(box, log2_T)
        assert len(np.unique(slots)) == len(slots), "hash collision in the test lattice"
        pos = box.astype(float)
        if kind == "simplex":
            pos = lattice.unskew(pos)
        tables[l, slots, 0] = fn(pos / (float(np.float32(scales[l])) if fp32_scale else float(scales[l])))
    return tables


@pytest.mark.parametrize("n", [2, 3, 4])
def test_simplex_reproduces_affine_fields(n):
    """Barycentric interpolation (Sec. 4.3) is exact on affine functions: with every
    vertex holding a.x + b at its unskewed position, the encoding returns a.x~ + b,
    where x~ is the binary32 point the lattice actually sees."""
    g = synth.rng(40 + n)
    a, b = g.standard_normal(n), 0.3
    L, growth = 3, 1.5
    base, log2_T = (4.0, 20) if n < 4 else (3.0, 22)
    tables = _collision_free_tables("simplex", n, L, base, growth, log2_T, lambda p: p @ a + b)
    x = np.concatenate([synth.uniform_points(300, n, 41), synth.edge_points(n, 42, per_kind=4)])
    out = encoding.simplex_encode(x, tables, base_res=base, growth=growth)
    scales = lattice.simplex_level_scales_fp32(n, L, base, growth)
    for l in range(L):
        q = lattice.scaled_skewed_fp32(x, scales[l]).astype(np.float64)
        x_seen = lattice.unskew(q) / float(scales[l])
        np.testing.assert_allclose(out[:, l], x_seen @ a + b, rtol=0, atol=1e-11)
        np.testing.assert_allclose(out[:, l], x.astype(float) @ a + b, rtol=0, atol=1e-5)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_grid_reproduces_multilinear_fields(n):
    """Algorithm 1 (n-linear interpolation) is exact on functions that are affine in each
    coordinate separately, e.g. prod_i (1 + c_i x_i)."""
    g = synth.rng(50 + n)
    cc = g.standard_normal(n)
    L, base, growth = 3, 4.0, 1.5
    fn = lambda p: np.prod(1.0 + cc * p, axis=-1)
    if n == 4:
        base, log2_T = 3.0, 22
    else:
        log2_T = 20
    tables = _collision_free_tables("grid", n, L, base, growth, log2_T, fn)
    x = np.concatenate([synth.uniform_points(300, n, 51), synth.edge_points(n, 52, per_kind=4)])
    out = encoding.grid_encode(x, tables, base_res=base, growth=growth)
    for l, N in enumerate(lattice.level_resolutions(L, base, growth)):
        x_seen = (x * np.float32(N)).astype(np.float64) / N
        np.testing.assert_allclose(out[:, l], fn(x_seen), rtol=0, atol=1e-11)


def test_grid_1d_slice_is_linear_interpolation():
    """A point on an axis-aligned line inside one cell: the 2-D grid reduces to 1-D linear
    interpolation between the two corner values (textbook np.interp)."""
    L, T = 1, 1 << 12
    tab = synth.uniform_tables(L, T, 1, 3)[0].astype(np.float64)
    N = 16
    xs = np.linspace(0.0, 1.0 / N, 33, dtype=np.float32)[:-1]
    x = np.stack([xs, np.zeros_like(xs)], axis=1)
    out = encoding.grid_encode(x, tab, base_res=N, growth=1.0)[:, 0]
    s0, s1 = lattice.hash_slot(np.array([[0, 0], [1, 0]]), 12)
    want = np.interp((xs * np.float32(N)).astype(np.float64), [0.0, 1.0], [tab[0, s0, 0], tab[0, s1, 0]])
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 5])
def test_grid_weights_are_products(n):
    """The corner weights of the recursive interpolation are prod_i (f_i or 1 - f_i), sum to 1."""
    f = synth.rng(60 + n).random((50, n))
    w = encoding.grid_level_corner_weights(f)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-14)
    for j, b in enumerate(itertools.product((0, 1), repeat=n)):
        want = np.prod(np.where(np.array(b)[None, :] == 1, f, 1.0 - f), axis=1)
        np.testing.assert_allclose(w[:, j], want, atol=1e-15)


@pytest.mark.parametrize("kind", ["simplex", "grid"])
@pytest.mark.parametrize("n", [2, 3])
def test_backward_is_adjoint_of_forward(kind, n):
    """The encoding is linear in the tables, so <enc(H), D> = <H, enc_bwd(D)>."""
    L, log2_T, F = 4, 10, 2
    H = synth.uniform_tables(L, 1 << log2_T, F, 7, scale=1.0)[0].astype(np.float64)
    x = synth.uniform_points(700, n, 8)
    D = synth.normal_grads(700, L * F, 9).astype(np.float64)
    kw = dict(base_res=8.0, growth=1.7)
    if kind == "simplex":
        out = encoding.simplex_encode(x, H, **kw)
        G = encoding.simplex_encode_bwd(x, D, n_levels=L, log2_T=log2_T, n_features=F, **kw)
    else:
        out = encoding.grid_encode(x, H, **kw)
        G = encoding.grid_encode_bwd(x, D, n_levels=L, log2_T=log2_T, n_features=F, **kw)
    lhs = float(np.sum(out * D))
    rhs = float(sum(np.sum(H[l] * G[l]) for l in range(L)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_backward_finite_differences():
    """Central differences of <enc(H), D> in single table entries equal enc_bwd(D) there."""
    n, L, log2_T, F = 2, 3, 8, 2
    H = synth.uniform_tables(L, 1 << log2_T, F, 11, scale=1.0)[0].astype(np.float64)
    x = synth.uniform_points(300, n, 12)
    D = synth.normal_grads(300, L * F, 13).astype(np.float64)
    kw = dict(base_res=6.0, growth=1.5)
    G = encoding.simplex_encode_bwd(x, D, n_levels=L, log2_T=log2_T, n_features=F, **kw)
    g = synth.rng(14)
    for _ in range(20):
        l, t, f = int(g.integers(L)), int(g.integers(1 << log2_T)), int(g.integers(F))
        Hp, Hm = H.copy(), H.copy()
        Hp[l, t, f] += 0.5
        Hm[l, t, f] -= 0.5
        fd = (np.sum(encoding.simplex_encode(x, Hp, **kw) * D) - np.sum(encoding.simplex_encode(x, Hm, **kw) * D))
        assert fd == pytest.approx(G[l][t, f], abs=1e-10)


def test_simplex_uses_n_plus_one_slots_per_level():
    """Sec. 5: each level reads n+1 entries per point (weights for the rest are zero)."""
    x = synth.uniform_points(64, 3, 15)
    slots, w, V = encoding.simplex_level_vertices(x, np.float32(20.0), 12)
    assert slots.shape == (64, 4) and w.shape == (64, 4) and V.shape == (64, 4, 3)


# ----------------------------------------------------------------------------
# network, loss, optimiser
# ----------------------------------------------------------------------------
def _mlp(seed, dims):
    g = synth.rng(seed)
    return [g.standard_normal((dims[i + 1], dims[i])) / math.sqrt(dims[i]) for i in range(len(dims) - 1)]


def test_mlp_matches_independent_autograd():
    """Forward and backward agree with PyTorch's CPU autograd in FP64 on the same network."""
    torch = pytest.importorskip("torch")
    Ws = _mlp(1, [32, 64, 64, 3])
    e = synth.rng(2).standard_normal((40, 32))
    dy = synth.rng(3).standard_normal((40, 3))
    y, acts = mlp.mlp_forward(Ws, e)
    dWs, de = mlp.mlp_backward(Ws, acts, dy)
    tW = [torch.tensor(W, requires_grad=True) for W in Ws]
    te = torch.tensor(e, requires_grad=True)
    h = te
    for i, W in enumerate(tW):
        h = h @ W.T
        if i < len(tW) - 1:
            h = torch.relu(h)
    (h * torch.tensor(dy)).sum().backward()
    np.testing.assert_allclose(y, h.detach().numpy(), rtol=1e-13, atol=1e-13)
    for a, b in zip(dWs, tW):
        np.testing.assert_allclose(a, b.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(de, te.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_mlp_finite_differences():
    """Central differences of the L2 loss in weights and inputs match the backward pass."""
    Ws = _mlp(4, [8, 16, 16, 2])
    e = synth.rng(5).standard_normal((10, 8))
    tgt = synth.rng(6).standard_normal((10, 2))

    def loss(Ws_, e_):
        return mlp.l2_loss(mlp.mlp_forward(Ws_, e_)[0], tgt)[0]

    y, acts = mlp.mlp_forward(Ws, e)
    _, dy = mlp.l2_loss(y, tgt)
    dWs, de = mlp.mlp_backward(Ws, acts, dy)
    h = 1e-6
    g = synth.rng(7)
    for _ in range(15):
        i = int(g.integers(len(Ws)))
        r, c = int(g.integers(Ws[i].shape[0])), int(g.integers(Ws[i].shape[1]))
        Wp = [W.copy() for W in Ws]
        Wm = [W.copy() for W in Ws]
        Wp[i][r, c] += h
        Wm[i][r, c] -= h
        assert (loss(Wp, e) - loss(Wm, e)) / (2 * h) == pytest.approx(dWs[i][r, c], rel=1e-5, abs=1e-9)
    for _ in range(10):
        r, c = int(g.integers(10)), int(g.integers(8))
        ep, em = e.copy(), e.copy()
        ep[r, c] += h
        em[r, c] -= h
        assert (loss(Ws, ep) - loss(Ws, em)) / (2 * h) == pytest.approx(de[r, c], rel=1e-5, abs=1e-9)


def test_mlp_hand_example():
    """A 2-1 network worked by hand: W1 = [[1,-1],[2,0.5]], W2 = [[3,-2]], e = (1, 2):
    z1 = (-1, 3) -> h1 = (0, 3), y = -6; with dy = 1: dW2 = (0, 3), dW1 row 0 = 0,
    row 1 = -2 * (1, 2), de = -2 * (2, 0.5)."""
    W1 = np.array([[1.0, -1.0], [2.0, 0.5]])
    W2 = np.array([[3.0, -2.0]])
    y, acts = mlp.mlp_forward([W1, W2], np.array([[1.0, 2.0]]))
    assert y.tolist() == [[-6.0]]
    dWs, de = mlp.mlp_backward([W1, W2], acts, np.array([[1.0]]))
    assert dWs[1].tolist() == [[0.0, 3.0]]
    assert dWs[0].tolist() == [[0.0, 0.0], [-2.0, -4.0]]
    assert de.tolist() == [[-4.0, -1.0]]


def test_l2_loss_closed_form():
    y = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 0.0]])
    t = np.array([[1.0, 1.0, 1.0], [1.0, 0.0, -1.0]])
    loss, dy = mlp.l2_loss(y, t)
    assert loss == pytest.approx((0 + 1 + 4 + 1 + 0 + 1) / 6.0)
    np.testing.assert_allclose(dy, 2 * (y - t) / 6.0)


def test_adam_matches_library_and_skips_zero_grads():
    """Entries with a nonzero gradient follow an independent library Adam; entries whose
    gradient is exactly 0 keep parameter and moments (the skip rule)."""
    torch = pytest.importorskip("torch")
    g = synth.rng(8)
    theta = g.standard_normal(1000)
    grads = [g.standard_normal(1000) * (g.random(1000) < 0.7) for _ in range(4)]
    hp = dict(lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15)
    m = np.zeros(1000)
    v = np.zeros(1000)
    th = theta.copy()
    for t, gr in enumerate(grads, start=1):
        th_new, m_new, v_new = adam.adam_step(th, gr, m, v, t, skip_zero_grad=True, **hp)
        zero = gr == 0
        assert np.array_equal(th_new[zero], th[zero]) and np.array_equal(m_new[zero], m[zero])
        th, m, v = th_new, m_new, v_new
    th_skip = th
    # without skipping, every entry follows torch.optim.Adam exactly
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=hp["lr"], betas=(hp["beta1"], hp["beta2"]), eps=hp["eps"])
    th, m, v = theta.copy(), np.zeros(1000), np.zeros(1000)
    for t, gr in enumerate(grads, start=1):
        p.grad = torch.tensor(gr)
        opt.step()
        th, m, v = adam.adam_step(th, gr, m, v, t, skip_zero_grad=False, **hp)
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-12)
    # with skipping, entries that had a gradient at every step took every step: the same values
    always = np.all([gr != 0 for gr in grads], axis=0)
    assert always.sum() > 100
    np.testing.assert_allclose(th_skip[always], p.detach().numpy()[always], rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# input gradients
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 3, 4])
def test_simplex_dx_of_affine_field(n):
    """On an affine field a.x + b the encoding is a.x + b for every point (Sec. 4.3), so the
    gradient of sum dout * out with respect to x is sum_l dout_l a, exactly (up to the
    rounding of the binary32 skew constant), also on faces and ties."""
    g = synth.rng(140 + n)
    a, b = g.standard_normal(n), -0.2
    L, growth = 3, 1.5
    base, log2_T = (4.0, 20) if n < 4 else (3.0, 22)
    tables = _collision_free_tables("simplex", n, L, base, growth, log2_T, lambda p: p @ a + b)
    x = np.concatenate([synth.uniform_points(200, n, 141), synth.edge_points(n, 142, per_kind=4)])
    dout = synth.normal_grads(len(x), L, 143).astype(np.float64)
    dx = encoding.simplex_encode_dx(x, tables, dout, base_res=base, growth=growth)
    want = dout.sum(axis=1)[:, None] * a[None, :]
    scale = np.abs(dout).sum(axis=1)[:, None] * np.abs(a).sum()
    assert np.all(np.abs(dx - want) <= 1e-6 * scale)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_grid_dx_of_multilinear_field(n):
    """The n-linear interpolant of prod_i (1 + c_i x_i) is that function on every cell, so its
    x-gradient is c_j prod_{i != j} (1 + c_i x_i) at the binary32 point the grid sees."""
    g = synth.rng(150 + n)
    cc = g.standard_normal(n)
    L, base, growth = 3, 4.0, 1.5
    log2_T = 20 if n < 4 else 22
    if n == 4:
        base = 3.0
    fn = lambda p: np.prod(1.0 + cc * p, axis=-1)
    tables = _collision_free_tables("grid", n, L, base, growth, log2_T, fn)
    x = np.concatenate([synth.uniform_points(200, n, 151), synth.edge_points(n, 152, per_kind=4)])
    dout = synth.normal_grads(len(x), L, 153).astype(np.float64)
    dx = encoding.grid_encode_dx(x, tables, dout, base_res=base, growth=growth)
    want = np.zeros_like(dx)
    for l, N in enumerate(lattice.level_resolutions(L, base, growth)):
        xs = (x * np.float32(N)).astype(np.float64) / N
        for j in range(n):
            others = np.prod(np.delete(1.0 + cc * xs, j, axis=1), axis=1)
            want[:, j] += dout[:, l] * cc[j] * others
    np.testing.assert_allclose(dx, want, rtol=1e-9, atol=1e-9)


def _same_cells(kind, x, n, L, base, growth, log2_T):
    """Per level, the slot sets of the cell that contains each point."""
    out = []
    if kind == "simplex":
        scales = lattice.simplex_level_scales_fp32(n, L, base, growth)
        for l in range(L):
            out.append(np.sort(encoding.simplex_level_vertices(x, scales[l], log2_T)[0], axis=1))
    else:
        for N in lattice.grid_level_scales_fp32(L, base, growth):
            out.append(encoding.grid_level_vertices(x, N, log2_T)[0])
    return out


@pytest.mark.parametrize("kind,n", [("simplex", 2), ("simplex", 3), ("simplex", 5), ("grid", 2), ("grid", 3)])
def test_dx_matches_central_differences(kind, n):
    """Random tables: the input gradient equals the central difference of the forward pass for
    points whose cell (at every level) is the same at x - h e_j and x + h e_j."""
    L, base, growth, log2_T, F = 3, 4.0, 1.5, 12, 2
    tables = synth.uniform_tables(L, 1 << log2_T, F, 160 + n, scale=1.0)[0].astype(np.float64)
    x = synth.uniform_points(400, n, 161 + n)
    x = np.clip(x, 0.01, 0.99).astype(np.float32)
    dout = synth.normal_grads(len(x), L * F, 162).astype(np.float64)
    enc = encoding.simplex_encode if kind == "simplex" else encoding.grid_encode
    dxf = encoding.simplex_encode_dx if kind == "simplex" else encoding.grid_encode_dx
    dx, den = dxf(x, tables, dout, base_res=base, growth=growth, with_denominator=True)
    h = np.float32(2.0 ** -13)
    cells = _same_cells(kind, x, n, L, base, growth, log2_T)
    checked = 0
    for j in range(n):
        xp, xm = x.copy(), x.copy()
        xp[:, j] += h
        xm[:, j] -= h
        ok = np.ones(len(x), dtype=bool)
        for xx in (xp, xm):
            for c0, c1 in zip(cells, _same_cells(kind, xx, n, L, base, growth, log2_T)):
                ok &= np.all(c0 == c1, axis=1)
        fd = ((enc(xp, tables, base_res=base, growth=growth) - enc(xm, tables, base_res=base, growth=growth))
              * dout).sum(axis=1) / (2.0 * float(h))
        assert np.all(np.abs(fd - dx[:, j])[ok] <= 2e-3 * den[ok, j] + 1e-12)
        checked += ok.sum()
    assert checked > 100 * n


# --------------------------------------------------------------------------
# optional direct indexing of coarse levels
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n", [("simplex", 2), ("simplex", 3), ("simplex", 5), ("grid", 2), ("grid", 4)])
def test_dense_box_holds_every_vertex(kind, n):
    """The box width is N_l + 2 (the skewed unit cube spans [0, N_l]^n, Sec. 5.1) and every
    vertex of every point of [0,1]^n, faces and corners included, lies inside it."""
    L, base, growth = 4, 5.0, 1.7
    x = np.concatenate([synth.uniform_points(3000, n, 170), synth.edge_points(n, 171, per_kind=16)])
    if kind == "simplex":
        scales = lattice.simplex_level_scales_fp32(n, L, base, growth)
    else:
        scales = lattice.grid_level_scales_fp32(L, base, growth)
    for l, N in enumerate(lattice.level_resolutions(L, base, growth)):
        B = lattice.dense_box_width(kind, n, scales[l])
        assert B == N + 2
        if kind == "simplex":
            V = encoding.simplex_level_vertices(x, scales[l], 20)[2]
        else:
            c, _ = encoding.grid_level_cell(x, scales[l])
            V = c[:, None, :] + encoding._corner_offsets(n)[None]
        assert V.min() >= 0 and V.max() <= B - 1
        assert V.max() == B - 1                        # the corner x = 1 reaches the far face


@pytest.mark.parametrize("n", [2, 3, 4])
def test_dense_slots_are_a_bijection_of_the_box(n):
    B, log2_T = 7, 14
    box = np.stack(np.meshgrid(*([np.arange(B)] * n), indexing="ij"), -1).reshape(-1, n)
    s = lattice.dense_slot(box, B, log2_T)
    assert len(np.unique(s)) == B ** n and s.min() == 0 and s.max() == B ** n - 1
    # axis 0 fastest
    e = np.eye(n, dtype=np.int64)
    assert list(lattice.dense_slot(e, B, log2_T)) == [B ** i for i in range(n)]


def test_dense_levels_are_exactly_those_that_fit():
    L, base, growth, log2_T, n = 8, 16.0, 2.0, 16, 2
    scales = lattice.simplex_level_scales_fp32(n, L, base, growth)
    w = lattice.level_box_widths("simplex", n, scales, log2_T, lattice.INDEX_DENSE_COARSE)
    Ns = lattice.level_resolutions(L, base, growth)
    assert w == [N + 2 if (N + 2) ** 2 <= (1 << log2_T) else 0 for N in Ns]
    assert w[:4] == [18, 34, 66, 130] and w[4:] == [0] * 4          # 258^2 > 2^16
    assert lattice.level_box_widths("simplex", n, scales, log2_T, lattice.INDEX_HASH) == [0] * L
    # at the boundary: a grid level of resolution 254 needs a box of 256 = 2^8 coordinates, whose
    # 2^16 vertices exactly fill a table of 2^16 entries (stored directly); resolution 255 does not fit
    dense = lattice.INDEX_DENSE_COARSE
    assert lattice.level_box_widths("grid", 2, [np.float32(254), np.float32(255)], 16, dense) == [256, 0]


@pytest.mark.parametrize("kind,n", [("simplex", 2), ("simplex", 3), ("grid", 2), ("grid", 3)])
def test_dense_levels_reproduce_fields_with_a_small_table(kind, n):
    """With T far below what a collision-free hash needs, the directly indexed levels still
    reproduce affine (simplex) / multilinear (grid) fields exactly."""
    g = synth.rng(180 + n)
    a = g.standard_normal(n)
    fn = (lambda p: p @ a + 0.5) if kind == "simplex" else (lambda p: np.prod(1.0 + a * p, axis=-1))
    L, base, growth, log2_T = 4, 4.0, 1.5, 12
    T = 1 << log2_T
    if kind == "simplex":
        scales = lattice.simplex_level_scales_fp32(n, L, base, growth)
    else:
        scales = lattice.grid_level_scales_fp32(L, base, growth)
    widths = lattice.level_box_widths(kind, n, scales, log2_T, lattice.INDEX_DENSE_COARSE)
    assert all(widths)
    tables = np.zeros((L, T, 1))
    for l in range(L):
        B = widths[l]
        box = np.stack(np.meshgrid(*([np.arange(B)] * n), indexing="ij"), -1).reshape(-1, n)
        pos = lattice.unskew(box.astype(float)) if kind == "simplex" else box.astype(float)
        tables[l, lattice.dense_slot(box, B, log2_T), 0] = fn(pos / float(scales[l]))
    x = np.concatenate([synth.uniform_points(300, n, 181), synth.edge_points(n, 182, per_kind=4)])
    if kind == "simplex":
        out = encoding.simplex_encode(x, tables, base_res=base, growth=growth, index_mode=lattice.INDEX_DENSE_COARSE)
    else:
        out = encoding.grid_encode(x, tables, base_res=base, growth=growth, index_mode=lattice.INDEX_DENSE_COARSE)
    for l in range(L):
        if kind == "simplex":
            q = lattice.scaled_skewed_fp32(x, scales[l]).astype(np.float64)
            xs = lattice.unskew(q) / float(scales[l])
        else:
            xs = (x * np.float32(scales[l])).astype(np.float64) / float(scales[l])
        np.testing.assert_allclose(out[:, l], fn(xs), rtol=0, atol=1e-11)


# --------------------------------------------------------------------------
# forward paths with the level scale and skew in FP64
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 3, 4])
def test_fp64_paths_reproduce_affine_and_multilinear_fields(n):
    """With the scale and skew in FP64 the simplex encoding returns a.x + b at the point itself
    (not at a binary32 rounding of it), and the grid encoding prod_i (1 + c_i x_i)."""
    g = synth.rng(240 + n)
    a, b, cc = g.standard_normal(n), 0.4, g.standard_normal(n)
    L, growth = 3, 1.5
    base, log2_T = (4.0, 20) if n < 4 else (3.0, 22)
    x = np.concatenate([synth.uniform_points(300, n, 241), synth.edge_points(n, 242, per_kind=4)]).astype(np.float64)
    x[:50] += synth.rng(243).uniform(-1e-9, 1e-9, size=(50, n))       # off the binary32 grid
    x = np.clip(x, 0.0, 1.0)
    tab = _collision_free_tables("simplex", n, L, base, growth, log2_T, lambda p: p @ a + b, fp32_scale=False)
    out = encoding.simplex_encode_fp64(x, tab, base_res=base, growth=growth)
    for l in range(L):
        np.testing.assert_allclose(out[:, l], x @ a + b, rtol=0, atol=1e-11)
    fn = lambda p: np.prod(1.0 + cc * p, axis=-1)
    tab = _collision_free_tables("grid", n, L, base, growth, log2_T, fn)
    out = encoding.grid_encode_fp64(x, tab, base_res=base, growth=growth)
    for l in range(L):
        np.testing.assert_allclose(out[:, l], fn(x), rtol=0, atol=1e-11)


@pytest.mark.parametrize("kind,n", [("simplex", 2), ("simplex", 3), ("simplex", 5), ("grid", 2), ("grid", 4)])
def test_fp64_paths_agree_with_binary32_conditioned_paths(kind, n):
    """On binary32 points the FP64 paths differ from the binary32-conditioned ones only by the
    rounding of the scaled (skewed) coordinate: a few ulps of |q| times the interpolant's slope,
    bounded by 2 max |H| per unit of q (continuity carries the bound across cell faces)."""
    L, base, growth, log2_T, F = 4, 8.0, 1.5, 14, 2
    tables = synth.uniform_tables(L, 1 << log2_T, F, 250 + n, scale=1.0)[0].astype(np.float64)
    x = np.concatenate([synth.uniform_points(2000, n, 251 + n), synth.edge_points(n, 252, per_kind=8)])
    if kind == "simplex":
        a = encoding.simplex_encode(x, tables, base_res=base, growth=growth)
        b = encoding.simplex_encode_fp64(x, tables, base_res=base, growth=growth)
        top = np.array(lattice.simplex_level_scales_fp64(n, L, base, growth)) * (1 + n * lattice.skew_factor(n))
    else:
        a = encoding.grid_encode(x, tables, base_res=base, growth=growth)
        b = encoding.grid_encode_fp64(x, tables, base_res=base, growth=growth)
        top = np.array(lattice.level_resolutions(L, base, growth), dtype=float)
    for l in range(L):
        bound = (n + 2) * n * 2.0 ** -24 * top[l] * 2 * np.abs(tables[l]).max()
        assert np.abs(a[:, l * F:(l + 1) * F] - b[:, l * F:(l + 1) * F]).max() <= bound
    assert np.abs(a - b).max() > 0                       # the rounding is visible somewhere


def _fp64_cells(kind, x, n, L, base, growth, log2_T):
    """Per level, the sorted slot sets of the cell of each point under the FP64 scale and skew."""
    out = []
    if kind == "simplex":
        for s in lattice.simplex_level_scales_fp64(n, L, base, growth):
            c, order, _ = lattice.subdivide(lattice.skew(x * s))
            out.append(np.sort(lattice.slot_of(lattice.simplex_vertices(c, order), log2_T), axis=1))
    else:
        offs = np.array(list(itertools.product((0, 1), repeat=n)), dtype=np.int64)
        for N in lattice.level_resolutions(L, base, growth):
            c = np.floor(x * float(N)).astype(np.int64)
            out.append(lattice.slot_of(c[:, None, :] + offs[None], log2_T))
    return out


@pytest.mark.parametrize("kind,n", [("simplex", 2), ("simplex", 3), ("simplex", 4), ("grid", 2), ("grid", 3)])
def test_fp64_central_differences_equal_the_input_gradient(kind, n):
    """Central differences of the FP64 forward (h = 1e-7, exact on a linear piece up to FP64
    rounding) equal the input-gradient formula wherever the point's cells do not change, within
    1e-6 of the sum of the magnitudes of its terms (the formula uses the binary32 constants)."""
    L, base, growth, log2_T, F = 3, 4.0, 1.5, 12, 2
    tables = synth.uniform_tables(L, 1 << log2_T, F, 260 + n, scale=1.0)[0].astype(np.float64)
    x = np.clip(synth.uniform_points(400, n, 261 + n), 0.01, 0.99).astype(np.float32)
    dout = synth.normal_grads(len(x), L * F, 262).astype(np.float64)
    fwd = encoding.simplex_encode_fp64 if kind == "simplex" else encoding.grid_encode_fp64
    dxf = encoding.simplex_encode_dx if kind == "simplex" else encoding.grid_encode_dx
    dx, den = dxf(x, tables, dout, base_res=base, growth=growth, with_denominator=True)
    x64, h = x.astype(np.float64), 1e-7
    cells = _fp64_cells(kind, x64, n, L, base, growth, log2_T)
    checked = 0
    for j in range(n):
        xp, xm = x64.copy(), x64.copy()
        xp[:, j] += h
        xm[:, j] -= h
        ok = np.ones(len(x), dtype=bool)
        for xx in (xp, xm):
            for c0, c1 in zip(cells, _fp64_cells(kind, xx, n, L, base, growth, log2_T)):
                ok &= np.all(c0 == c1, axis=1)
        fd = ((fwd(xp, tables, base_res=base, growth=growth) - fwd(xm, tables, base_res=base, growth=growth))
              * dout).sum(axis=1) / (2.0 * h)
        assert np.all(np.abs(fd - dx[:, j])[ok] <= 1e-6 * den[ok, j] + 1e-12)
        checked += ok.sum()
    assert checked > 300 * n
