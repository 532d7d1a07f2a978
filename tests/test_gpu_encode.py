"""GPU parity of the encoding kernels against the FP64 oracle (through the C ABI).

Slots are compared bit for bit; weights, encodings and table gradients within the
tolerances of ``conftest.ENC_TOL`` measured against the sum of absolute terms."""
import numpy as np
import pytest
import torch

from conftest import ENC_ATOL, ENC_TOL, record_error, rel_err, worst_ratio
from oracle import encoding as O
from oracle import render as OR
from oracle import lattice
from paper_2311_15439_gb300 import synth

pytestmark = pytest.mark.gpu

# (d, L, F, log2_T, base, growth, table dtype, out dtype, P)
CASES = [
    (2, 8, 2, 14, 16.0, 1.5, "f32", "f32", 65536),       # plain FP32 workload, full size
    (2, 16, 2, 22, 16.0, 2.0, "f16", "f16", 1 << 14),     # image-style tables
    (3, 16, 2, 19, 16.0, 1.38, "bf16", "bf16", 1 << 13),  # SDF-style tables
    (3, 16, 2, 19, 16.0, 1.38, "f16", "f32", 5000),
    (4, 16, 2, 19, 16.0, 1.38, "f16", "f16", 3000),
    (5, 16, 2, 19, 16.0, 1.38, "f16", "f16", 3000),
    (2, 4, 1, 12, 8.0, 2.0, "f32", "f32", 4999),
    (3, 5, 4, 12, 8.0, 2.0, "f32", "bf16", 3001),
    (4, 3, 8, 10, 4.0, 1.5, "f32", "f32", 777),
    (2, 32, 1, 12, 4.0, 1.2, "f32", "f32", 2000),        # the most levels (32), a power of two
    (3, 20, 2, 13, 8.0, 1.15, "f16", "f16", 1500),       # levels not a power of two
]


def _ids(c):
    return "d%d_L%d_F%d_T%d_%s_%s_P%d" % (c[0], c[1], c[2], c[3], c[6], c[7], c[8])


def _points(d, P, seed):
    return np.concatenate([synth.uniform_points(P, d, seed), synth.edge_points(d, seed + 1, per_kind=8)])


def _setup(cuda_lib, case, kind, seed=0):
    from paper_2311_15439_gb300.api import Encoder
    d, L, F, log2_T, base, growth, tdt, odt, P = case
    enc = Encoder(d, L, F, log2_T, base, growth, kind=kind, table_dtype=tdt, out_dtype=odt)
    vals, store = synth.uniform_tables(L, 1 << log2_T, F, seed + 2, dtype=tdt, scale=1e-4)
    t = torch.from_numpy(store.astype(np.int16) if tdt == "bf16" else store).cuda()
    if tdt == "bf16":
        t = t.view(torch.bfloat16)
    x = _points(d, P, seed + 3)
    return enc, vals, t, x


@pytest.mark.parametrize("kind", ["simplex", "grid"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_vertices_bit_exact(cuda_lib, case, kind):
    """Lattice slots equal the oracle's bit for bit (given the same binary32 skewed point);
    weights agree to binary32 rounding."""
    enc, _, _, x = _setup(cuda_lib, case, kind)
    d, L, F, log2_T, base, growth = case[:6]
    slots, w = enc.encode_vertices(torch.from_numpy(x).cuda())
    slots, w = slots.cpu().numpy(), w.cpu().numpy()
    if kind == "simplex":
        scales = lattice.simplex_level_scales_fp32(d, L, base, growth)
        for l in range(L):
            s_ref, w_ref, _ = O.simplex_level_vertices(x, scales[l], log2_T)
            assert np.array_equal(slots[:, l, :].astype(np.int64), s_ref), "level %d" % l
            assert np.max(np.abs(w[:, l, :] - w_ref)) <= 2.0 ** -23
    else:
        res = lattice.grid_level_scales_fp32(L, base, growth)
        for l in range(L):
            s_ref, w_ref = O.grid_level_vertices(x, res[l], log2_T)
            assert np.array_equal(slots[:, l, :].astype(np.int64), s_ref), "level %d" % l
            assert np.max(np.abs(w[:, l, :] - w_ref)) <= (2 * d + 1) * 2.0 ** -24


@pytest.mark.parametrize("kind", ["simplex", "grid"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_forward_matches_oracle(cuda_lib, case, kind):
    enc, vals, t, x = _setup(cuda_lib, case, kind)
    base, growth = case[4], case[5]
    out = enc.encode_fwd(torch.from_numpy(x).cuda(), t).float().cpu().numpy()
    if kind == "simplex":
        ref, den = O.simplex_encode(x, vals, base_res=base, growth=growth, with_denominator=True)
    else:
        ref = O.grid_encode(x, vals, base_res=base, growth=growth)
        den = O.grid_encode(x, np.abs(vals), base_res=base, growth=growth)   # weights are >= 0
    tol = ENC_TOL[case[7]]
    r = worst_ratio(out, ref, den, tol, ENC_ATOL[case[7]])
    record_error("encode_fwd %s output, %s tables (%s)" % (case[7], case[6], kind), r * tol, tol, "sum_k |w_k H_k| (+ fp16 subnormal spacing)")
    assert r <= 1.0
    if case[7] == "f32":
        # reported, not a parity gate: the binary32 rounding of the scaled (skewed) coordinate, the
        # library against the oracle's path that scales and skews in FP64
        f64 = O.simplex_encode_fp64 if kind == "simplex" else O.grid_encode_fp64
        ref64 = f64(x.astype(np.float64), vals, base_res=base, growth=growth)
        record_error("binary32 quantisation of the skewed coordinate (%s, reported only)" % kind,
                     rel_err(out, ref64, den), 1.0, "sum_k |w_k H_k|")


@pytest.mark.parametrize("kind", ["simplex", "grid"])
@pytest.mark.parametrize("case", [c for c in CASES if c[3] <= 19], ids=_ids)
def test_backward_matches_oracle(cuda_lib, case, kind):
    """Table gradients (binary32 atomics) agree with the FP64 scatter-add within 1e-5 of
    sum |w_k dout|; untouched entries stay exactly zero."""
    enc, _, _, x = _setup(cuda_lib, case, kind)
    d, L, F, log2_T, base, growth = case[:6]
    dout = synth.normal_grads(len(x), L * F, 7)
    grad = torch.zeros((L, 1 << log2_T, F), dtype=torch.float32, device="cuda")
    enc.encode_bwd(torch.from_numpy(x).cuda(), torch.from_numpy(dout).cuda(), grad)
    g = grad.cpu().numpy()
    kw = dict(n_levels=L, log2_T=log2_T, n_features=F, base_res=base, growth=growth)
    if kind == "simplex":
        ref, den = O.simplex_encode_bwd(x, dout, with_denominator=True, **kw)
    else:
        ref = O.grid_encode_bwd(x, dout, **kw)
        den = O.grid_encode_bwd(x, np.abs(dout), **kw)
    for l in range(L):
        e = record_error("encode_bwd table gradient (%s)" % kind, rel_err(g[l], ref[l], den[l]), 1e-5, "sum_k |w_k dout| per entry")
        assert e <= 1e-5, "level %d" % l
        assert np.all(g[l][den[l] == 0] == 0)


def test_full_size_image_workload(cuda_lib):
    """2^18 points, L = 16, T = 2^22 fp16 tables, the launch the benchmark times: every output
    and every table-gradient entry of all 16 levels against the oracle."""
    case = (2, 16, 2, 22, 16.0, 2.0, "f16", "f16", 1 << 18)
    enc, vals, t, x = _setup(cuda_lib, case, "simplex", seed=11)
    x = x[: 1 << 18]
    xd = torch.from_numpy(x).cuda()
    out = enc.encode_fwd(xd, t).float().cpu().numpy()
    ref, den = O.simplex_encode(x, vals, base_res=16.0, growth=2.0, with_denominator=True)
    r = worst_ratio(out, ref, den, ENC_TOL["f16"], ENC_ATOL["f16"])
    record_error("encode_fwd f16 output, image workload at full size", r * ENC_TOL["f16"], ENC_TOL["f16"], "sum_k |w_k H_k| (+ fp16 subnormal spacing)")
    assert r <= 1.0
    dout = synth.normal_grads(len(x), 32, 12)
    grad = torch.zeros((16, 1 << 22, 2), dtype=torch.float32, device="cuda")
    enc.encode_bwd(xd, torch.from_numpy(dout).cuda(), grad)
    for l in range(16):                                  # every level, one at a time (1 GiB of FP64 each)
        ref, den = O.simplex_encode_bwd(x, dout, n_levels=16, log2_T=22, n_features=2, base_res=16.0, growth=2.0,
                                        levels=[l], with_denominator=True)
        g = grad[l].cpu().numpy()
        e = record_error("encode_bwd table gradient, image workload at full size", rel_err(g, ref[l], den[l]), 1e-5,
                         "sum_k |w_k dout| per entry")
        assert e <= 1e-5, "level %d" % l
        assert np.all(g[den[l] == 0] == 0), "level %d" % l


def test_strided_gradient_and_touched_bitmap(cuda_lib):
    """Gradients written into interleaved records (stride 4F, offset 3F) equal the dense ones,
    nothing else in the records changes, and exactly the entries with a term are marked."""
    case = (3, 6, 2, 12, 8.0, 1.7, "f16", "f16", 3000)
    enc, _, _, x = _setup(cuda_lib, case, "simplex")
    L, F, T = 6, 2, 1 << 12
    xd = torch.from_numpy(x).cuda()
    dout = torch.from_numpy(synth.normal_grads(len(x), L * F, 3)).cuda()
    dense = torch.zeros((L, T, F), dtype=torch.float32, device="cuda")
    enc.encode_bwd(xd, dout, dense)
    state = torch.randn((L * T, 4 * F), device="cuda")
    state[:, 3 * F:] = 0
    before = state.clone()
    touched = torch.zeros(((L * T + 31) // 32,), dtype=torch.int32, device="cuda")
    enc.encode_bwd(xd, dout, state, grad_stride=4 * F, grad_offset=3 * F, touched=touched)
    torch.cuda.synchronize()
    assert torch.equal(state[:, :3 * F], before[:, :3 * F])
    g_dense = dense.reshape(L * T, F).cpu().numpy()
    g_rec = state[:, 3 * F:].cpu().numpy()
    assert np.max(np.abs(g_dense - g_rec)) <= 1e-5 * np.max(np.abs(g_dense))
    bits = touched.cpu().numpy().view(np.uint32)
    marked = ((bits[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1).ravel()[: L * T].astype(bool)
    scales = lattice.simplex_level_scales_fp32(3, L, 8.0, 1.7)
    want = np.zeros(L * T, dtype=bool)
    for l in range(L):
        s, _, _ = O.simplex_level_vertices(x, scales[l], 12)
        want[l * T + s.ravel()] = True
    assert np.array_equal(marked, want)


def test_zero_points_and_errors(cuda_lib):
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300._lib import SxeError
    enc = Encoder(2, 4, 2, 10, 8.0, 1.5, table_dtype="f32")
    t = torch.zeros((4, 1024, 2), device="cuda")
    out = enc.encode_fwd(torch.zeros((0, 2), device="cuda"), t)
    assert out.shape == (0, 8)
    with pytest.raises(TypeError):
        enc.encode_fwd(torch.zeros((4, 2), device="cuda", dtype=torch.float64), t)
    with pytest.raises(SxeError):
        enc.encode_bwd(torch.zeros((4, 2), device="cuda"), torch.zeros((4, 8), device="cuda"),
                       torch.zeros((4 * 1024 * 3,), device="cuda"), grad_stride=3)


def test_out_of_domain_points_stay_in_bounds(cuda_lib):
    """Points outside [0,1]^d (negative, > 1, huge) and NaN still produce slots inside the
    table (defined behaviour for finite points, no out-of-bounds access for NaN)."""
    from paper_2311_15439_gb300.api import Encoder
    enc = Encoder(3, 8, 2, 12, 16.0, 1.5, table_dtype="f32")
    x = np.array([[-0.5, 2.0, 0.3], [1e4, -1e4, 5.0], [np.nan, 0.2, 0.3], [1.0, 1.0, 1.0]], dtype=np.float32)
    slots, w = enc.encode_vertices(torch.from_numpy(x).cuda())
    s = slots.cpu().numpy()
    assert s.min() >= 0 and s.max() < 4096
    scales = lattice.simplex_level_scales_fp32(3, 8, 16.0, 1.5)
    for l in range(8):
        ref, _, _ = O.simplex_level_vertices(x[[0, 1, 3]], scales[l], 12)
        assert np.array_equal(s[[0, 1, 3], l, :].astype(np.int64), ref)


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_plain_path_matches_oracle(cuda_lib, d):
    """The plain binary32 comparator path (bubble sort, scalar loads and atomics) computes the
    same encoding and table gradient as the oracle."""
    from paper_2311_15439_gb300.api import Encoder
    L, log2_T = 8, 14
    enc = Encoder(d, L, 2, log2_T, 16.0, 1.5, table_dtype="f32")
    vals = synth.uniform_tables(L, 1 << log2_T, 2, 20 + d, scale=1e-4)[0]
    x = _points(d, 3000, 30 + d)
    xd = torch.from_numpy(x).cuda()
    out = enc.encode_plain_fwd(xd, torch.from_numpy(vals).cuda()).cpu().numpy()
    ref, den = O.simplex_encode(x, vals, base_res=16.0, growth=1.5, with_denominator=True)
    assert record_error("encode_plain_fwd f32 output", rel_err(out, ref, den), 1e-5, "sum_k |w_k H_k| (+ fp16 subnormal spacing)") <= 1e-5
    dout = synth.normal_grads(len(x), L * 2, 40 + d)
    grad = torch.zeros((L, 1 << log2_T, 2), device="cuda")
    enc.encode_plain_bwd(xd, torch.from_numpy(dout).cuda(), grad)
    gref, gden = O.simplex_encode_bwd(x, dout, n_levels=L, log2_T=log2_T, n_features=2, base_res=16.0,
                                      growth=1.5, with_denominator=True)
    g = grad.cpu().numpy()
    for l in range(L):
        assert record_error("encode_plain_bwd table gradient", rel_err(g[l], gref[l], gden[l]), 1e-5, "sum_k |w_k dout| per entry") <= 1e-5


def test_full_size_sdf_workload(cuda_lib):
    """SDF-style configuration at full size: d = 3, L = 16, F = 2, T = 2^19 bf16 tables and
    output, growth 1.38, 2^20 points (half near a union of spheres and tori): every output
    against the oracle, gradients of three levels."""
    from paper_2311_15439_gb300.api import Encoder
    enc = Encoder(3, 16, 2, 19, 16.0, 1.38, table_dtype="bf16", out_dtype="bf16")
    vals, bits = synth.uniform_tables(16, 1 << 19, 2, 70, dtype="bf16", scale=1e-4)
    t = torch.from_numpy(bits.astype(np.int16)).cuda().view(torch.bfloat16)
    x = synth.sdf_points(1 << 20, 71)
    xd = torch.from_numpy(x).cuda()
    out = enc.encode_fwd(xd, t).float().cpu().numpy()
    ref, den = O.simplex_encode(x, vals, base_res=16.0, growth=1.38, with_denominator=True)
    r = worst_ratio(out, ref, den, ENC_TOL["bf16"], ENC_ATOL["bf16"])
    record_error("encode_fwd bf16 output, SDF workload at full size", r * ENC_TOL["bf16"], ENC_TOL["bf16"], "sum_k |w_k H_k| (+ fp16 subnormal spacing)")
    assert r <= 1.0
    dout = synth.normal_grads(len(x), 32, 72)
    grad = torch.zeros((16, 1 << 19, 2), dtype=torch.float32, device="cuda")
    enc.encode_bwd(xd, torch.from_numpy(dout).cuda(), grad)
    levels = [0, 8, 15]
    gref, gden = O.simplex_encode_bwd(x, dout, n_levels=16, log2_T=19, n_features=2, base_res=16.0, growth=1.38,
                                      levels=levels, with_denominator=True)
    for l in levels:
        e = rel_err(grad[l].cpu().numpy(), gref[l], gden[l])
        assert record_error("encode_bwd table gradient, SDF workload at full size", e, 1e-5, "sum_k |w_k dout| per entry") <= 1e-5


DX_CASES = [c for c in CASES if c[8] <= 1 << 14]


@pytest.mark.parametrize("kind", ["simplex", "grid"])
@pytest.mark.parametrize("case", DX_CASES, ids=_ids)
def test_input_gradient_matches_oracle(cuda_lib, case, kind):
    """dL/dx through the C ABI against the oracle's chain rule, every point and axis, within
    1e-5 of the sum of the magnitudes of the terms (binary32 products and sums)."""
    enc, vals, t, x = _setup(cuda_lib, case, kind, seed=20)
    d, L, F = case[:3]
    if kind == "grid" and d > 4:                # 2^5 corners: 400 uniform points and every edge point
        x = np.concatenate([x[:400], x[case[8]:]])
    base, growth = case[4], case[5]
    dout = synth.normal_grads(len(x), L * F, 21)
    dx = enc.encode_bwd_input(torch.from_numpy(x).cuda(), t, torch.from_numpy(dout).cuda()).cpu().numpy()
    f = O.simplex_encode_dx if kind == "simplex" else O.grid_encode_dx
    ref, den = f(x, vals, dout, base_res=base, growth=growth, with_denominator=True)
    e = float(np.max(np.abs(dx - ref) / (den + 1e-30)))
    record_error("encode_bwd_input dL/dx (%s)" % kind, e, 1e-5, "sum of |terms| of each dL/dx_i")
    assert np.all(np.abs(dx - ref) <= 1e-5 * den + 1e-30)


def test_input_gradient_accumulates_and_handles_empty(cuda_lib):
    from paper_2311_15439_gb300.api import Encoder
    enc = Encoder(3, 6, 2, 12, 8.0, 2.0, table_dtype="f32")
    vals, _ = synth.uniform_tables(6, 1 << 12, 2, 30)
    t = torch.from_numpy(vals).cuda()
    x = torch.from_numpy(synth.uniform_points(1000, 3, 31)).cuda()
    dout = torch.from_numpy(synth.normal_grads(1000, 12, 32)).cuda()
    once = enc.encode_bwd_input(x, t, dout)
    twice = enc.encode_bwd_input(x, t, dout, dx=once.clone())
    torch.testing.assert_close(twice, 2 * once, rtol=1e-6, atol=0)
    empty = enc.encode_bwd_input(x[:0], t, dout[:0])
    assert empty.shape == (0, 3)


def test_input_gradient_full_size_sdf(cuda_lib):
    """SDF-style configuration at full size (d = 3, L = 16, T = 2^19 bf16, 2^20 points, one
    launch as the training path runs it): a 4096-point sample against the oracle."""
    from paper_2311_15439_gb300.api import Encoder
    enc = Encoder(3, 16, 2, 19, 16.0, 1.38, table_dtype="bf16")
    vals, bits = synth.uniform_tables(16, 1 << 19, 2, 80, dtype="bf16", scale=1e-2)
    t = torch.from_numpy(bits.astype(np.int16)).cuda().view(torch.bfloat16)
    x = synth.sdf_points(1 << 20, 81)
    dout = synth.normal_grads(len(x), 32, 82)
    dx = enc.encode_bwd_input(torch.from_numpy(x).cuda(), t, torch.from_numpy(dout).cuda()).cpu().numpy()
    idx = synth.rng(83).choice(len(x), 4096, replace=False)
    ref, den = O.simplex_encode_dx(x[idx], vals, dout[idx], base_res=16.0, growth=1.38, with_denominator=True)
    assert np.all(np.abs(dx[idx] - ref) <= 1e-5 * den + 1e-30)


DENSE_CASES = [
    (2, 8, 2, 16, 16.0, 2.0, "f16", "f16", 5000),      # levels 0-3 direct (130^2 <= 2^16 < 258^2)
    (3, 6, 2, 16, 8.0, 1.5, "f32", "f32", 3000),
    (4, 4, 2, 18, 4.0, 1.5, "bf16", "bf16", 2000),
    (5, 3, 1, 20, 3.0, 1.5, "f32", "f32", 1500),
]


@pytest.mark.parametrize("kind", ["simplex", "grid"])
@pytest.mark.parametrize("case", DENSE_CASES, ids=_ids)
def test_dense_coarse_levels_match_oracle(cuda_lib, case, kind):
    """Direct indexing of the levels that fit: box widths equal the oracle's, slots bit for
    bit, forward, table gradient and input gradient within the usual tolerances."""
    from paper_2311_15439_gb300.api import Encoder
    from oracle.lattice import INDEX_DENSE_COARSE, level_box_widths
    d, L, F, log2_T, base, growth, tdt, odt, P = case
    enc = Encoder(d, L, F, log2_T, base, growth, kind=kind, table_dtype=tdt, out_dtype=odt, index_mode="dense_coarse")
    vals, store = synth.uniform_tables(L, 1 << log2_T, F, 90, dtype=tdt, scale=1e-2)
    t = torch.from_numpy(store.astype(np.int16) if tdt == "bf16" else store).cuda()
    if tdt == "bf16":
        t = t.view(torch.bfloat16)
    x = _points(d, P, 91)
    xd = torch.from_numpy(x).cuda()
    if kind == "simplex":
        scales = lattice.simplex_level_scales_fp32(d, L, base, growth)
    else:
        scales = lattice.grid_level_scales_fp32(L, base, growth)
    widths = level_box_widths(kind, d, scales, log2_T, INDEX_DENSE_COARSE)
    assert list(enc.level_index()) == widths and any(widths)
    slots = enc.encode_vertices(xd)[0].cpu().numpy()
    for l in range(L):
        if kind == "simplex":
            s_ref = O.simplex_level_vertices(x, scales[l], log2_T, widths[l])[0]
        else:
            s_ref = O.grid_level_vertices(x, scales[l], log2_T, widths[l])[0]
        assert np.array_equal(slots[:, l, :].astype(np.int64), s_ref), "level %d" % l
    kw = dict(base_res=base, growth=growth, index_mode=INDEX_DENSE_COARSE)
    out = enc.encode_fwd(xd, t).float().cpu().numpy()
    if kind == "simplex":
        ref, den = O.simplex_encode(x, vals, with_denominator=True, **kw)
    else:
        ref = O.grid_encode(x, vals, **kw)
        den = O.grid_encode(x, np.abs(vals), **kw)
    assert worst_ratio(out, ref, den, ENC_TOL[odt], ENC_ATOL[odt]) <= 1.0
    dout = synth.normal_grads(len(x), L * F, 92)
    dd = torch.from_numpy(dout).cuda()
    grad = torch.zeros((L, 1 << log2_T, F), dtype=torch.float32, device="cuda")
    enc.encode_bwd(xd, dd, grad)
    g = grad.cpu().numpy()
    bkw = dict(n_levels=L, log2_T=log2_T, n_features=F, **kw)
    if kind == "simplex":
        gref, gden = O.simplex_encode_bwd(x, dout, with_denominator=True, **bkw)
    else:
        gref = O.grid_encode_bwd(x, dout, **bkw)
        gden = O.grid_encode_bwd(x, np.abs(dout), **bkw)
    for l in range(L):
        assert rel_err(g[l], gref[l], gden[l]) <= 1e-5, "level %d" % l
    if not (kind == "grid" and d == 5):
        dx = enc.encode_bwd_input(xd, t, dd).cpu().numpy()
        f = O.simplex_encode_dx if kind == "simplex" else O.grid_encode_dx
        xref, xden = f(x, vals, dout, with_denominator=True, **kw)
        assert np.all(np.abs(dx - xref) <= 1e-5 * xden + 1e-30)


@pytest.mark.parametrize("kind,index_mode", [("simplex", "hash"), ("grid", "dense_coarse")])
def test_backward_by_level_ranges(cuda_lib, kind, index_mode):
    """sxe_encode_bwd_levels: ranges that cut through the shared-memory coarse levels and the
    rest, run one after the other, give the oracle's gradient and bitmap; a single range adds
    and marks nothing outside its levels."""
    from paper_2311_15439_gb300.api import Encoder
    from oracle.lattice import INDEX_DENSE_COARSE, INDEX_HASH
    d, L, F, log2_T, base, growth = 2, 6, 2, 14, 8.0, 1.6
    T = 1 << log2_T
    enc = Encoder(d, L, F, log2_T, base, growth, kind=kind, table_dtype="f32", index_mode=index_mode)
    P = 40000
    assert enc.bwd_kernel_count(P) == 2
    ranges = [(0, 1), (1, 1), (1, 3), (3, 4), (4, 6)]
    assert sum(enc.bwd_kernel_count(P, levels=r) for r in ranges) >= 4
    x = synth.uniform_points(P, d, 98)
    xd = torch.from_numpy(x).cuda()
    dout = synth.normal_grads(P, L * F, 99)
    dd = torch.from_numpy(dout).cuda()
    state = torch.zeros((L * T, 4 * F), device="cuda")
    bm = torch.zeros(((L * T + 31) // 32,), dtype=torch.int32, device="cuda")
    enc.encode_bwd(xd, dd, state, grad_stride=4 * F, grad_offset=3 * F, touched=bm, levels=(1, 3))
    grad = state[:, 3 * F:].reshape(L, T, F)
    bits = np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little").astype(bool)[: L * T]
    outside = np.r_[0:T, 3 * T:L * T]
    assert torch.all(grad[0] == 0) and torch.all(grad[3:] == 0) and not bits[outside].any()
    assert bits[T:3 * T].any()
    state.zero_()
    bm.zero_()
    for r in ranges:
        enc.encode_bwd(xd, dd, state, grad_stride=4 * F, grad_offset=3 * F, touched=bm, levels=r)
    grad = state[:, 3 * F:].reshape(L, T, F).cpu().numpy()
    mode = INDEX_DENSE_COARSE if index_mode == "dense_coarse" else INDEX_HASH
    kw = dict(n_levels=L, log2_T=log2_T, n_features=F, base_res=base, growth=growth, index_mode=mode)
    if kind == "simplex":
        ref, den = O.simplex_encode_bwd(x, dout, with_denominator=True, **kw)
        scales = lattice.simplex_level_scales_fp32(d, L, base, growth)
    else:
        ref = O.grid_encode_bwd(x, dout, **kw)
        den = O.grid_encode_bwd(x, np.abs(dout), **kw)
        scales = lattice.grid_level_scales_fp32(L, base, growth)
    widths = lattice.level_box_widths(kind, d, scales, log2_T, mode)
    want = np.zeros(L * T, dtype=bool)
    for l in range(L):
        assert rel_err(grad[l], ref[l], den[l]) <= 1e-5, "level %d" % l
        vert = O.simplex_level_vertices if kind == "simplex" else O.grid_level_vertices
        want[l * T + np.unique(vert(x, scales[l], log2_T, widths[l])[0])] = True
    bits = np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little").astype(bool)[: L * T]
    assert np.array_equal(bits, want)


@pytest.mark.parametrize("kind,d,points,index_mode", [("simplex", 3, "rays", "hash"), ("grid", 3, "rays", "hash"),
                                                      ("simplex", 2, "uniform", "hash"),
                                                      ("simplex", 3, "rays", "dense_coarse"),
                                                      ("simplex", 5, "uniform", "hash")])
def test_aggregated_backward_matches_oracle(cuda_lib, kind, d, points, index_mode):
    """Backward with warp-level sums of colliding terms (sxe_encoder_set_bwd_aggregation): the
    gradient equals the oracle's and the bitmap marks exactly the entries that received a term,
    on coherent ray samples (many lanes of a warp share vertices) and on uniform points (almost
    none do), with a ragged last block of points; also through a level range."""
    from paper_2311_15439_gb300.api import Encoder
    from oracle.lattice import INDEX_DENSE_COARSE, INDEX_HASH
    L, F, log2_T, base, growth = 8, 2, 14, 6.0, 1.5
    T = 1 << log2_T
    enc = Encoder(d, L, F, log2_T, base, growth, kind=kind, table_dtype="f32", index_mode=index_mode)
    enc.set_bwd_aggregation(True)
    if points == "rays":
        R, S = 301, 33
        o, dd, tn, tf = synth.camera_rays(R, 120)
        x = OR.ray_samples_fp32(o, dd, tn, tf, S)[0]
    else:
        x = synth.uniform_points(20011, d, 121)
    P = x.shape[0]
    dout = synth.normal_grads(P, L * F, 122)
    xd, dd_ = torch.from_numpy(x).cuda(), torch.from_numpy(dout).cuda()
    state = torch.zeros((L * T, 4 * F), device="cuda")
    bm = torch.zeros(((L * T + 31) // 32,), dtype=torch.int32, device="cuda")
    enc.encode_bwd(xd, dd_, state, grad_stride=4 * F, grad_offset=3 * F, touched=bm, levels=(0, 3))
    enc.encode_bwd(xd, dd_, state, grad_stride=4 * F, grad_offset=3 * F, touched=bm, levels=(3, L))
    grad = state[:, 3 * F:].reshape(L, T, F).cpu().numpy()
    mode = INDEX_DENSE_COARSE if index_mode == "dense_coarse" else INDEX_HASH
    kw = dict(n_levels=L, log2_T=log2_T, n_features=F, base_res=base, growth=growth, index_mode=mode)
    if kind == "simplex":
        ref, den = O.simplex_encode_bwd(x, dout, with_denominator=True, **kw)
        scales = lattice.simplex_level_scales_fp32(d, L, base, growth)
    else:
        ref = O.grid_encode_bwd(x, dout, **kw)
        den = O.grid_encode_bwd(x, np.abs(dout), **kw)
        scales = lattice.grid_level_scales_fp32(L, base, growth)
    widths = lattice.level_box_widths(kind, d, scales, log2_T, mode)
    want = np.zeros(L * T, dtype=bool)
    for l in range(L):
        assert rel_err(grad[l], ref[l], den[l]) <= 1e-5, "level %d" % l
        vert = O.simplex_level_vertices if kind == "simplex" else O.grid_level_vertices
        want[l * T + np.unique(vert(x, scales[l], log2_T, widths[l])[0])] = True
    bits = np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little").astype(bool)[: L * T]
    assert np.array_equal(bits, want)


@pytest.mark.parametrize("kind,d,index_mode", [("simplex", 2, "hash"), ("simplex", 3, "hash"), ("grid", 2, "hash"),
                                               ("simplex", 2, "dense_coarse"), ("grid", 3, "dense_coarse")])
def test_coarse_levels_summed_per_block(cuda_lib, kind, d, index_mode):
    """Backward with the coarse levels summed per thread block in shared memory (two kernels):
    gradients in interleaved records equal the oracle's, points outside the box (x in
    [-0.3, 1.3]) included, and the bitmap marks exactly the entries that received a term."""
    from paper_2311_15439_gb300.api import Encoder
    from oracle.lattice import INDEX_DENSE_COARSE, INDEX_HASH
    L, F, log2_T, base, growth = 6, 2, 14, 8.0, 1.6
    T = 1 << log2_T
    enc = Encoder(d, L, F, log2_T, base, growth, kind=kind, table_dtype="f32", index_mode=index_mode)
    P = 40000
    assert enc.bwd_kernel_count(P) == 2
    g = synth.rng(95 + d)
    x = g.uniform(-0.3, 1.3, size=(P, d)).astype(np.float32)
    x[: P // 2] = synth.uniform_points(P // 2, d, 96)
    xd = torch.from_numpy(x).cuda()
    dout = synth.normal_grads(P, L * F, 97)
    state = torch.zeros((L * T, 4 * F), device="cuda")
    bm = torch.zeros(((L * T + 31) // 32,), dtype=torch.int32, device="cuda")
    enc.encode_bwd(xd, torch.from_numpy(dout).cuda(), state, grad_stride=4 * F, grad_offset=3 * F, touched=bm)
    grad = state[:, 3 * F:].reshape(L, T, F).cpu().numpy()
    assert torch.all(state[:, :3 * F] == 0)
    mode = INDEX_DENSE_COARSE if index_mode == "dense_coarse" else INDEX_HASH
    kw = dict(n_levels=L, log2_T=log2_T, n_features=F, base_res=base, growth=growth, index_mode=mode)
    if kind == "simplex":
        ref, den = O.simplex_encode_bwd(x, dout, with_denominator=True, **kw)
        scales = lattice.simplex_level_scales_fp32(d, L, base, growth)
    else:
        ref = O.grid_encode_bwd(x, dout, **kw)
        den = O.grid_encode_bwd(x, np.abs(dout), **kw)
        scales = lattice.grid_level_scales_fp32(L, base, growth)
    widths = lattice.level_box_widths(kind, d, scales, log2_T, mode)
    want = np.zeros(L * T, dtype=bool)
    for l in range(L):
        assert rel_err(grad[l], ref[l], den[l]) <= 1e-5, "level %d" % l
        if kind == "simplex":
            sl = O.simplex_level_vertices(x, scales[l], log2_T, widths[l])[0]
        else:
            sl = O.grid_level_vertices(x, scales[l], log2_T, widths[l])[0]
        want[l * T + np.unique(sl)] = True
    bits = np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little").astype(bool)[: L * T]
    assert np.array_equal(bits, want)


# Sec. 5.2's equal-memory setting: every simplex level scaled by (n+1)^((n-1)/(2n)), so that the
# touched simplex lattice is as large as the grid's at the same N_l (the comparison setting).
EQ_CASES = [
    (2, 16, 2, 19, 16.0, 1.38, "f16", "f16", 4000),
    (3, 16, 2, 19, 16.0, 1.38, "bf16", "bf16", 4000),
    (4, 16, 2, 19, 16.0, 1.38, "f16", "f32", 3000),
    (5, 16, 2, 19, 16.0, 1.38, "f16", "f16", 3000),
    (2, 16, 2, 22, 16.0, 2.0, "f16", "f16", 1 << 14),      # image-style tables, finest N = 524288
    (3, 6, 4, 12, 8.0, 2.0, "f32", "f32", 2001),
]


def _eq_setup(case, seed=40):
    from paper_2311_15439_gb300.api import Encoder
    d, L, F, log2_T, base, growth, tdt, odt, P = case
    enc = Encoder(d, L, F, log2_T, base, growth, res_mode="equal_mem", table_dtype=tdt, out_dtype=odt)
    vals, store = synth.uniform_tables(L, 1 << log2_T, F, seed, dtype=tdt, scale=1e-4)
    t = torch.from_numpy(store.astype(np.int16) if tdt == "bf16" else store).cuda()
    if tdt == "bf16":
        t = t.view(torch.bfloat16)
    return enc, vals, t, _points(d, P, seed + 1)


@pytest.mark.parametrize("case", EQ_CASES, ids=_ids)
def test_equal_mem_vertices_forward_backward(cuda_lib, case):
    """res_mode = equal_mem: the binary32 level multipliers equal the oracle's, slots are bit-exact,
    weights within 2^-23, encodings and table gradients within the stated tolerances."""
    d, L, F, log2_T, base, growth, tdt, odt, P = case
    enc, vals, t, x = _eq_setup(case)
    eq = lattice.RES_EQUAL_MEM
    scales = lattice.simplex_level_scales_fp32(d, L, base, growth, eq)
    assert np.array_equal(enc.level_params()[0], scales)
    assert np.all(scales > lattice.simplex_level_scales_fp32(d, L, base, growth))
    xd = torch.from_numpy(x).cuda()
    slots, w = enc.encode_vertices(xd)
    slots, w = slots.cpu().numpy(), w.cpu().numpy()
    for l in range(L):
        s_ref, w_ref, _ = O.simplex_level_vertices(x, scales[l], log2_T)
        assert np.array_equal(slots[:, l, :].astype(np.int64), s_ref), "level %d" % l
        assert np.max(np.abs(w[:, l, :] - w_ref)) <= 2.0 ** -23
    out = enc.encode_fwd(xd, t).float().cpu().numpy()
    ref, den = O.simplex_encode(x, vals, base_res=base, growth=growth, res_mode=eq, with_denominator=True)
    r = worst_ratio(out, ref, den, ENC_TOL[odt], ENC_ATOL[odt])
    record_error("encode_fwd %s output, %s tables (simplex, equal_mem)" % (odt, tdt), r * ENC_TOL[odt], ENC_TOL[odt],
                 "sum_k |w_k H_k| (+ fp16 subnormal spacing)")
    assert r <= 1.0
    dout = synth.normal_grads(len(x), L * F, 42)
    grad = torch.zeros((L, 1 << log2_T, F), dtype=torch.float32, device="cuda")
    enc.encode_bwd(xd, torch.from_numpy(dout).cuda(), grad)
    gref, gden = O.simplex_encode_bwd(x, dout, n_levels=L, log2_T=log2_T, n_features=F, base_res=base,
                                      growth=growth, res_mode=eq, with_denominator=True)
    g = grad.cpu().numpy()
    for l in range(L):
        e = record_error("encode_bwd table gradient (simplex, equal_mem)", rel_err(g[l], gref[l], gden[l]), 1e-5,
                         "sum_k |w_k dout| per entry")
        assert e <= 1e-5, "level %d" % l
        assert np.all(g[l][gden[l] == 0] == 0)
    if log2_T <= 19:
        dx = enc.encode_bwd_input(xd, t, torch.from_numpy(dout).cuda()).cpu().numpy()
        dref, dden = O.simplex_encode_dx(x, vals, dout, base_res=base, growth=growth, res_mode=eq,
                                         with_denominator=True)
        record_error("encode_bwd_input dL/dx (simplex, equal_mem)", np.max(np.abs(dx - dref) / (dden + 1e-30)), 1e-5,
                     "sum of |terms| of each dL/dx_i")
        assert np.all(np.abs(dx - dref) <= 1e-5 * dden + 1e-30)


def test_equal_mem_full_size_sdf_workload(cuda_lib):
    """The SDF-style configuration at full size (d = 3, L = 16, T = 2^19 bf16, 2^20 points, half near
    a union of spheres and tori) in the equal-memory setting: every output, and every table-gradient
    entry of all 16 levels, against the oracle."""
    from paper_2311_15439_gb300.api import Encoder
    eq = lattice.RES_EQUAL_MEM
    enc = Encoder(3, 16, 2, 19, 16.0, 1.38, res_mode="equal_mem", table_dtype="bf16", out_dtype="bf16")
    vals, bits = synth.uniform_tables(16, 1 << 19, 2, 73, dtype="bf16", scale=1e-4)
    t = torch.from_numpy(bits.astype(np.int16)).cuda().view(torch.bfloat16)
    x = synth.sdf_points(1 << 20, 74)
    xd = torch.from_numpy(x).cuda()
    out = enc.encode_fwd(xd, t).float().cpu().numpy()
    ref, den = O.simplex_encode(x, vals, base_res=16.0, growth=1.38, res_mode=eq, with_denominator=True)
    r = worst_ratio(out, ref, den, ENC_TOL["bf16"], ENC_ATOL["bf16"])
    record_error("encode_fwd bf16 output, SDF workload at full size (equal_mem)", r * ENC_TOL["bf16"],
                 ENC_TOL["bf16"], "sum_k |w_k H_k| (+ fp16 subnormal spacing)")
    assert r <= 1.0
    dout = synth.normal_grads(len(x), 32, 75)
    grad = torch.zeros((16, 1 << 19, 2), dtype=torch.float32, device="cuda")
    enc.encode_bwd(xd, torch.from_numpy(dout).cuda(), grad)
    g = grad.cpu().numpy()
    for l in range(16):
        gref, gden = O.simplex_encode_bwd(x, dout, n_levels=16, log2_T=19, n_features=2, base_res=16.0,
                                          growth=1.38, res_mode=eq, levels=[l], with_denominator=True)
        e = rel_err(g[l], gref[l], gden[l])
        record_error("encode_bwd table gradient, SDF workload at full size (equal_mem)", e, 1e-5, "sum_k |w_k dout| per entry")
        assert e <= 1e-5, "level %d" % l


def test_full_size_volumetric_encoding(cuda_lib):
    """The volumetric configuration at full size, in the benchmark's launch: 2^16 rays x 1024
    midpoint samples = 2^26 points (generated on the host by the oracle's binary32 sampler), d = 3,
    L = 16, T = 2^19 fp16 tables.  The fp16 encoding of 20 000 sampled points against the oracle;
    the backward of all 2^26 points through adjointness, <enc(H), D> = <H, bwd(D)>, a property that
    holds at any size, with both sides from the library (encoding in binary32 for this check)."""
    from paper_2311_15439_gb300.api import Encoder
    R, S, L = 1 << 16, 1024, 16
    rays = synth.camera_rays(R, 60)
    x, _ = OR.ray_samples_fp32(*rays, S)
    P = x.shape[0]
    assert P == 1 << 26
    vals, store = synth.uniform_tables(L, 1 << 19, 2, 61, dtype="f16", scale=1.0)
    t = torch.from_numpy(store).cuda()
    xd = torch.from_numpy(x).cuda()
    enc = Encoder(3, L, 2, 19, 16.0, 1.38, table_dtype="f16", out_dtype="f16")
    out = enc.encode_fwd(xd, t)
    idx = np.sort(synth.rng(62).choice(P, 20000, replace=False))
    got = out[torch.from_numpy(idx).cuda()].float().cpu().numpy()
    del out
    ref, den = O.simplex_encode(x[idx], vals, base_res=16.0, growth=1.38, with_denominator=True)
    r = worst_ratio(got, ref, den, ENC_TOL["f16"], ENC_ATOL["f16"])
    record_error("encode_fwd f16 output, volumetric workload at full size (sampled)", r * ENC_TOL["f16"],
                 ENC_TOL["f16"], "sum_k |w_k H_k| (+ fp16 subnormal spacing)")
    assert r <= 1.0
    # adjointness over every point: binary32 encoding, N(0, 1) upstream gradients drawn on the device
    enc32 = Encoder(3, L, 2, 19, 16.0, 1.38, table_dtype="f16", out_dtype="f32")
    gen = torch.Generator(device="cuda").manual_seed(63)
    D = torch.randn((P, L * 2), device="cuda", generator=gen)
    lhs = float(torch.sum(enc32.encode_fwd(xd, t).double() * D.double()))
    G = torch.zeros((L, 1 << 19, 2), dtype=torch.float32, device="cuda")
    enc32.encode_bwd(xd, D, G)
    H = t.double()
    rhs = float(torch.sum(H * G.double()))
    Ga = torch.zeros_like(G)
    enc32.encode_bwd(xd, D.abs(), Ga)
    scale = float(torch.sum(H.abs() * Ga.double()))            # sum over all terms of |w H D|
    del D, G, Ga
    torch.cuda.empty_cache()
    e = abs(lhs - rhs) / scale
    record_error("encode fwd/bwd adjointness, volumetric workload at full size", e, 1e-5, "sum of |w H D| over all terms")
    assert e <= 1e-5, (lhs, rhs, scale)


@pytest.mark.parametrize("kind,d,tdt,odt,index_mode", [
    ("simplex", 2, "f16", "f16", "hash"), ("simplex", 3, "bf16", "bf16", "dense_coarse"),
    ("simplex", 5, "f32", "f32", "hash"), ("grid", 2, "f16", "f32", "hash"), ("grid", 4, "f32", "f16", "dense_coarse")])
def test_forward_orders_agree(cuda_lib, kind, d, tdt, odt, index_mode):
    """The forward in point-major and in level-major work-item order (sxe_encoder_set_fwd_order)
    gives the same encoding bit for bit and marks the same bitmap, on a ragged number of points
    (a partial last block in every level); the level-major encoding also matches the oracle."""
    from paper_2311_15439_gb300.api import Encoder
    from oracle.lattice import INDEX_DENSE_COARSE, INDEX_HASH
    L, F, log2_T, base, growth = 7, 2, 13, 6.0, 1.6
    T = 1 << log2_T
    enc = Encoder(d, L, F, log2_T, base, growth, kind=kind, table_dtype=tdt, out_dtype=odt, index_mode=index_mode)
    P = 3 * 256 + 77
    x = synth.uniform_points(P, d, 131)
    vals = synth.uniform_tables(L, T, F, 132, dtype="f32", scale=1.0)[0]
    tab = torch.from_numpy(vals).to(torch_dtype_of(tdt)).cuda()
    xd = torch.from_numpy(x).cuda()
    outs, bms = {}, {}
    for order in ("point", "level", "auto"):
        enc.set_fwd_order(order)
        bm = torch.zeros(((L * T + 31) // 32,), dtype=torch.int32, device="cuda")
        outs[order] = enc.encode_fwd(xd, tab, touched=bm)
        bms[order] = bm
    assert torch.equal(outs["point"], outs["level"]) and torch.equal(outs["point"], outs["auto"])
    assert torch.equal(bms["point"], bms["level"]) and torch.equal(bms["point"], bms["auto"])
    H = tab.double().cpu().numpy()
    mode = INDEX_DENSE_COARSE if index_mode == "dense_coarse" else INDEX_HASH
    if kind == "simplex":
        ref = O.simplex_encode(x, H, base_res=base, growth=growth, index_mode=mode)
    else:
        ref = O.grid_encode(x, H, base_res=base, growth=growth, index_mode=mode)
    got = outs["level"].double().cpu().numpy()
    ulp = {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}[odt]
    assert np.all(np.abs(got - ref) <= (2 * ulp + 1e-5) * np.maximum(np.abs(ref), 1.0))


def torch_dtype_of(name):
    return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[name]
