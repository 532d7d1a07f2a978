"""C ABI: the library builds, loads without a GPU, exports every declared symbol, and its
host-side logic (argument validation, level constants) is right.  No device calls."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import lattice


@pytest.fixture(scope="module")
def L():
    from paper_2311_15439_gb300 import build, _lib
    build.build()
    return _lib


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "simplexenc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sxe_[a-z0-9_]+)\s*\(", src)))


def test_header_lists_every_binding(L):
    assert sorted(L.EXPORTS) == _declared_functions()


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert b"sm_103a" in lib.sxe_version()


def test_library_exports_nothing_undeclared(L):
    """The product library's dynamic symbols are exactly the header's entry points (the
    bench-only random-access probe lives in its own library, beside the benchmark)."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("sxe_")})
    assert exported == _declared_functions()
    assert "sxe_probe_random_access" not in exported


def _desc(L, **kw):
    base = dict(d=2, n_levels=8, n_features=2, log2_T=14, base_res=16.0, growth=1.5, kind=L.SXE_SIMPLEX,
                res_mode=L.SXE_RES_RAW, table_dtype=L.SXE_F32, out_dtype=L.SXE_F32)
    base.update(kw)
    return L.EncodingDesc(**base)


def _create(L, **kw):
    h = ctypes.c_void_p()
    st = L.lib().sxe_encoder_create(ctypes.byref(_desc(L, **kw)), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("bad,status", [
    (dict(d=7), -2), (dict(d=0), -1), (dict(n_levels=0), -1), (dict(n_levels=33), -1),
    (dict(n_features=3), -1), (dict(log2_T=3), -1), (dict(log2_T=27), -1), (dict(base_res=0.5), -1),
    (dict(growth=0.9), -1), (dict(kind=5), -1), (dict(res_mode=2), -1), (dict(table_dtype=9), -1),
    (dict(kind=1, res_mode=1), -1), (dict(base_res=float("nan")), -1), (dict(index_mode=2), -1),
])
def test_encoder_create_rejects_bad_descriptions(L, bad, status):
    st, h = _create(L, **bad)
    assert st == status
    assert L.lib().sxe_last_error()


def test_server_entry_points_validate_on_the_host(L):
    import ctypes
    lib = L.lib()
    h = ctypes.c_void_p()
    assert lib.sxe_server_create(None, ctypes.byref(h)) == -1
    for arena, nbytes, slots, maxb, prio in ((None, 1 << 20, 2, 100, 0), (4096 + 16, 1 << 20, 2, 100, 0),
                                             (4096, 0, 2, 100, 0), (4096, 1 << 20, 0, 100, 0),
                                             (4096, 1 << 20, 17, 100, 0), (4096, 1 << 20, 2, 0, 0),
                                             (4096, 1 << 20, 2, 100, -1)):
        desc = L.ServerDesc(arena, nbytes, slots, maxb, prio)
        assert lib.sxe_server_create(ctypes.byref(desc), ctypes.byref(h)) == -1
    rid, st = ctypes.c_int64(0), ctypes.c_int32(0)
    assert lib.sxe_server_add_field(None, None, None, None, None) == -1
    assert lib.sxe_server_start(None) == -1
    assert lib.sxe_server_submit(None, 2, None, 1, None, ctypes.byref(rid)) == -1
    assert lib.sxe_server_wait(None, 0, 0, ctypes.byref(st), None) == -1
    assert lib.sxe_server_stop(None, 1) == -1
    assert lib.sxe_server_destroy(None) == 0


def test_selftest_wait_checks_its_limit_on_the_host(L):
    lib = L.lib()
    assert lib.sxe_selftest_wait(1, 0, None) == -1
    assert lib.sxe_selftest_wait(1, -5, None) == -1
    assert lib.sxe_selftest_wait(0, 3_000_000_000, None) == -1


def test_entry_points_validate_before_launch(L):
    lib = L.lib()
    st, h = _create(L)
    assert st == 0
    try:
        # NULL encoder / negative sizes / NULL buffers are refused on the host
        assert lib.sxe_encode_fwd(None, 16, 10, 16, 16, None) == -1
        assert lib.sxe_encode_fwd(h, 16, -1, 16, 16, None) == -1
        assert lib.sxe_encode_fwd(h, None, 10, 16, 16, None) == -1
        assert lib.sxe_encode_fwd(h, 16, 10, None, 16, None) == -1
        assert lib.sxe_encode_fwd(h, 12, 10, 16, 16, None) == -1            # x misaligned for d = 2
        assert lib.sxe_encode_bwd(h, 16, 10, 16, 16, 3, None, None) == -1    # stride not a multiple of F
        assert lib.sxe_encode_bwd(h, 16, 10, 16, 20, 2, None, None) == -1    # grad entries misaligned
        # level ranges of the backward: inside [0, L] and not reversed; an empty range does nothing
        assert lib.sxe_encode_bwd_levels(h, 16, 10, 16, 16, 2, None, 3, 2, None) == -1
        assert lib.sxe_encode_bwd_levels(h, 16, 10, 16, 16, 2, None, -1, 2, None) == -1
        assert lib.sxe_encode_bwd_levels(h, 16, 10, 16, 16, 2, None, 0, 99, None) == -1
        assert lib.sxe_encode_bwd_levels(h, 16, 10, 16, 16, 2, None, 2, 2, None) == 0
        assert lib.sxe_encode_bwd_levels_kernel_count(h, 10, 2, 2) == 0
        assert lib.sxe_encode_bwd_levels_kernel_count(h, 10, 0, 99) == 0
        assert lib.sxe_encode_bwd_coarse_levels(None, 10) == 0
        assert lib.sxe_encode_bwd_coarse_levels(h, 0) == 0
        # backward strategy switch: 0 or 1 only
        assert lib.sxe_encoder_set_bwd_aggregation(None, 1) == -1
        assert lib.sxe_encoder_set_bwd_aggregation(h, 2) == -1
        assert lib.sxe_encoder_set_bwd_aggregation(h, 1) == 0
        assert lib.sxe_encoder_set_bwd_aggregation(h, 0) == 0
        # forward work-item order: 0 (automatic), 1 (point-major) or 2 (level-major)
        assert lib.sxe_encoder_set_fwd_order(None, 1) == -1
        assert lib.sxe_encoder_set_fwd_order(h, 3) == -1
        assert lib.sxe_encoder_set_fwd_order(h, -1) == -1
        for order in (2, 1, 0):
            assert lib.sxe_encoder_set_fwd_order(h, order) == 0
        # zero points: nothing to do, no pointer needed
        assert lib.sxe_encode_fwd(h, None, 0, None, None, None) == 0
        assert lib.sxe_encode_bwd(h, None, 0, None, None, 2, None, None) == 0
    finally:
        lib.sxe_encoder_destroy(h)
    m = L.MlpDesc(32, 64, 2, 3, L.SXE_F16)
    assert lib.sxe_mlp_n_params(ctypes.byref(m)) == 32 * 64 + 64 * 64 + 3 * 64
    assert lib.sxe_mlp_fwd(ctypes.byref(L.MlpDesc(32, 128, 2, 3, L.SXE_F16)), 16, 16, 8, 16, None, None) == -2
    assert lib.sxe_mlp_fwd(ctypes.byref(L.MlpDesc(32, 64, 2, 17, L.SXE_F16)), 16, 16, 8, 16, None, None) == -1
    assert lib.sxe_mlp_fwd(ctypes.byref(L.MlpDesc(32, 64, 2, 3, L.SXE_F32)), 16, 16, 8, 16, None, None) == -1
    assert lib.sxe_mlp_bwd(ctypes.byref(m), 16, 16, 16, ctypes.c_float(1.0), 8, None, 16, 16, 4, None) == -4  # workspace too small
    # one part of a batch: the batch must hold the part; an empty part without a squared-residual
    # sum enqueues nothing (with one it writes a zero there: a device write, covered on the GPU)
    part = lib.sxe_mlp_train_l2_part
    assert part(ctypes.byref(m), 16, 16, 16, ctypes.c_float(1.0), 8, 7, None, 16, 16, 16, 1 << 30, None) == -1
    assert part(ctypes.byref(m), 16, 16, None, ctypes.c_float(1.0), 8, 16, None, 16, 16, 16, 1 << 30, None) == -1
    assert part(ctypes.byref(m), 16, 16, 16, ctypes.c_float(1.0), 0, 0, None, 16, None, 16, 0, None) == 0
    assert lib.sxe_mlp_train_l2(ctypes.byref(m), None, None, None, ctypes.c_float(1.0), 0, None, None, None, None, 0,
                                None) == 0
    assert part(ctypes.byref(m), 16, 16, 16, ctypes.c_float(1.0), 8, 16, None, 16, 16, 16, 4, None) == -4
    a = L.AdamDesc(1e-2, 0.9, 0.99, 1e-15, 0)
    assert lib.sxe_step(ctypes.byref(a), 0, 4, 16, 16, 16, 16, None, 0, None) == -1                         # t = 0
    assert lib.sxe_step(ctypes.byref(L.AdamDesc(1e-2, 1.0, 0.99, 1e-15, 0)), 1, 4, 16, 16, 16, 16, None, 0, None) == -1


@pytest.mark.parametrize("kind", ["simplex", "grid"])
@pytest.mark.parametrize("cfg", [(2, 8, 16.0, 1.5), (2, 16, 16.0, 2.0), (3, 16, 16.0, 1.38), (4, 16, 16.0, 1.38),
                                 (5, 12, 8.0, 1.6)])
def test_level_constants_match_oracle(L, kind, cfg):
    """The library's binary32 level multipliers and resolutions equal the oracle's bit for bit."""
    d, nl, base, growth = cfg
    for res_mode in ([0, 1] if kind == "simplex" else [0]):
        st, h = _create(L, d=d, n_levels=nl, base_res=base, growth=growth,
                        kind=L.SXE_SIMPLEX if kind == "simplex" else L.SXE_GRID, res_mode=res_mode)
        assert st == 0
        s = np.zeros(nl, np.float32)
        r = np.zeros(nl, np.int32)
        assert L.lib().sxe_encoder_level_params(h, s.ctypes.data, r.ctypes.data) == 0
        L.lib().sxe_encoder_destroy(h)
        assert r.tolist() == lattice.level_resolutions(nl, base, growth)
        if kind == "simplex":
            want = lattice.simplex_level_scales_fp32(d, nl, base, growth, res_mode)
        else:
            want = lattice.grid_level_scales_fp32(nl, base, growth)
        assert np.array_equal(s.view(np.uint32), want.view(np.uint32))
        for index_mode in (L.SXE_INDEX_HASH, L.SXE_INDEX_DENSE_COARSE):
            for log2_T in (12, 19, 22):
                st, h = _create(L, d=d, n_levels=nl, base_res=base, growth=growth, log2_T=log2_T,
                                kind=L.SXE_SIMPLEX if kind == "simplex" else L.SXE_GRID, res_mode=res_mode,
                                index_mode=index_mode)
                assert st == 0
                w = np.zeros(nl, np.int32)
                assert L.lib().sxe_encoder_level_index(h, w.ctypes.data) == 0
                L.lib().sxe_encoder_destroy(h)
                assert w.tolist() == lattice.level_box_widths(kind, d, want, log2_T, index_mode)


def test_product_path_refuses_to_run_without_library(tmp_path):
    """The binding raises (no CPU fallback) when the shared library is missing."""
    from paper_2311_15439_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            _lib.lib(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def test_render_entries_validate_before_launch(L):
    """Argument errors of the rendering entries are caught on the host (no GPU needed)."""
    lib = L.lib()
    assert lib.sxe_vr_samples(16, 16, 16, 16, 4, 0, 16, 16, None) == L.SXE_EINVAL          # S = 0
    assert lib.sxe_vr_samples(16, 16, 16, 16, -1, 4, 16, 16, None) == L.SXE_EINVAL         # R < 0
    assert lib.sxe_vr_field(16, 16, 4, 8, L.SXE_F32, 16, 16, None) == L.SXE_EINVAL        # f32 colour input
    assert lib.sxe_vr_field(8, 16, 4, 8, L.SXE_F16, 16, 16, None) == L.SXE_EINVAL         # misaligned rows
    assert lib.sxe_vr_composite(None, 16, 16, 4, 8, 16, None, None, None) == L.SXE_EINVAL
    assert lib.sxe_vr_composite(16, 16, 16, 0, 8, 16, None, None, None) == L.SXE_OK       # no rays: nothing
    assert lib.sxe_encode_bwd_input(None, 16, 4, 16, 16, 16, None) == L.SXE_EINVAL         # NULL encoder
    # the fused field: the saved form needs both intermediate buffers, 16-byte aligned
    import ctypes
    dd, dc = L.MlpDesc(32, 64, 1, 16, L.SXE_F16), L.MlpDesc(32, 64, 2, 3, L.SXE_F16)
    args = (ctypes.byref(dd), 16, ctypes.byref(dc), 16, 16, 16, 4, 8, 16, 16)
    assert lib.sxe_vr_field_mlp_saved(*args, None, 16, None) == L.SXE_EINVAL              # no density_out
    assert lib.sxe_vr_field_mlp_saved(*args, 16, None, None) == L.SXE_EINVAL              # no color_in
    assert lib.sxe_vr_field_mlp_saved(*args, 8, 16, None) == L.SXE_EINVAL                 # misaligned
    assert lib.sxe_vr_field_mlp_saved(*args[:6], 0, 8, 16, 16, None, None, None) == L.SXE_OK   # no rays
    bad = L.MlpDesc(32, 64, 2, 16, L.SXE_F16)                                               # 2 hidden layers
    assert lib.sxe_vr_field_mlp_saved(ctypes.byref(bad), *args[1:], 16, 16, None) == L.SXE_EUNSUPPORTED
