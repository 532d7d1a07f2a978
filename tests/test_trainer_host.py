"""Host-side logic of the training step (CPU only): level ranges of the overlapped table step,
the table-layout rule and the loss scale."""
import math
import types

import pytest
import torch

pytest.importorskip("paper_2311_15439_gb300._lib")


def _encoder(**kw):
    from paper_2311_15439_gb300 import _lib as L
    try:
        L.lib()
    except RuntimeError as e:                      # the library is built by __graft_entry__.build()
        pytest.skip(str(e))
    from paper_2311_15439_gb300.api import Encoder
    args = dict(d=2, n_levels=16, n_features=2, log2_T=22, base_res=16.0, growth=2.0, table_dtype="f16")
    args.update(kw)
    return Encoder(**args)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 16, 40])
def test_level_chunks_cover_the_levels_in_order(k):
    from paper_2311_15439_gb300.trainer import level_chunks
    enc = _encoder()
    chunks = level_chunks(enc, 1 << 18, k)
    assert 1 <= len(chunks) <= min(k, enc.n_levels)
    assert chunks[0][0] == 0 and chunks[-1][1] == enc.n_levels
    assert all(lb < le for lb, le in chunks)
    assert all(a[1] == b[0] for a, b in zip(chunks, chunks[1:]))
    if k == 1:
        assert chunks == [(0, enc.n_levels)]


def test_level_chunks_balance_the_touched_entries():
    """Each range's estimate min(T, box, V P) summed over its levels is close to the total / k: the
    coarse levels (small boxes) group together and the fine levels (capped at V P) split evenly."""
    from paper_2311_15439_gb300.trainer import level_chunks
    enc = _encoder()
    P, k = 1 << 18, 4
    est = [min(float(enc.T), (math.floor(16.0 * 2.0 ** l) + 2.0) ** 2, 3.0 * P) for l in range(16)]
    chunks = level_chunks(enc, P, k)
    assert len(chunks) == k
    sums = [sum(est[lb:le]) for lb, le in chunks]
    # no range exceeds the ideal share by more than one level's estimate
    assert max(sums) <= sum(est) / k + max(est)
    assert chunks[0][1] > 1                         # the small coarse levels share the first range


def _fake_l2(monkeypatch, l2_bytes):
    props = types.SimpleNamespace(L2_cache_size=l2_bytes)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: props)


def test_table_layout_rule(monkeypatch):
    from paper_2311_15439_gb300.trainer import DENSE_L2_FRACTION, choose_table_layout
    l2 = 126 << 20
    _fake_l2(monkeypatch, l2)
    image = _encoder()                                                # 16 x 2^22 x 2 x 4 B = 512 MiB
    sdf = _encoder(d=3, log2_T=19, growth=1.38, table_dtype="bf16")   # 64 MiB
    assert choose_table_layout(image, "cuda:0") == "records"
    assert choose_table_layout(sdf, "cuda:0") == "dense"
    for layout in ("records", "dense"):                               # an explicit choice is kept
        assert choose_table_layout(image, "cuda:0", layout) == layout
        assert choose_table_layout(sdf, "cuda:0", layout) == layout
    with pytest.raises(ValueError):
        choose_table_layout(sdf, "cuda:0", "sparse")
    # the threshold itself: a gradient array of DENSE_L2_FRACTION of L2 is dense; with an L2 a
    # little smaller it is not
    grad = 4 * sdf.n_levels * sdf.T * sdf.n_features
    _fake_l2(monkeypatch, int(math.ceil(grad / DENSE_L2_FRACTION)))
    assert choose_table_layout(sdf, "cuda:0") == "dense"
    _fake_l2(monkeypatch, int(grad / DENSE_L2_FRACTION) - 1024)
    assert choose_table_layout(sdf, "cuda:0") == "records"


@pytest.mark.parametrize("P,n_out", [(1, 1), (1, 3), (4096, 3), (1 << 18, 3), (1 << 20, 1), (1000, 7)])
def test_default_loss_scale(P, n_out):
    from paper_2311_15439_gb300.trainer import default_loss_scale
    s = default_loss_scale(P, n_out)
    assert s >= 1.0 and math.log2(s) == int(math.log2(s))            # a power of two (exact in binary32)
    target = max(1.0, P * n_out / 2.0)
    assert target / 2.0 < s <= target                                # the largest power of two <= P n_out / 2
