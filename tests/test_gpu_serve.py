"""Serving loop: answers equal the kernels' answers alone and in the mix, memory admission
holds, bad requests fail alone, and values match the oracle."""
import numpy as np
import pytest
import torch

from oracle import encoding as OE
from oracle import mlp as OM
from paper_2311_15439_gb300 import synth

pytestmark = pytest.mark.gpu


def _fields(log2_T=14):
    from paper_2311_15439_gb300.serve import make_field
    return {d: make_field(d, log2_T=log2_T, seed=10 + d) for d in (2, 3, 4, 5)}


@pytest.fixture(params=["python", "native"])
def server_cls(request):
    """The scheduler in Python (``FieldServer``) and in the library (``NativeFieldServer``)."""
    from paper_2311_15439_gb300.serve import FieldServer, NativeFieldServer
    return {"python": FieldServer, "native": NativeFieldServer}[request.param]


def _alone(f, x, server_cls=None):
    """The request computed by itself: the encoding, then the network's forward pass on the
    kernel the server's loop takes (the library's loop: mma.sync under the automatic choice)."""
    from paper_2311_15439_gb300 import _lib as L
    from paper_2311_15439_gb300.serve import NativeFieldServer
    enc = f.encoder.encode_fwd(x.cuda(), f.tables)
    if server_cls is not NativeFieldServer or L.lib().sxe_mlp_get_kernel() != L.SXE_MLP_KERNEL_AUTO:
        return f.mlp.mlp_fwd(f.weights, enc).cpu()
    assert L.lib().sxe_mlp_set_kernel(L.SXE_MLP_KERNEL_MMA_SYNC) == 0
    try:
        return f.mlp.mlp_fwd(f.weights, enc).cpu()
    finally:
        L.lib().sxe_mlp_set_kernel(L.SXE_MLP_KERNEL_AUTO)


def test_alone_equals_mixed(cuda_lib, server_cls):
    """Each request's values are bitwise the same when merged with others (continuous batching
    over 4 stream slots) as when computed alone."""
    _alone_equals_mixed(server_cls, server_cls)


@pytest.mark.parametrize("priority_points", [0, 1 << 12])
def test_native_size_classes_alone_equal_mixed(cuda_lib, priority_points):
    """The library's loop with one size class (priority_points 0: every batch at normal priority)
    and with a small class of at most 4096 points: merged values equal those computed alone."""
    import functools
    from paper_2311_15439_gb300.serve import NativeFieldServer
    _alone_equals_mixed(functools.partial(NativeFieldServer, priority_points=priority_points), NativeFieldServer)


def test_native_server_on_the_tcgen05_forward(cuda_lib):
    """Under SXE_MLP_KERNEL_TCGEN05_3TILE the library's loop runs its network forward on the
    three-tile tcgen05 kernel: merged values equal that kernel's values alone."""
    from paper_2311_15439_gb300 import _lib as L
    from paper_2311_15439_gb300.serve import NativeFieldServer
    prev = L.lib().sxe_mlp_get_kernel()
    assert L.lib().sxe_mlp_set_kernel(L.SXE_MLP_KERNEL_TCGEN05_3TILE) == 0
    try:
        _alone_equals_mixed(NativeFieldServer, NativeFieldServer)
    finally:
        L.lib().sxe_mlp_set_kernel(prev)


def _alone_equals_mixed(make_server, server_cls):
    fields = _fields()
    g = synth.rng(1)
    reqs_in = []
    for i in range(40):
        d = int(g.choice([2, 3, 4, 5]))
        P = int(np.exp(g.uniform(np.log(100), np.log(70000))))
        reqs_in.append((d, torch.from_numpy(synth.uniform_points(P, d, 100 + i)).pin_memory()))
    srv = make_server(fields, mem_budget_bytes=64 << 20, n_slots=4, max_batch_points=1 << 18).start()
    reqs = [srv.submit(d, x) for d, x in reqs_in]
    for r in reqs:
        assert r.wait(60)
    srv.stop()
    assert srv.n_batches < len(reqs)                     # requests were merged
    for (d, x), r in zip(reqs_in, reqs):
        assert r.error is None
        assert torch.equal(r.y, _alone(fields[d], x, server_cls))


def test_memory_admission_and_rejections(cuda_lib, server_cls):
    """With a budget that fits about one request, requests wait instead of overcommitting;
    malformed, unknown-dimension and oversize requests fail without disturbing the rest."""
    fields = _fields()
    budget = 40000 * fields[2].bytes_per_point() + 1024
    srv = server_cls(fields, mem_budget_bytes=budget, n_slots=3, max_batch_points=1 << 16).start()
    good = [(2, torch.from_numpy(synth.uniform_points(30000, 2, i)).pin_memory()) for i in range(6)]
    bad = [(7, torch.zeros((10, 7)).pin_memory()),                      # no field of that dimension
           (3, torch.zeros((10, 2)).pin_memory()),                      # wrong width
           (2, torch.from_numpy(synth.uniform_points(100000, 2, 9)).pin_memory())]   # over the budget
    reqs = []
    for i, (d, x) in enumerate(good):
        reqs.append(srv.submit(d, x))
        if i < len(bad):
            reqs.append(srv.submit(*bad[i]))
    for r in reqs:
        assert r.wait(60)
    srv.stop()
    assert srv.peak_used <= budget
    errs = [r for r in reqs if r.error is not None]
    assert len(errs) == len(bad)
    for r in reqs:
        if r.error is None:
            assert torch.equal(r.y, _alone(fields[r.d], r.x, server_cls))


@pytest.mark.parametrize("d", [2, 5])
def test_served_values_match_oracle(cuda_lib, d, server_cls):
    """Served values equal the FP64 oracle's encoding + network on the same fp16 tables and
    weights (encoding rounded to fp16 as the network reads it), within the network bound."""
    from test_gpu_mlp import _dens
    f = _fields()[d]
    x = synth.uniform_points(5000, d, 3)
    srv = server_cls({d: f}, mem_budget_bytes=64 << 20).start()
    r = srv.submit(d, torch.from_numpy(x).pin_memory())
    assert r.wait(60)
    srv.stop()
    tables = f.tables.float().cpu().numpy()
    enc = OE.simplex_encode(x, tables, base_res=16.0, growth=1.38)
    enc16 = enc.astype(np.float16).astype(np.float64)
    Ws = [w.astype(np.float64) for w in f.mlp.split(f.weights.float().cpu().numpy())]
    y, _ = OM.mlp_forward(Ws, enc16)
    yden, _, _ = _dens(Ws, enc16, np.zeros_like(y))
    tol = 6 * 2.0 ** -11
    # forward only: a ReLU decision flipped by rounding changes a value by no more than the
    # rounding itself, so the forward bound needs no slack
    err = np.abs(r.y.numpy().astype(np.float64) - y)
    assert np.all(err <= tol * yden)


def test_native_server_stops_without_draining_and_reports_failures(cuda_lib):
    """Stopping the native server without draining fails what is still queued (each request
    completes, with an error) while batches already launched finish with their values (200
    one-batch requests, one slot: the stop lands long before the queue drains); a server refuses
    submissions once stopped."""
    from paper_2311_15439_gb300.serve import NativeFieldServer
    fields = _fields()
    srv = NativeFieldServer(fields, mem_budget_bytes=8 << 20, n_slots=1, max_batch_points=1 << 16).start()
    xs = [torch.from_numpy(synth.uniform_points(1 << 16, 3, 500 + i)).pin_memory() for i in range(200)]
    reqs = [srv.submit(3, x) for x in xs]        # one request per batch, one batch in flight
    assert reqs[0].wait(60)
    srv.stop(drain=False)
    for r in reqs:
        assert r.wait(60)
    done = [r for r in reqs if r.error is None]
    failed = [r for r in reqs if r.error is not None]
    assert done[0] is reqs[0] and all(torch.equal(r.y, _alone(fields[3], r.x, NativeFieldServer)) for r in done)
    assert failed and all("stopped" in r.error for r in failed)
    assert all(r.rid > q.rid for r in failed for q in done)     # the queue's tail failed, in order
    late = srv.submit(3, xs[0])
    assert late.wait(1) and late.error is not None


def test_native_server_takes_requests_from_several_threads(cuda_lib):
    """Four client threads submit and wait concurrently (submit and wait are thread-safe in the
    library); every answer equals the request computed alone, and sizes above the batch limit are
    refused with an error request."""
    import threading
    from paper_2311_15439_gb300.serve import NativeFieldServer
    fields = _fields()
    srv = NativeFieldServer(fields, mem_budget_bytes=64 << 20, n_slots=4, max_batch_points=1 << 17,
                            priority_points=1 << 12).start()
    results, errors = {}, []

    def client(k):
        try:
            g = synth.rng(200 + k)
            mine = []
            for i in range(30):
                d = int(g.choice([2, 3, 4, 5]))
                P = int(np.exp(g.uniform(np.log(50), np.log(1 << 17))))
                x = torch.from_numpy(synth.uniform_points(P, d, 1000 * k + i)).pin_memory()
                mine.append((d, x, srv.submit(d, x)))
            for d, x, r in mine:
                assert r.wait(60) and r.error is None
                results[(k, r.rid)] = (d, x, r.y)
        except Exception as exc:         # surfaced in the main thread
            errors.append(exc)

    threads = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(120)
    big = srv.submit(2, torch.zeros((1 << 17) + 1, 2).pin_memory())
    srv.stop()
    assert not errors, errors[0]
    assert len(results) == 120
    for d, x, y in results.values():
        assert torch.equal(y, _alone(fields[d], x, NativeFieldServer))
    assert big.wait(1) and big.error is not None


def test_native_server_concurrent_stops_and_restart(cuda_lib):
    """Two threads stop a draining server at once: both calls return, every queued request has
    run; the server then starts again and answers as before."""
    import threading
    from paper_2311_15439_gb300.serve import NativeFieldServer
    fields = _fields()
    srv = NativeFieldServer(fields, mem_budget_bytes=16 << 20, n_slots=2, max_batch_points=1 << 16).start()
    xs = [torch.from_numpy(synth.uniform_points(20000, 3, 300 + i)).pin_memory() for i in range(40)]
    reqs = [srv.submit(3, x) for x in xs]
    errors = []

    def stopper():
        try:
            srv.stop(drain=True)
        except Exception as exc:         # surfaced in the main thread
            errors.append(exc)

    threads = [threading.Thread(target=stopper) for _ in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(60)
    assert not any(t.is_alive() for t in threads) and not errors, errors
    assert all(r.wait(1) and r.error is None for r in reqs)
    assert all(torch.equal(r.y, _alone(fields[3], x, NativeFieldServer)) for r, x in zip(reqs, xs))
    srv.start()
    again = srv.submit(2, xs[0][:, :2].contiguous().pin_memory())
    assert again.wait(60) and again.error is None
    srv.stop()
    assert torch.equal(again.y, _alone(fields[2], xs[0][:, :2].contiguous(), NativeFieldServer))
