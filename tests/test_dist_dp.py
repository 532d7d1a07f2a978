"""Data-parallel training by points (``data_parallel``), its host orchestration on CPU: two gloo
ranks each compute the gradients of their shard of the batch with the FP64 oracle (encoding,
network + L2 loss, backward, scatter into the tables), the step averages them with one all-reduce
and applies Adam; after several steps both ranks hold identical parameters, equal to those of one
process that trained on the union of the points."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

L, LOG2_T, F, BASE, GROWTH = 4, 10, 2, 8.0, 1.5
SHAPES = [(64, L * F), (64, 64), (3, 64)]
P_UNION, STEPS = 600, 3
HP = dict(lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleReplica:
    """One rank's replica with the oracle doing the per-rank work: FP64 tables [L, T, F], network
    weights, Adam moments, and a flat float64 buffer [table gradient | network gradient | sq sum]."""

    def __init__(self):
        from paper_2311_15439_gb300 import synth
        T = 1 << LOG2_T
        self.H = synth.uniform_tables(L, T, F, 3, dtype="f32", scale=1e-1)[0].astype(np.float64)
        g = np.random.Generator(np.random.PCG64(4))
        self.W = [g.uniform(-np.sqrt(6 / fi), np.sqrt(6 / fi), size=(fo, fi)) for fo, fi in SHAPES]
        self.mH, self.vH = np.zeros_like(self.H), np.zeros_like(self.H)
        self.mW = [np.zeros_like(w) for w in self.W]
        self.vW = [np.zeros_like(w) for w in self.W]
        self.n_tab = self.H.size
        self.n_w = sum(w.size for w in self.W)
        self.flat = torch.zeros(self.n_tab + self.n_w + 1, dtype=torch.float64)
        self.t = 0

    def local(self, x, tgt):
        from oracle import encoding as OE
        from oracle import mlp as OM
        e = OE.simplex_encode(x, self.H, base_res=BASE, growth=GROWTH)
        y, acts = OM.mlp_forward(self.W, e)
        loss, dy = OM.l2_loss(y, tgt)
        dW, de = OM.mlp_backward(self.W, acts, dy)
        g = OE.simplex_encode_bwd(x, de, n_levels=L, log2_T=LOG2_T, n_features=F, base_res=BASE, growth=GROWTH)
        f = self.flat.numpy()
        f[:self.n_tab] += np.stack([g[l] for l in range(L)]).ravel()
        f[self.n_tab:self.n_tab + self.n_w] += np.concatenate([w.ravel() for w in dW])
        f[-1] = loss * y.size                           # the batch's sum of squared residuals

    def apply(self):
        from oracle import adam as OA
        self.t += 1
        f = self.flat.numpy()
        gH = f[:self.n_tab].reshape(self.H.shape)
        self.H, self.mH, self.vH = OA.adam_step(self.H, gH, self.mH, self.vH, self.t, skip_zero_grad=True, **HP)
        o = self.n_tab
        for i, w in enumerate(self.W):
            gw = f[o:o + w.size].reshape(w.shape)
            self.W[i], self.mW[i], self.vW[i] = OA.adam_step(w, gw, self.mW[i], self.vW[i], self.t,
                                                             skip_zero_grad=False, **HP)
            o += w.size
        f[:-1] = 0.0


def _batches():
    from paper_2311_15439_gb300 import synth
    img = synth.ProceduralImage(8, size=1024, n_waves=8)
    out = []
    for k in range(STEPS):
        x = synth.uniform_points(P_UNION, 2, 70 + k)
        out.append((x, img.sample(x).astype(np.float64)))
    return out


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2311_15439_gb300.data_parallel import DataParallelStep, shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rep = OracleReplica()
        dp = DataParallelStep(rep.flat, rep.local, rep.apply)
        losses = []
        for x, t in _batches():
            s = shard(len(x), rank, world)
            dp.step(x[s], t[s])
            losses.append(float(rep.flat[-1]) / (len(x[s]) * 3))
        q.put((rank, rep.H, [w.copy() for w in rep.W], losses))
    finally:
        dist.destroy_process_group()


def test_shard_covers_every_point_once():
    from paper_2311_15439_gb300.data_parallel import shard
    for n in (0, 1, 7, 600, 1001):
        for world in (1, 2, 3, 8):
            idx = np.concatenate([np.arange(n)[shard(n, r, world)] for r in range(world)])
            assert np.array_equal(idx, np.arange(n))
            sizes = [len(range(n)[shard(n, r, world)]) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def test_two_ranks_train_like_one_process_on_the_union():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, H0, W0, loss0), (_, H1, W1, loss1) = out
    # the replicas stay identical: the same averaged gradient, the same update
    assert np.array_equal(H0, H1) and all(np.array_equal(a, b) for a, b in zip(W0, W1))
    assert loss0 == loss1
    # one process on the union of the points (no exchange: world of one)
    from paper_2311_15439_gb300.data_parallel import DataParallelStep
    ref = OracleReplica()
    dp = DataParallelStep(ref.flat, ref.local, ref.apply)
    ref_losses = []
    for x, t in _batches():
        dp.step(x, t)
        ref_losses.append(float(ref.flat[-1]) / (len(x) * 3))
    assert ref.t == STEPS
    np.testing.assert_allclose(loss0, ref_losses, rtol=1e-12)
    moved = np.abs(ref.H - OracleReplica().H) > 0
    assert moved.sum() > 1000                         # the steps updated many table entries
    np.testing.assert_allclose(H0, ref.H, rtol=0, atol=1e-9)
    for a, b in zip(W0, ref.W):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-9)
