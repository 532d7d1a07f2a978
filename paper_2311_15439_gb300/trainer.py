"""Training step of the image-fitting and SDF-style workloads (Sec. 6.1 of arXiv 2311.15439).

One ``step(x, target)`` runs, on the caller's stream and entirely in libsimplexenc
kernels:

1. ``sxe_encode_fwd``   -- multiresolution encoding of the batch from the low-precision
                           tables (Sec. 5 a-d); optionally (``mark_touched_in_forward``, records
                           layout) ``sxe_encode_fwd_marked``, which also marks the touched entries
                           that the backward then leaves unmarked;
2. ``sxe_mlp_train_l2`` -- network forward, L2 loss, network backward, dL/d(encoding)
                           (Sec. 5 d-e);
3. ``sxe_encode_bwd``   -- scatter-add of dL/d(encoding) into the table gradients (Sec. 5 e):
                           the gradient field of the interleaved records, marking touched
                           entries, or the dense gradient array (see the layouts below);
4. ``sxe_step_touched`` -- Adam on the marked table entries, or ``sxe_step`` over the dense
                           arrays (both with the zero-gradient skip rule), refreshing the
                           low-precision tables;
5. ``sxe_step``         -- Adam on the network weights, refreshing their low-precision copy.

The step count lives on the device (``sxe_adam_advance`` increments it and writes the bias
corrections that both Adam launches read), so a step has no host-side value that changes from
one step to the next: ``capture`` records it once into a CUDA graph and ``replay`` reruns it
with a single launch.

Table state layout in HBM (``choose_table_layout``), for tables far larger than L2 of which a
step touches a small part: one binary32 record {param[F], m[F], v[F], grad[F]} per entry (32
bytes for F = 2: one DRAM sector), entries ordered [level][slot], and a bitmap of L*T bits that
marks the entries that received a gradient in the current step; for tables whose gradient array
fits in L2: separate dense binary32 arrays (the backward's reductions then stay in L2) and a dense
Adam that skips zero gradients.  Either way a separate dense [L][T][F] low-precision copy is what
the forward pass gathers from.
"""
from __future__ import annotations

import math

import torch

from . import synth
from .api import Adam, Encoder, Mlp, torch_dtype


def level_chunks(enc: Encoder, P: int, k: int) -> list[tuple[int, int]]:
    """Split the levels into at most k contiguous ranges that each hold about the same number of
    touched table entries, estimated per level as min(T, lattice box of [0,1]^d, vertices * P)."""
    m = (enc.d + 1.0) ** ((enc.d - 1.0) / (2.0 * enc.d)) if enc.res_mode == "equal_mem" else 1.0
    est = []
    for l in range(enc.n_levels):
        N = math.floor(enc.base_res * enc.growth ** l) * (m if enc.kind == "simplex" else 1.0)
        est.append(min(float(enc.T), (N + 2.0) ** enc.d, float(enc.n_vertices * P)))
    k = max(1, min(k, enc.n_levels))
    total, acc, out, lb = sum(est), 0.0, [], 0
    for l, e in enumerate(est):
        acc += e
        if len(out) < k - 1 and acc >= total * (len(out) + 1) / k and l + 1 < enc.n_levels:
            out.append((lb, l + 1))
            lb = l + 1
    out.append((lb, enc.n_levels))
    return out


DENSE_L2_FRACTION = 0.6


def choose_table_layout(encoder: Encoder, device, layout: str = "auto") -> str:
    """"records": one binary32 record {param, m, v, grad} per entry, a bitmap of the entries a step
    touched and an optimiser sweep over those only -- for tables far larger than L2 of which a
    step touches a small part.  "dense": separate binary32 arrays, the gradient a dense [L][T][F]
    array that the backward's reductions keep in L2, and a dense Adam that skips zero gradients
    (the same update) -- for tables whose gradient array fits in L2.  "auto" picks "dense" when
    the gradient array is at most DENSE_L2_FRACTION of the device's L2."""
    if layout in ("records", "dense"):
        return layout
    if layout != "auto":
        raise ValueError("table layout must be 'auto', 'records' or 'dense'")
    l2 = getattr(torch.cuda.get_device_properties(torch.device(device)), "L2_cache_size", 0) or (96 << 20)
    grad_bytes = 4 * encoder.n_levels * encoder.T * encoder.n_features
    return "dense" if grad_bytes <= DENSE_L2_FRACTION * l2 else "records"


class TableState:
    """Master table parameters, Adam moments and gradients in one of the two layouts of
    ``choose_table_layout``, with the low-precision copy the forward pass gathers from."""

    def __init__(self, encoder: Encoder, init: torch.Tensor, layout: str, device, split_coarse="auto"):
        F = encoder.n_features
        n_entries = encoder.n_levels * encoder.T
        self.enc, self.layout, self.device = encoder, layout, torch.device(device)
        self.split_coarse, self._side = False, None
        # records layout: mark the touched entries in the forward pass (``forward``) instead of the
        # backward; the owner turns it on when its step runs this state's forward and backward on
        # the same points
        self.mark_in_forward = False
        self.set_split_coarse(layout == "dense" if split_coarse == "auto" else split_coarse)
        self.tables = init.to(torch_dtype(encoder.table_dtype)).reshape(encoder.table_shape()).contiguous()
        if layout == "records":
            self.state = torch.zeros((n_entries, 4 * F), dtype=torch.float32, device=device)
            self.state[:, :F] = init
            self.touched = torch.zeros(((n_entries + 31) // 32,), dtype=torch.int32, device=device)
        else:
            self.state = self.touched = None
            self.param = init.reshape(-1).clone()
            self.m = torch.zeros_like(self.param)
            self.v = torch.zeros_like(self.param)
            self.grad = torch.zeros_like(self.param)

    def set_split_coarse(self, on: bool) -> None:
        """Run the levels that the backward sums per block in shared memory
        (``Encoder.bwd_coarse_levels``) on a second, high-priority stream while the other levels
        run on the caller's stream.  In one stream the coarse levels' few long blocks run alone
        before the direct-path kernel fills the GPU; the two level ranges share no gradient
        address or bitmap word, so the result is the same sum.  "auto" (the constructor's default)
        turns it on for the dense layout, whose reductions hit L2 (SDF-style step 0.805 -> 0.779 ms,
        volumetric 3.86 -> 3.71 ms on GB300), and off for the records layout, whose direct-path
        reductions miss L2 and slowed down beside the coarse blocks (image step 0.667 -> 0.742 ms)."""
        self.split_coarse = bool(on)
        if self.split_coarse and self._side is None:
            self._side = torch.cuda.Stream(device=self.device, priority=-1)
            self._fork, self._join = torch.cuda.Event(), torch.cuda.Event()

    def forward(self, x, out, stream=None) -> None:
        """The encoding of x from the low-precision tables into out; with the records layout and
        ``mark_in_forward`` it also sets the touched bits of every entry it reads
        (``sxe_encode_fwd_marked``), exactly the entries the backward of the same points adds to,
        so that the backward's reductions run without the bitmap's reads and ORs."""
        mark = self.touched if (self.layout == "records" and self.mark_in_forward) else None
        self.enc.encode_fwd(x, self.tables, out, stream=stream, touched=mark)

    def backward(self, x, d_enc, stream=None, levels=None) -> None:
        """Table gradients of one step (into the records' gradient fields or the dense array)."""
        if levels is None and self.split_coarse and self.enc.T >= 32:
            L = self.enc.n_levels
            lc = self.enc.bwd_coarse_levels(x.shape[0])
            if 0 < lc < L:
                main = torch.cuda.current_stream(self.device) if stream is None else stream
                self._fork.record(main)
                self._side.wait_event(self._fork)
                self._backward(x, d_enc, self._side, (0, lc))
                self._backward(x, d_enc, main, (lc, L))
                self._join.record(self._side)
                main.wait_event(self._join)
                return
        self._backward(x, d_enc, stream, levels)

    def _backward(self, x, d_enc, stream, levels) -> None:
        F = self.enc.n_features
        if self.layout == "records":
            self.enc.encode_bwd(x, d_enc, self.state, grad_stride=4 * F, grad_offset=3 * F,
                                touched=None if self.mark_in_forward else self.touched, levels=levels, stream=stream)
        else:
            self.enc.encode_bwd(x, d_enc, self.grad, levels=levels, stream=stream)

    def adam(self, adam: Adam, corrections, stream=None) -> None:
        """Adam on every entry with a nonzero gradient; refreshes the low-precision tables."""
        if self.layout == "records":
            adam.step_touched_dev(corrections, self.state, self.touched, self.tables, self.enc.n_features,
                                  stream=stream)
        else:
            adam.step_dev(corrections, self.param, self.m, self.v, self.grad, lowp=self.tables.view(-1),
                          stream=stream)

    def params(self) -> torch.Tensor:
        F = self.enc.n_features
        p = self.state[:, :F] if self.layout == "records" else self.param
        return p.reshape(self.enc.table_shape())

    def grads(self) -> torch.Tensor:
        """The gradient accumulated since the last Adam step, [L, T, F]."""
        F = self.enc.n_features
        g = self.state[:, 3 * F:] if self.layout == "records" else self.grad
        return g.reshape(self.enc.table_shape())


def default_loss_scale(P: int, n_out: int) -> float:
    """Power of two near P*n_out/2 so that the scaled L2 gradient 2 r / (P n_out) is O(r)."""
    return float(2.0 ** max(0, math.floor(math.log2(max(1.0, P * n_out / 2.0)))))


class Trainer:
    def __init__(self, encoder: Encoder, mlp: Mlp, batch: int, *, seed: int = 0, device="cuda",
                 table_init: float = 1e-4, lr: float = 1e-2, betas=(0.9, 0.99), eps: float = 1e-15,
                 table_chunks: int = 1, table_layout: str = "auto", split_coarse="auto", split_batch: int = 1,
                 mark_touched_in_forward: bool = False):
        if mlp.n_in != encoder.n_out:
            raise ValueError("network input %d != encoding width %d" % (mlp.n_in, encoder.n_out))
        self.enc, self.mlp, self.P = encoder, mlp, batch
        self.device = torch.device(device)
        F = encoder.n_features
        n_entries = encoder.n_levels * encoder.T
        # seeded host values U(-table_init, table_init), so any checker can regenerate them
        vals = synth.uniform_tables(encoder.n_levels, encoder.T, F, seed, dtype="f32", scale=table_init)[0]
        init = torch.from_numpy(vals.reshape(n_entries, F)).to(self.device)
        self.tab = TableState(encoder, init, choose_table_layout(encoder, self.device, table_layout), self.device,
                              split_coarse=split_coarse)
        self.tables, self.state, self.touched = self.tab.tables, self.tab.state, self.tab.touched
        W0 = torch.from_numpy(mlp.init_weights(seed + 1)).to(self.device)
        self.W = W0.clone()
        self.W_lowp = W0.to(torch_dtype(mlp.dtype))
        self.mW = torch.zeros_like(W0)
        self.vW = torch.zeros_like(W0)
        self.dW = torch.zeros_like(W0)
        self.enc_out = torch.empty((batch, encoder.n_out), dtype=torch_dtype(encoder.out_dtype), device=self.device)
        self.d_enc = torch.empty((batch, encoder.n_out), dtype=torch.float32, device=self.device)
        # the batch's sum of squared residuals, one entry per part of a split step (sq_sum: the first)
        self.split = max(1, int(split_batch))
        self.sq_parts = torch.zeros((self.split,), dtype=torch.float32, device=self.device)
        self.sq_sum = self.sq_parts[:1]
        self.stage_events = None
        self.stage_only = None            # a set of stage names: mark only those stages
        self.ws = mlp.workspace(batch, self.device)
        self.loss_scale = default_loss_scale(batch, mlp.n_out)
        self.adam_tables = Adam(lr, betas[0], betas[1], eps, skip_zero_grad=True)
        self.adam_mlp = Adam(lr, betas[0], betas[1], eps, skip_zero_grad=False)
        self.t = 0
        self.t_dev = torch.zeros((1,), dtype=torch.int64, device=self.device)
        self.corrections = torch.zeros((2,), dtype=torch.float32, device=self.device)
        self.graph = None
        self.mark_touched_in_forward = bool(mark_touched_in_forward)
        self.set_table_chunks(table_chunks)
        if self.split > 1:
            if len(self.chunks) > 1:
                raise ValueError("split_batch and table_chunks > 1 cannot be combined")
            self._bwd_stream = torch.cuda.Stream(device=self.device)
            self._part_ready = [torch.cuda.Event() for _ in range(self.split)]
            self._bwd_done = torch.cuda.Event()

    def set_table_chunks(self, k: int) -> None:
        """Run the table backward and the table Adam in k level ranges: the Adam of range i runs on
        a second (high-priority) stream while the backward of range i+1 runs on the step's stream.
        Entries of different levels share no state record or bitmap word (T >= 32), so the ranges
        are independent; k = 1 is the plain two-pass step."""
        if k > 1 and (self.enc.T < 32 or self.tab.layout != "records"):
            k = 1
        self.chunks = level_chunks(self.enc, self.P, k)
        # the level-range step marks entries in its backward (per range); the plain step in the forward
        self.tab.mark_in_forward = len(self.chunks) == 1 and self.mark_touched_in_forward
        if len(self.chunks) > 1:
            self._aux = torch.cuda.Stream(device=self.device, priority=-1)
            self._ready = [torch.cuda.Event() for _ in self.chunks]
            self._joined = torch.cuda.Event()

    @property
    def n_launches_per_step(self) -> int:
        # the device step counter, encode_fwd, network training + its partial reduction, encode_bwd
        # per level range (coarse levels in shared memory, then the rest), table Adam per range,
        # network Adam
        if self.split > 1:
            bwd = sum(self.enc.bwd_kernel_count(b - a) for a, b in self.parts())
            return 4 + 2 * self.split + bwd
        bwd = sum(self.enc.bwd_kernel_count(self.P, levels=c) for c in self.chunks)
        return 5 + bwd + len(self.chunks)

    def parts(self):
        """Row ranges of the parts of a split step (the whole batch when it is not split)."""
        cut = [i * self.P // self.split for i in range(self.split + 1)]
        return [(cut[i], cut[i + 1]) for i in range(self.split)]

    def _mark(self, name, stream):
        """Record a timing event on `stream` when ``stage_events`` (a dict name -> list) is set (and
        the stage is in ``stage_only``, when that is set).  Inside a graph recording (``capture``)
        the event becomes one of the graph's nodes, so it records the time each replay of that graph
        reaches it."""
        stage = name[:-4] if name.endswith("_end") else name
        if self.stage_events is not None and (self.stage_only is None or stage in self.stage_only):
            if torch.cuda.is_current_stream_capturing():
                ev = torch.cuda.Event(enable_timing=True, external=True)
            else:
                ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            self.stage_events.setdefault(name, []).append(ev)

    def step(self, x: torch.Tensor, target: torch.Tensor, stream=None) -> None:
        """One optimisation step on batch (x [P, d] float32, target [P, n_out] float32); asynchronous."""
        if self.split > 1:
            self._step_split(x, target, stream)
            return
        self.t += 1
        main = torch.cuda.current_stream(self.device) if stream is None else stream
        self.adam_tables.advance(self.t_dev, self.corrections, stream=stream)
        self._mark("encode_fwd", main)
        self.tab.forward(x, self.enc_out, stream=stream)
        self._mark("encode_fwd_end", main)
        self._mark("mlp_train_l2", main)
        self.mlp.mlp_train_l2(self.W_lowp, self.enc_out, target, self.dW, self.sq_sum, din=self.d_enc,
                              loss_scale=self.loss_scale, workspace=self.ws, stream=stream)
        self._mark("mlp_train_l2_end", main)
        if len(self.chunks) == 1:
            self._mark("encode_bwd", main)
            self.tab.backward(x, self.d_enc, stream=stream)
            self._mark("encode_bwd_end", main)
            self._mark("adam_tables", main)
            self.tab.adam(self.adam_tables, self.corrections, stream=stream)
            self._mark("adam_tables_end", main)
        else:
            self._table_step_overlapped(x, stream)
        self.adam_mlp.step_dev(self.corrections, self.W, self.mW, self.vW, self.dW, lowp=self.W_lowp, stream=stream)
        self._mark("adam_mlp_end", main)
        if len(self.chunks) > 1:
            main = torch.cuda.current_stream(self.device) if stream is None else stream
            main.wait_event(self._joined)

    def _step_split(self, x, target, stream) -> None:
        """The step with the batch in ``split`` parts: the encoding forward of the whole batch, then
        per part the network pass (``sxe_mlp_train_l2_part``, normalised by the whole batch) on the
        step's stream and that part's table backward on a second stream, so that a part's backward
        (random reductions, waiting on memory) runs beside the next part's network pass (tensor
        cores, waiting on its product chain); then Adam on the tables and the network.  The table
        gradient is the same sum of the same terms as the unsplit step's (atomic additions in
        another order); the network gradient sums the parts' partials."""
        main = torch.cuda.current_stream(self.device) if stream is None else stream
        side = self._bwd_stream
        self.t += 1
        self.adam_tables.advance(self.t_dev, self.corrections, stream=main)
        self._mark("encode_fwd", main)
        self.tab.forward(x, self.enc_out, stream=main)
        self._mark("encode_fwd_end", main)
        for i, (a, b) in enumerate(self.parts()):
            self._mark("mlp_train_l2", main)
            self.mlp.mlp_train_l2_part(self.W_lowp, self.enc_out[a:b], target[a:b], self.dW, self.sq_parts[i:i + 1],
                                       self.P, din=self.d_enc[a:b], loss_scale=self.loss_scale, workspace=self.ws,
                                       stream=main)
            self._mark("mlp_train_l2_end", main)
            self._part_ready[i].record(main)
            side.wait_event(self._part_ready[i])
            self._mark("encode_bwd", side)
            self.tab.backward(x[a:b], self.d_enc[a:b], stream=side)
            self._mark("encode_bwd_end", side)
        self._bwd_done.record(side)
        main.wait_event(self._bwd_done)
        self._mark("adam_tables", main)
        self.tab.adam(self.adam_tables, self.corrections, stream=main)
        self._mark("adam_tables_end", main)
        self.adam_mlp.step_dev(self.corrections, self.W, self.mW, self.vW, self.dW, lowp=self.W_lowp, stream=main)
        self._mark("adam_mlp_end", main)

    def _table_step_overlapped(self, x, stream) -> None:
        F, T = self.enc.n_features, self.enc.T
        main = torch.cuda.current_stream(self.device) if stream is None else stream
        flat = self.tables.view(-1)
        for i, (lb, le) in enumerate(self.chunks):
            self.enc.encode_bwd(x, self.d_enc, self.state, grad_stride=4 * F, grad_offset=3 * F,
                                touched=self.touched, levels=(lb, le), stream=main)
            self._ready[i].record(main)
            self._aux.wait_event(self._ready[i])
            a, b = lb * T, le * T
            self.adam_tables.step_touched_dev(self.corrections, self.state[a:b], self.touched[a // 32:b // 32],
                                              flat[a * F:b * F], F, stream=self._aux)
        self._joined.record(self._aux)

    def capture(self, x: torch.Tensor, target: torch.Tensor, warmup: int = 2) -> None:
        """Record one step on the fixed input buffers x and target into a CUDA graph (after
        ``warmup`` ordinary steps on them, which train like any other step)."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.step(x, target)
        torch.cuda.current_stream(self.device).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step(x, target)
        self.t -= 1                      # recording did not run the step
        self._graph_io = (x, target)

    def replay(self) -> None:
        """One step on the current contents of the buffers given to ``capture``."""
        self.t += 1
        self.graph.replay()

    def loss(self) -> float:
        """Mean squared error of the last step (synchronises)."""
        return float(self.sq_parts.sum().item()) / (self.P * self.mlp.n_out)

    def table_params(self) -> torch.Tensor:
        """binary32 master table parameters as [L, T, F]."""
        return self.tab.params()

    def table_grads(self) -> torch.Tensor:
        """Table gradient accumulated since the last Adam step, [L, T, F]."""
        return self.tab.grads()


class HostFeed:
    """Trains from batches in pinned host memory with the copies off the critical path.

    Two input-buffer pairs live on the device, each with its own recording of the training step
    (a CUDA graph).  ``step(x_host, target_host)`` copies the batch into the free pair on a copy
    stream, replays that pair's graph on the current stream once the copy has landed, and sends the
    step's loss back to pinned host memory; it then returns the loss of the step before, so the
    host stays one step ahead of the device and the copy of batch k+1 runs while step k computes.
    Every step still moves its whole batch host -> device and its loss device -> host."""

    def __init__(self, trainer: Trainer, first_batch, warmup: int = 2):
        tr = self.tr = trainer
        x0, t0 = first_batch
        dev = tr.device
        self.bx = [torch.empty(x0.shape, dtype=x0.dtype, device=dev) for _ in range(2)]
        self.bt = [torch.empty(t0.shape, dtype=t0.dtype, device=dev) for _ in range(2)]
        for i in range(2):
            self.bx[i].copy_(x0)
            self.bt[i].copy_(t0)
        tr.capture(self.bx[0], self.bt[0], warmup=warmup)
        g0 = tr.graph
        tr.capture(self.bx[1], self.bt[1], warmup=0)
        self.graphs = [g0, tr.graph]
        self.copy = torch.cuda.Stream(device=dev)
        self.copy.wait_stream(torch.cuda.current_stream(dev))
        self._ready = [torch.cuda.Event() for _ in range(2)]
        self._free = [torch.cuda.Event() for _ in range(2)]
        self._done = [torch.cuda.Event() for _ in range(2)]
        self._loss = torch.zeros((2, tr.split), dtype=torch.float32).pin_memory()   # per pair: the parts' sums
        self._scale = 1.0 / (tr.P * tr.mlp.n_out)
        self.k = 0

    def step(self, x_host: torch.Tensor, target_host: torch.Tensor):
        """Queue one step on a pinned host batch; returns the previous step's loss (None at first)."""
        i = self.k % 2
        main = torch.cuda.current_stream(self.tr.device)
        if self.k >= 2:
            self.copy.wait_event(self._free[i])          # step k-2, which read this pair, is done
        with torch.cuda.stream(self.copy):
            self.bx[i].copy_(x_host, non_blocking=True)
            self.bt[i].copy_(target_host, non_blocking=True)
            self._ready[i].record(self.copy)
        main.wait_event(self._ready[i])
        self.tr.t += 1
        self.graphs[i].replay()
        self._free[i].record(main)
        self._loss[i].copy_(self.tr.sq_parts, non_blocking=True)
        self._done[i].record(main)
        prev = None
        if self.k >= 1:
            j = 1 - i
            self._done[j].synchronize()
            prev = float(self._loss[j].sum()) * self._scale
        self.k += 1
        return prev

    def finish(self) -> float:
        """Waits for the last queued step and returns its loss."""
        j = (self.k - 1) % 2
        self._done[j].synchronize()
        return float(self._loss[j].sum()) * self._scale


def _main(argv=None):
    """Train on seeded synthetic batches and print the time per step:
    ``python -m paper_2311_15439_gb300.trainer --workload sdf`` (d = 3, L = 16, F = 2, T = 2^19
    bf16, network 32-64-1, 2^20 points per step: half uniform, half near a seeded union of spheres
    and tori, target their signed distance) or ``--workload image`` (d = 2, L = 16, F = 2,
    T = 2^22 fp16, network 32-64-64-3, 2^18 points of a procedural image per step)."""
    import argparse
    ap = argparse.ArgumentParser(description=_main.__doc__)
    ap.add_argument("--workload", default="sdf", choices=["sdf", "image"])
    ap.add_argument("--kind", default="simplex", choices=["simplex", "grid"])
    ap.add_argument("--points", type=int, default=0, help="points per step (default: the workload's)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--repeat", type=int, default=10)
    ap.add_argument("--split-coarse", default="auto", choices=["auto", "on", "off"])
    a = ap.parse_args(argv)
    split = {"auto": "auto", "on": True, "off": False}[a.split_coarse]
    dev = torch.device("cuda")
    if a.workload == "sdf":
        P = a.points or 1 << 20
        scene = synth.SphereTorusScene(5)
        xs = [synth.sdf_points(P, 300 + i) for i in range(4)]
        batches = [(torch.from_numpy(x).to(dev), torch.from_numpy(scene.sdf(x)).to(dev)) for x in xs]
        tr = Trainer(Encoder(3, 16, 2, 19, 16.0, 1.38, kind=a.kind, table_dtype="bf16"),
                     Mlp(32, 1, n_hidden=1, dtype="bf16"), P, seed=6, device=dev, split_coarse=split)
    else:
        P = a.points or 1 << 18
        img = synth.ProceduralImage(1, size=16384, n_waves=64)
        xs = [synth.uniform_points(P, 2, 400 + i) for i in range(4)]
        batches = [(torch.from_numpy(x).to(dev), torch.from_numpy(img.sample(x)).to(dev)) for x in xs]
        tr = Trainer(Encoder(2, 16, 2, 22, 16.0, 2.0, kind=a.kind, table_dtype="f16"),
                     Mlp(32, 3, n_hidden=2, dtype="f16"), P, seed=3, device=dev, split_coarse=split)
    for i in range(a.warmup):
        tr.step(*batches[i % 4])
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for i in range(a.repeat):
        tr.step(*batches[i % 4])
    e.record()
    torch.cuda.synchronize()
    print("train %s %s: %d points, %s layout, coarse levels on a second stream: %s: %.3f ms per step, loss %.4g" %
          (a.workload, a.kind, P, tr.tab.layout, tr.tab.split_coarse, s.elapsed_time(e) / a.repeat, tr.loss()))


if __name__ == "__main__":
    _main()
