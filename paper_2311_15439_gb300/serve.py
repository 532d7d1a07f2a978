"""Continuous-batching query server for trained fields (encoding + network resident on the GPU).

Two implementations of the same loop: ``NativeFieldServer`` runs it in the library
(``sxe_server_*``: a C++ scheduler thread, stream slots with high- and normal-priority streams,
completion by host callbacks; the production path) and ``FieldServer`` below in Python (the
readable form, kept as a reference and for comparison).

Requests carry a dimension d and a block of points in pinned host memory; the answer is
the field value at each point (``sxe_encode_fwd`` then ``sxe_mlp_fwd``).  One scheduler
thread owns the GPU work:

* **admission by memory** -- a batch is launched only if the device bytes it needs (points,
  encoding, output) fit in the budget next to the batches already in flight; otherwise it
  waits for completions.  A request that can never fit is answered with an error;
* **continuous batching** -- queued requests of the same d are merged (FIFO order, up to
  ``max_batch_points``) into one launch when a stream slot is free, while earlier batches
  are still running;
* **overlap** -- each admitted batch runs on its own CUDA stream slot: host-to-device copy
  of its points, the two kernels, device-to-host copy of the values; batches on different
  slots overlap on the device.

Every point's value depends only on that point (the kernels have no cross-point
arithmetic), so a request's answer is the same whether it ran alone or merged.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .api import Encoder, Mlp


@dataclass
class Field:
    """A trained field of dimension d: encoder, its low-precision tables, network and weights."""
    encoder: Encoder
    tables: torch.Tensor
    mlp: Mlp
    weights: torch.Tensor

    @property
    def d(self) -> int:
        return self.encoder.d

    def bytes_per_point(self) -> int:
        return 4 * self.encoder.d + 2 * self.encoder.n_out + 4 * self.mlp.n_out


@dataclass(eq=False)          # identity equality: requests are removed from queues by identity
class Request:
    d: int
    x: torch.Tensor                        # [P, d] float32, pinned host memory
    rid: int = 0
    t_arrival: float = 0.0
    t_done: float = 0.0
    y: torch.Tensor | None = None          # [P, n_out] float32, pinned host memory
    error: str | None = None
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def n_points(self) -> int:
        return int(self.x.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival

    def wait(self, timeout: float | None = None) -> bool:
        return self.done.wait(timeout)


class _Batch:
    def __init__(self, reqs, slot, nbytes, bufs, event):
        self.reqs, self.slot, self.nbytes, self.bufs, self.event = reqs, slot, nbytes, bufs, event


class FieldServer:
    def __init__(self, fields: dict[int, Field], *, mem_budget_bytes: int = 2 << 30, n_slots: int = 4,
                 max_batch_points: int = 1 << 22, device="cuda"):
        self.fields = fields
        self.device = torch.device(device)
        self.budget = int(mem_budget_bytes)
        self.max_batch = int(max_batch_points)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_slots)]
        self.free_slots = collections.deque(range(n_slots))
        self.queue: collections.deque[Request] = collections.deque()
        self.inflight: list[_Batch] = []
        self.used = 0
        self.lock = threading.Lock()
        self.wake = threading.Event()
        self.running = False
        self.thread = None
        self.n_batches = 0
        self.n_launch_kernels = 0
        self.peak_used = 0
        self.failure = None
        self._next_id = 0

    # ---- client side --------------------------------------------------------------
    def submit(self, d: int, x_host: torch.Tensor, y_host: torch.Tensor | None = None) -> Request:
        """Queue a request; ``y_host`` (pinned, [P, n_out] float32) receives the values if given."""
        r = Request(d=d, x=x_host, y=y_host)
        with self.lock:
            r.rid = self._next_id
            self._next_id += 1
            r.t_arrival = time.perf_counter()
            self.queue.append(r)
        self.wake.set()
        return r

    def start(self):
        self.running = True
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()
        return self

    def stop(self, drain: bool = True):
        if drain:
            while self.thread is not None and self.thread.is_alive():
                with self.lock:
                    if not self.queue and not self.inflight:
                        break
                time.sleep(1e-4)
        self.running = False
        self.wake.set()
        if self.thread is not None:
            self.thread.join()

    # ---- scheduler ------------------------------------------------------------------
    def _need_bytes(self, f: Field, P: int) -> int:
        return P * f.bytes_per_point() + 3 * 256

    def _finish(self, b: _Batch):
        now = time.perf_counter()
        for r in b.reqs:
            r.t_done = now
            r.done.set()
        self.used -= b.nbytes
        self.free_slots.append(b.slot)

    def _reject(self, r: Request, msg: str):
        r.error = msg
        r.t_done = time.perf_counter()
        r.done.set()

    _REJECTED = "rejected"

    def _take_batch(self):
        """Head request plus later queued requests of the same d, up to max_batch points.
        Returns the batch, None if it must wait for memory, or _REJECTED."""
        head = self.queue[0]
        f = self.fields.get(head.d)
        if (f is None or head.x.dim() != 2 or head.x.shape[1] != head.d or head.x.dtype != torch.float32
                or head.n_points == 0):
            self.queue.popleft()
            self._reject(head, "no field of dimension %d, or malformed / empty points" % head.d)
            return self._REJECTED
        if head.n_points > self.max_batch or self._need_bytes(f, head.n_points) > self.budget:
            self.queue.popleft()
            self._reject(head, "request of %d points exceeds the admission limits" % head.n_points)
            return self._REJECTED
        group, P = [], 0
        for r in list(self.queue):
            if (r.d == head.d and P + r.n_points <= self.max_batch and r.x.dim() == 2 and r.x.shape[1] == r.d
                    and r.n_points > 0 and r.x.dtype == torch.float32):
                group.append(r)
                P += r.n_points
        need = self._need_bytes(f, P)
        if self.used + need > self.budget:
            # shrink to what fits now (at least the head if it alone fits once memory frees up)
            while len(group) > 1 and self.used + self._need_bytes(f, P) > self.budget:
                P -= group.pop().n_points
            need = self._need_bytes(f, P)
            if self.used + need > self.budget:
                return None
        for r in group:
            self.queue.remove(r)
        return f, group, P, need

    def _launch(self, f: Field, group, P: int, need: int):
        slot = self.free_slots.popleft()
        s = self.streams[slot]
        with torch.cuda.stream(s):
            x = torch.empty((P, f.d), dtype=torch.float32, device=self.device)
            enc = torch.empty((P, f.encoder.n_out), dtype=f.tables.dtype, device=self.device)
            y = torch.empty((P, f.mlp.n_out), dtype=torch.float32, device=self.device)
            o = 0
            for r in group:
                x[o:o + r.n_points].copy_(r.x, non_blocking=True)
                o += r.n_points
            f.encoder.encode_fwd(x, f.tables, enc, stream=s)
            f.mlp.mlp_fwd(f.weights, enc, y, stream=s)
            o = 0
            for r in group:
                if r.y is None or tuple(r.y.shape) != (r.n_points, f.mlp.n_out):
                    r.y = torch.empty((r.n_points, f.mlp.n_out), dtype=torch.float32, pin_memory=True)
                r.y.copy_(y[o:o + r.n_points], non_blocking=True)
                o += r.n_points
            ev = torch.cuda.Event()
            ev.record(s)
        self.used += need
        self.peak_used = max(self.peak_used, self.used)
        self.n_batches += 1
        self.n_launch_kernels += 2
        self.inflight.append(_Batch(group, slot, need, (x, enc, y), ev))

    def _loop(self):
        try:
            self._serve()
        except BaseException as exc:           # never leave a client waiting on a dead scheduler
            with self.lock:
                pending = list(self.queue) + [r for b in self.inflight for r in b.reqs]
                self.queue.clear()
                self.inflight.clear()
            for r in pending:
                if not r.done.is_set():
                    self._reject(r, "scheduler failed: %r" % (exc,))
            self.failure = exc

    def _serve(self):
        while self.running or self.queue or self.inflight:
            progressed = False
            with self.lock:
                for b in [b for b in self.inflight if b.event.query()]:
                    self.inflight.remove(b)
                    self._finish(b)
                    progressed = True
                while self.queue and self.free_slots:
                    taken = self._take_batch()
                    if taken is None:
                        break                      # wait for memory to free up
                    if taken is not self._REJECTED:
                        self._launch(*taken)
                    progressed = True
            if not progressed:
                self.wake.wait(timeout=5e-5)
                self.wake.clear()


class NativeRequest:
    """A request of ``NativeFieldServer``: same interface as ``Request`` (wait, latency, y, error)."""

    def __init__(self, server, d: int, x: torch.Tensor, y: torch.Tensor, rid: int | None, error: str | None = None):
        self.server, self.d, self.x, self.y, self.rid = server, d, x, y, rid
        self.error = error
        self._latency = 0.0 if error is not None else None

    @property
    def n_points(self) -> int:
        return int(self.x.shape[0])

    @property
    def latency(self) -> float:
        return self._latency

    def wait(self, timeout: float | None = None) -> bool:
        """True once the request has completed (or failed); its latency is measured in the
        library, from submission to the completion callback."""
        if self._latency is not None:
            return True
        import ctypes
        from . import _lib as L
        state, lat = ctypes.c_int32(0), ctypes.c_double(0.0)
        t_us = -1 if timeout is None else int(timeout * 1e6)
        while True:
            step = 1_000_000 if t_us < 0 else max(0, min(t_us, 1_000_000))
            L.check(L.lib().sxe_server_wait(self.server._h, self.rid, step, ctypes.byref(state), ctypes.byref(lat)),
                    "sxe_server_wait")
            if state.value != 0:
                self._latency = lat.value
                if state.value == 2:
                    self.error = L.lib().sxe_last_error().decode(errors="replace")
                return True
            if t_us >= 0:
                t_us -= step
                if t_us <= 0:
                    return False


class NativeFieldServer:
    """The same serving loop as ``FieldServer`` run by the library (``sxe_server_*``): a native
    scheduler thread, the batches' buffers carved from one device arena of ``mem_budget_bytes``
    (allocated here by torch), a stream per slot and a host callback completing each batch;
    batches of at most ``priority_points`` points run on high-priority streams.
    ``submit`` answers a request the library refuses (unknown d, malformed, oversize) with a
    request that carries the error, as ``FieldServer`` does."""

    def __init__(self, fields: dict[int, Field], *, mem_budget_bytes: int = 2 << 30, n_slots: int = 4,
                 max_batch_points: int = 1 << 22, priority_points: int = 1 << 20, device="cuda"):
        import ctypes
        from . import _lib as L
        self.fields = fields
        self.device = torch.device(device)
        self._L = L.lib()                   # kept for __del__, which may run at interpreter exit
        self.arena = torch.empty((int(mem_budget_bytes),), dtype=torch.uint8, device=self.device)
        desc = L.ServerDesc(self.arena.data_ptr(), int(mem_budget_bytes), int(n_slots), int(max_batch_points),
                            int(priority_points))
        h = ctypes.c_void_p()
        L.check(L.lib().sxe_server_create(ctypes.byref(desc), ctypes.byref(h)), "sxe_server_create")
        self._h = h
        for d, f in fields.items():
            L.check(L.lib().sxe_server_add_field(h, f.encoder._h, f.tables.data_ptr(), ctypes.byref(f.mlp.desc),
                                                 f.weights.data_ptr()), "sxe_server_add_field")

    def start(self):
        from . import _lib as L
        L.check(L.lib().sxe_server_start(self._h), "sxe_server_start")
        return self

    def submit(self, d: int, x_host: torch.Tensor, y_host: torch.Tensor | None = None) -> NativeRequest:
        import ctypes
        from . import _lib as L
        f = self.fields.get(d)
        if (f is None or x_host.dim() != 2 or x_host.shape[1] != d or x_host.dtype != torch.float32
                or not x_host.is_contiguous() or x_host.shape[0] == 0):
            return NativeRequest(self, d, x_host, None, None, error="no field of dimension %d, or malformed / empty "
                                                                     "points" % d)
        if y_host is None or tuple(y_host.shape) != (x_host.shape[0], f.mlp.n_out):
            y_host = torch.empty((x_host.shape[0], f.mlp.n_out), dtype=torch.float32, pin_memory=True)
        rid = ctypes.c_int64(-1)
        st = L.lib().sxe_server_submit(self._h, int(d), x_host.data_ptr(), int(x_host.shape[0]), y_host.data_ptr(),
                                       ctypes.byref(rid))
        if st != L.SXE_OK:
            return NativeRequest(self, d, x_host, y_host, None, error=L.lib().sxe_last_error().decode(errors="replace"))
        return NativeRequest(self, d, x_host, y_host, rid.value)

    def stop(self, drain: bool = True):
        from . import _lib as L
        L.check(L.lib().sxe_server_stop(self._h, 1 if drain else 0), "sxe_server_stop")

    def _stats(self):
        import ctypes
        from . import _lib as L
        nb, peak = ctypes.c_int64(0), ctypes.c_int64(0)
        L.check(L.lib().sxe_server_stats(self._h, ctypes.byref(nb), ctypes.byref(peak)), "sxe_server_stats")
        return nb.value, peak.value

    @property
    def n_batches(self) -> int:
        return self._stats()[0]

    @property
    def peak_used(self) -> int:
        return self._stats()[1]

    def __del__(self):
        h, lib = getattr(self, "_h", None), getattr(self, "_L", None)
        if h is not None and h.value and lib is not None:
            lib.sxe_server_destroy(h)
            self._h = None


def make_field(d: int, *, n_levels=16, n_features=2, log2_T=19, base_res=16.0, growth=1.38, kind="simplex",
               res_mode="raw", n_out=1, seed=0, device="cuda", table_dtype="f16") -> Field:
    """A field with seeded tables U(-1e-1, 1e-1) and He-uniform weights (a stand-in for a trained one:
    the serving cost does not depend on the values)."""
    from . import synth
    enc = Encoder(d, n_levels, n_features, log2_T, base_res, growth, kind=kind, res_mode=res_mode,
                  table_dtype=table_dtype)
    vals = synth.uniform_tables(n_levels, 1 << log2_T, n_features, seed, dtype="f32", scale=1e-1)[0]
    dt = {"f16": torch.float16, "bf16": torch.bfloat16, "f32": torch.float32}[table_dtype]
    tables = torch.from_numpy(vals).to(device=device, dtype=dt)
    mlp = Mlp(n_levels * n_features, n_out, n_hidden=2, dtype="f16")
    W = torch.from_numpy(mlp.init_weights(seed + 1)).to(device=device, dtype=torch.float16)
    return Field(enc, tables, mlp, W)


def poisson_load(rate_hz: float, n_requests: int, dims, p_min: int, p_max: int, seed: int):
    """Seeded arrival offsets (s), dimensions and log-uniform sizes of a request stream."""
    g = np.random.Generator(np.random.PCG64(seed))
    gaps = g.exponential(1.0 / rate_hz, size=n_requests)
    sizes = np.exp(g.uniform(np.log(p_min), np.log(p_max), size=n_requests)).astype(np.int64)
    ds = g.choice(np.asarray(dims), size=n_requests)
    return np.cumsum(gaps), ds, sizes


def run_load(server: FieldServer, arrivals, ds, sizes, host_points: dict[int, torch.Tensor], seed: int = 0):
    """Replay a request stream in real time; returns the list of completed requests."""
    g = np.random.Generator(np.random.PCG64(seed + 1))
    reqs = []
    t0 = time.perf_counter()
    for t, d, P in zip(arrivals, ds, sizes):
        src = host_points[int(d)]
        o = int(g.integers(0, src.shape[0] - P + 1))
        while True:                                     # sleep (releasing the GIL) until just before t
            ahead = t - (time.perf_counter() - t0)
            if ahead <= 0:
                break
            time.sleep(ahead - 5e-5 if ahead > 1e-4 else 0)
        reqs.append(server.submit(int(d), src[o:o + int(P)]))
    for r in reqs:
        if not r.wait(120.0):
            raise TimeoutError("request %d (%d points, d=%d) did not complete" % (r.rid, r.n_points, r.d))
    return reqs, time.perf_counter() - t0
