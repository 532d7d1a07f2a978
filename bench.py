"""Benchmark: simplex-encoding training step throughput (points/s) on one GB300.

Workload (the image-fitting configuration): d = 2, L = 16 levels, F = 2 features,
T = 2^22 entries per level in fp16, base resolution 16, growth 2.0, 64-wide network
32 -> 64 -> 64 -> 3 (fp16 tensor cores, fp32 accumulation), L2 loss against a
procedural 16384^2 RGB image, Adam on fp32 master copies, 2^18 uniformly drawn points
per step.  A step is one pass of the whole path: encode forward, network forward +
loss + backward, encode backward (scatter into the tables), Adam on the touched table
entries and on the network.

Prints one JSON line.  ``value`` is device-timed (inputs resident in HBM), ``e2e`` the
same metric through the public API with the batch copied from pinned host memory and
the loss read back every step.  ``--impl reference`` times the FP64 oracle on the
host cores instead.  Under torchrun every rank trains its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFG = dict(d=2, n_levels=16, n_features=2, log2_T=22, base_res=16.0, growth=2.0)
BATCH = 1 << 18
N_OUT = 3
WORKLOAD = "image_fit_2d_L16_F2_T2^22_fp16_mlp64x2_P2^18"
# The headline metric as the benchmark plan names it; the value is points/s of one whole training
# step of the image workload, which contains the encoding's forward and backward (see the line's
# config.step), and the grid, plain binary32 and serving figures are the line's extra records.
METRIC = "simplex encode fwd+bwd points/s vs 2^d grid & plain FP32 path; serve p50/p99 ms"
N_POOL = 8   # distinct resident batches cycled through the timed steps

# DRAM traffic of one step's launch of a stage (dram__bytes_read.sum + dram__bytes_write.sum of its
# kernels in one ncu capture of this workload, profiles/train_step_image2d_L16_T2^22_P2^18_dram_traffic.md),
# with the SHA-1 of the kernel sources it was taken on: reported only while those sources are unchanged.
TRAFFIC = {
    "encode_bwd": (35.8e6 + 755.7e6, "b8bc06d238dec3bd0fd796c812d8e2ac3a899f34",
                   ("encode.cu", "encode_common.cuh", "lattice.cuh")),
}


def _traffic(stage):
    import hashlib
    if stage not in TRAFFIC:
        return None
    nbytes, sha, files = TRAFFIC[stage]
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2311_15439_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return nbytes if h.hexdigest() == sha else None


_PROBE = None


def probe_lib():
    """The bench-only random-access probe (``bench_probe.cu`` beside this file), compiled for
    sm_103a into ``_build/libsxeprobe.so`` on first use and loaded with ctypes."""
    global _PROBE
    if _PROBE is None:
        import ctypes
        from paper_2311_15439_gb300 import build as B
        src = os.path.join(ROOT, "bench_probe.cu")
        so = os.path.join(ROOT, "_build", "libsxeprobe.so")
        os.makedirs(os.path.dirname(so), exist_ok=True)
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            subprocess.run([B.nvcc(), *B.ARCH, "-O3", "-lineinfo", "-shared", "-Xcompiler", "-fPIC", src,
                            "-o", so + ".tmp"], check=True)
            os.replace(so + ".tmp", so)
        lib = ctypes.CDLL(so)
        fn = lib.sxe_probe_random_access
        fn.restype = ctypes.c_int
        fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                       ctypes.c_void_p, ctypes.c_void_p]
        _PROBE = fn
    return _PROBE


def probe(kind, buf_ptr, n_slots, slot_floats, n_ops, seed, sink_ptr, stream):
    """One launch of the random-access probe; raises on an argument or launch error."""
    rc = probe_lib()(kind, buf_ptr, n_slots, slot_floats, n_ops, seed, sink_ptr, stream)
    if rc != 0:
        raise RuntimeError("sxe_probe_random_access failed with status %d" % rc)


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of every rank's value (the job's time is its slowest rank's); world 1: x."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank_step: int, steps: int, world: int, ms: float) -> float:
    """Whole-job points/s: every rank's points over the slowest rank's time (weak scaling)."""
    return points_per_rank_step * steps * world / (ms / 1e3)


def _tensor_peak():
    """Dense fp16 tensor peak for a kernel timed inside a long step: the measured sustained
    bf16 figure (fp16 and bf16 run at the same dense rate)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops_sustained"])
    except Exception:
        return 1700.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while active."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if "Active" in r[3 + i]
                          and "Not" not in r[3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------
def make_batches(n, seed0=1000):
    from paper_2311_15439_gb300 import synth
    img = synth.ProceduralImage(seed=7, size=16384, n_waves=64)
    xs, ts = [], []
    for i in range(n):
        x = synth.uniform_points(BATCH, 2, seed0 + i)
        xs.append(x)
        ts.append(img.sample(x))
    return xs, ts


def _stage_work(n_touched, F=2, L=16, d=2, width=64, n_in=32):
    """Algorithmic work of each timed kernel of one step:
    bytes for the memory-bound kernels, FLOPs for the network."""
    V = d + 1
    fwd = BATCH * (4 * d + L * V * 2 * F + L * F * 2)              # x, fp16 gathers, fp16 encoding
    bwd = BATCH * (4 * d + 4 * L * F + L * V * 2 * 4 * F)           # x, dL/d(enc), fp32 RMW per vertex
    adam = n_touched * (2 * 16 * F + 2 * F) + L * (1 << 22) // 8    # record r+w, fp16 copy; bitmap scan
    flops = 2 * (n_in * width + width * width + width * N_OUT)     # forward multiply-adds per point
    flops = 3 * flops * BATCH                                      # forward + delta + weight-gradient GEMMs
    return {"encode_fwd": ("hbm", fwd), "encode_bwd": ("hbm", bwd), "adam_tables": ("hbm", adam),
            "mlp_train_l2": ("tensor", flops)}


def count_touched(tr, x):
    """Entries that one batch touches (for the table stage's algorithmic bytes), and the 32-byte
    sectors of the fp16 table they lie in (8 entries of F = 2 fp16 values per sector: one byte
    of the touched bitmap)."""
    import torch
    enc = tr.enc
    dense = torch.zeros(enc.table_shape(), dtype=torch.float32, device=x.device)
    bm = torch.zeros_like(tr.touched)
    enc.encode_bwd(x, torch.ones((x.shape[0], enc.n_out), device=x.device), dense, touched=bm)
    bytes_ = bm.cpu().numpy().view(np.uint8)
    return int(np.unpackbits(bytes_).sum()), int(np.count_nonzero(bytes_))


def _graph_events_supported() -> bool:
    """Whether timing events can be recorded as nodes of a CUDA graph (``external`` events)."""
    import torch
    try:
        torch.cuda.Event(enable_timing=True, external=True)
    except TypeError:
        return False
    return True


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2311_15439_gb300 import build as B
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import HostFeed, Trainer

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    B.build()   # no-op when up to date

    from paper_2311_15439_gb300 import _lib
    _lib.check(_lib.lib().sxe_mlp_set_kernel({"auto": _lib.SXE_MLP_KERNEL_AUTO, "mma_sync": _lib.SXE_MLP_KERNEL_MMA_SYNC,
                                              "tcgen05": _lib.SXE_MLP_KERNEL_TCGEN05,
                                              "tcgen05_pipelined": _lib.SXE_MLP_KERNEL_TCGEN05_PIPELINED,
                                              "tcgen05_3tile": _lib.SXE_MLP_KERNEL_TCGEN05_3TILE}[args.mlp_kernel]),
               "sxe_mlp_set_kernel")
    enc = Encoder(**CFG, kind=args.kind, table_dtype="f16")
    mlp = Mlp(CFG["n_levels"] * CFG["n_features"], N_OUT, n_hidden=2, dtype="f16")
    tr = Trainer(enc, mlp, BATCH, seed=rank, device=dev, table_layout="records", split_batch=args.split_batch)
    xs, ts = make_batches(N_POOL, seed0=1000 + 100 * rank)
    xd = [torch.from_numpy(x).to(dev) for x in xs]
    td = [torch.from_numpy(t).to(dev) for t in ts]
    stream = torch.cuda.current_stream(dev)

    for i in range(args.warmup):
        tr.step(xd[i % N_POOL], td[i % N_POOL])
    torch.cuda.synchronize(dev)

    # ---- device-timed region: K steps, each a replay of a recording of Trainer.step (a CUDA graph,
    # as a training loop runs it) on one of the resident batches, every recording a distinct graph.
    # Timing events recorded while a step is recorded are nodes of its graph, on the stream that the
    # stage's kernels run on (the table backward of a split step on its second stream).  Each event
    # node costs about 2.5 us of the step, so the timed recordings carry events around the dominant
    # kernel's stage only; a shorter pass before it, on recordings with events around every stage,
    # gives the time of each stage and picks that kernel.
    names = ["encode_fwd", "mlp_train_l2", "encode_bwd", "adam_tables", "adam_mlp"]
    graphs = _graph_events_supported()

    def record(n, only):
        recs = []
        tr.stage_only = only
        for k in range(n):
            tr.stage_events = {}
            tr.capture(xd[k % N_POOL], td[k % N_POOL], warmup=0)
            recs.append((tr.graph, tr.stage_events))
        tr.stage_events, tr.stage_only = None, None
        for g, _ in recs:                       # first launches (graph upload) outside any timed span
            tr.t += 1
            g.replay()
        torch.cuda.synchronize(dev)
        return recs

    def stage_ms(evs, stages, n):
        evs = dict(evs)
        if "adam_mlp" in stages:
            evs["adam_mlp"] = evs["adam_tables_end"]
        return {m: float(sum(a.elapsed_time(b) for a, b in zip(evs[m], evs[m + "_end"]))) / n for m in stages}

    n_pre = max(8, args.steps // 4)
    if graphs:
        pre = record(n_pre, None)
        for g, _ in pre:
            tr.t += 1
            g.replay()
        torch.cuda.synchronize(dev)
        per_kernel = stage_ms({m: [e for _, r in pre for e in r[m]] for m in pre[0][1]}, names, n_pre)
        del pre
    else:                                       # no timing events inside graphs: eager steps
        tr.stage_events = {}
        for k in range(n_pre):
            tr.step(xd[k % N_POOL], td[k % N_POOL])
        torch.cuda.synchronize(dev)
        per_kernel = stage_ms(tr.stage_events, names, n_pre)
        tr.stage_events = None
    work = _stage_work(1)
    dom = max(work, key=lambda m: per_kernel[m])
    only = {dom, "adam_tables"} if dom == "adam_mlp" else {dom}
    recordings = record(args.steps, only) if graphs else []
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if not graphs:
        tr.stage_events, tr.stage_only = {}, only
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        if recordings:
            for g, _ in recordings:
                tr.t += 1
                g.replay()
        else:
            for k in range(args.steps):
                tr.step(xd[k % N_POOL], td[k % N_POOL])
        stop.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
    if recordings:
        ev = {m: [e for _, r in recordings for e in r[m]] for m in recordings[0][1]}
    else:
        ev, tr.stage_events, tr.stage_only = tr.stage_events, None, None
    dom_ms = stage_ms(ev, [dom], args.steps)[dom]
    step_form = "replays of recorded steps (CUDA graphs)" if recordings else "eager steps"
    del recordings, ev
    ms = start.elapsed_time(stop)
    ms = max_over_ranks(ms, world, dev)
    loss = tr.loss()
    n_touched, _ = count_touched(tr, xd[0])

    # ---- end to end through the public API (HostFeed): every step copies its batch from pinned
    # host memory to the device (copy stream, double-buffered), replays the recorded step and reads
    # its loss back to the host (one step behind)
    hx = [torch.from_numpy(x).pin_memory() for x in xs]
    ht = [torch.from_numpy(t).pin_memory() for t in ts]
    feed = HostFeed(tr, (hx[0], ht[0]))
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s2.record(stream)
    feed.copy.wait_stream(stream)                   # the first copy starts inside the timed region
    for k in range(e2e_steps):
        feed.step(hx[k % N_POOL], ht[k % N_POOL])
    e2.record(stream)
    feed.finish()
    torch.cuda.synchronize(dev)
    ms_e2e = s2.elapsed_time(e2)
    ms_e2e = max_over_ranks(ms_e2e, world, dev)

    # ---- comparators on the same GPU (encode forward + backward only, equal L, F, T)
    comparators = encode_sweep(dev) if (rank == 0 and not args.no_sweep) else None
    serving = serve_bench(dev) if (rank == 0 and not args.no_serve) else None
    peaks_ra = random_access_peaks(dev, tr.state.numel() * 4, tr.tables) if rank == 0 else None
    volume = volume_sweep(dev) if (rank == 0 and not args.no_volume) else None
    sdf = sdf_train(dev) if (rank == 0 and not args.no_sweep) else None
    grid_img = image_step_variants(dev, xd, td) if (rank == 0 and not args.no_sweep and
                                                     args.kind == "simplex") else None
    per_cfg = per_config_encode(dev) if (rank == 0 and not args.no_sweep) else None
    quality = (fit_quality(dev, args.quality_steps, max(1, args.quality_steps * 2 // 5))
               if (rank == 0 and args.quality_steps > 0) else None)

    if rank == 0:
        value = job_throughput(BATCH, args.steps, world, ms)
        work = _stage_work(n_touched)
        bound, amount = work[dom]
        hbm_peak, peak_src = _peaks()
        if bound == "hbm":
            achieved = amount / (dom_ms / 1e3) / 1e9
            peak, unit = hbm_peak, "GB/s"
        else:
            achieved = amount / (dom_ms / 1e3) / 1e12
            peak, unit = _tensor_peak(), "TFLOP/s"
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "kind": args.kind, "res_mode": "raw",
                       "step": "encode forward, network forward + L2 loss + backward, encode backward into the "
                               "table state, Adam on the touched table entries and on the network",
                       "split_batch": tr.split, "timed_steps": step_form,
                       "mlp_kernel": {"auto": "auto (three-tile tcgen05 kernel for this network)", "mma_sync": "mma_sync",
                                      "tcgen05": "tcgen05", "tcgen05_pipelined": "tcgen05_pipelined",
                                      "tcgen05_3tile": "tcgen05_3tile"}[args.mlp_kernel],
                       "global_batch": BATCH * world,
                       "points_per_step_per_gpu": BATCH, "parallelism": "replicas (one per GPU)",
                       "l2": "working set > L2: 256 MiB fp16 tables + 2 GiB fp32 table state records, no flush",
                       "batches": "%d resident distinct batches cycled" % N_POOL},
            "e2e": {"value": job_throughput(BATCH, e2e_steps, world, ms_e2e), "unit": "points/s",
                    "h2d_bytes_per_step": BATCH * (2 + N_OUT) * 4, "d2h_bytes_per_step": 4 * tr.split,
                    "api": "trainer.HostFeed.step (double-buffered copies on a copy stream, recorded step "
                           "replayed, loss read one step behind)"},
            "roofline": {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                         "frac": achieved / peak, "traffic": _traffic(dom), "peak_source": peak_src,
                         "work_per_step": amount, "touched_entries_per_step": n_touched,
                         "kernel_ms": dom_ms, "kernel_ms_source": "events around the kernel in each timed step"},
            "per_kernel_ms": per_kernel,
            "per_kernel_ms_source": "%d steps before the timed region, events around every stage" % n_pre,
            "gpu_launches": args.steps * tr.n_launches_per_step,
            "clocks": clk.summary(),
            "final_loss": loss,
        }
        contrib = BATCH * CFG["n_levels"] * (CFG["d"] + 1)
        pred_bwd = n_touched / peaks_ra["red_f2_miss"] + (contrib - n_touched) / peaks_ra["red_f2_l2"]
        line["random_access_roofline"] = {
            "kernel": "encode_bwd", "contributions": contrib, "touched_entries": n_touched,
            "peaks_ops_per_s": peaks_ra,
            "predicted_ms": pred_bwd * 1e3, "measured_ms": per_kernel["encode_bwd"],
            "frac": pred_bwd * 1e3 / per_kernel["encode_bwd"],
            "model": "first touch of an entry = one random float2 reduction missing L2; later ones hit"}
        if comparators is not None:
            line["comparators"] = comparators
        if quality is not None:
            line["fit_quality"] = quality
        if volume is not None:
            line["volume"] = volume
        if sdf is not None:
            line["sdf_train"] = sdf
        if grid_img is not None:
            line["image_step_variants"] = grid_img
        if per_cfg is not None:
            line["per_config_encode"] = per_cfg
        if serving is not None:
            line["serve"] = serving
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline_subprocess(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# The encoders every comparison runs on the same tables and points: the simplex encoding at the level
# scale of Sec. 5.1 ("raw"), the simplex encoding in Sec. 5.2's equal-memory setting (each level's
# resolution multiplied by (d+1)^((d-1)/(2d)), so that it touches as many lattice vertices as the
# grid), and the 2^d multilinear grid (Algorithm 1).
VARIANTS = (("simplex", "raw"), ("simplex", "equal_mem"), ("grid", "raw"))


def vname(kind, mode):
    return "grid" if kind == "grid" else "simplex_" + mode


def _ratios(row, key):
    """grid / simplex time ratios of one record, per res_mode of the simplex side."""
    return {"grid_over_simplex_" + m: row[vname("simplex", m)][key] / row["grid"][key]
            for m in ("raw", "equal_mem") if vname("simplex", m) in row}


def encode_sweep(dev, reps=20):
    """Encode forward+backward points/s at d = 2..5 (L = 16, F = 2, T = 2^19, fp16 tables, 2^20
    uniform points): the simplex encoder in both res_modes, the 2^d grid, and the binary32 paths
    (the optimised kernels on fp32 tables, and the plain one-thread-per-point path)."""
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.api import Encoder
    P = 1 << 20
    out = {}

    def timed(fn):
        for _ in range(3):
            fn()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        s.record()
        for _ in range(reps):
            fn()
        e.record()
        torch.cuda.synchronize(dev)
        return P * reps / (s.elapsed_time(e) / 1e3)

    for d in (2, 3, 4, 5):
        x = torch.from_numpy(synth.uniform_points(P, d, 50 + d)).to(dev)
        dout = torch.randn((P, 32), device=dev)
        row = {}
        for (kind, mode), tdt in [(v, "f16") for v in VARIANTS] + [(("simplex", "raw"), "f32")]:
            enc = Encoder(d, 16, 2, 19, 16.0, 1.38, kind=kind, res_mode=mode, table_dtype=tdt, out_dtype=tdt)
            tab = torch.zeros(enc.table_shape(), dtype=torch.float16 if tdt == "f16" else torch.float32, device=dev)
            grad = torch.zeros(enc.table_shape(), dtype=torch.float32, device=dev)
            o = torch.empty((P, 32), dtype=tab.dtype, device=dev)

            def fb():
                enc.encode_fwd(x, tab, o)
                enc.encode_bwd(x, dout, grad)
            name = vname(kind, mode) + ("" if tdt == "f16" else "_f32")
            row[name] = {"fwd_bwd_points_per_s": timed(fb), "res_mode": mode, "table_dtype": tdt}
            if tdt == "f32":                                # the plain binary32 path on the same tables
                def pl():
                    enc.encode_plain_fwd(x, tab, o)
                    enc.encode_plain_bwd(x, dout, grad)
                row["simplex_plain_f32"] = {"fwd_bwd_points_per_s": timed(pl), "res_mode": mode,
                                            "table_dtype": "f32"}
        for m in ("raw", "equal_mem"):
            row["grid_over_simplex_time_" + m] = (row[vname("simplex", m)]["fwd_bwd_points_per_s"]
                                                  / row["grid"]["fwd_bwd_points_per_s"])
        out["d%d" % d] = row
    return {"encode_fwd_bwd": out, "points": P,
            "config": "L=16 F=2 T=2^19 base 16 growth 1.38, 2^20 uniform points, fp16 tables unless _f32"}


def random_access_peaks(dev, state_bytes, table, n_ops=1 << 24, reps=5):
    """Peak rates of the scattered patterns that bound the table kernels, measured on this GPU
    with the bench-only probe: float2 reductions into random 32-byte records of a footprint the
    size of the table state (L2 misses) and of 8 MiB (L2 hits), and 4-byte gathers from the
    fp16 tables.  Returns ops/s."""
    import torch
    n_rec = 1 << int(math.log2(state_bytes // 32))
    buf = torch.zeros((n_rec, 8), dtype=torch.float32, device=dev)
    sink = torch.zeros((1,), dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    tab = table.view(torch.float32).reshape(-1)
    cases = {"red_f2_miss": (0, buf, n_rec, 8), "red_f2_l2": (0, buf, 1 << 18, 8),
             "rmw_32B_random_order": (2, buf, n_rec, 8),
             "gather_4B_table": (1, tab, 1 << int(math.log2(tab.numel())), 1),
             "gather_4B_l2": (1, buf, 1 << 20, 2)}
    out = {}
    for name, (kind, b, slots, sf) in cases.items():
        if sf < 2:          # 4-byte gathers: slots of 2 floats over the first half of the table words
            slots, sf = slots // 2, 2
        probe(kind, b.data_ptr(), slots, sf, n_ops, 1, sink.data_ptr(), st)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for r in range(reps):
            probe(kind, b.data_ptr(), slots, sf, n_ops, 2 + r, sink.data_ptr(), st)
        e.record()
        torch.cuda.synchronize(dev)
        out[name] = n_ops * reps / (s.elapsed_time(e) / 1e3)
    del buf
    return out


def volume_sweep(dev, n_rays=1 << 16, samples=(1, 4, 16, 64, 256, 1024), reps=3):
    """Volumetric rendering (Sec. 6.2): 2^16 rays from a sphere around the unit cube, S midpoint
    samples per ray, encoding (L=16, F=2, T=2^19 fp16, growth 1.38) -> density network -> field
    head -> colour network -> compositing.  Render time and encoding-stage time per S, simplex vs
    the 8-corner trilinear grid, and their ratio (the paper's Fig. of kernel run-time vs samples)."""
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.render import Renderer
    rays = [torch.from_numpy(a).to(dev) for a in synth.camera_rays(n_rays, 60)]
    res = {}
    for kind, mode in VARIANTS:
        enc = Encoder(3, 16, 2, 19, 16.0, 1.38, kind=kind, res_mode=mode, table_dtype="f16")
        vals, store = synth.uniform_tables(16, 1 << 19, 2, 61, dtype="f16", scale=1.0)
        tab = torch.from_numpy(store).to(dev)
        for S in samples:
            rr = Renderer(enc, n_rays, S, dtype="f16", device=dev)
            Wd, Wc = rr.init_weights(62)
            color = torch.empty((n_rays, 3), device=dev)
            rr.render(*rays, tab, Wd, Wc, color=color)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            torch.cuda.synchronize(dev)
            ev[0].record()
            for _ in range(reps):
                rr.render(*rays, tab, Wd, Wc, color=color)
            ev[1].record()
            x = rr.x[: n_rays * S]
            ev[2].record()
            for _ in range(reps):
                enc.encode_fwd(x, tab, rr.enc_out[: n_rays * S])
            ev[3].record()
            torch.cuda.synchronize(dev)
            res.setdefault(str(S), {})[vname(kind, mode)] = {"res_mode": mode,
                                                             "render_ms": ev[0].elapsed_time(ev[1]) / reps,
                                                             "encode_ms": ev[2].elapsed_time(ev[3]) / reps}
            del rr
            torch.cuda.empty_cache()
    for S, r in res.items():
        for m in ("raw", "equal_mem"):
            v = vname("simplex", m)
            r["grid_over_simplex_render_" + m] = r["grid"]["render_ms"] / r[v]["render_ms"]
            r["grid_over_simplex_encode_" + m] = r["grid"]["encode_ms"] / r[v]["encode_ms"]
    return {"rays": n_rays, "config": "d=3 L=16 F=2 T=2^19 fp16 growth 1.38; nets 32-64-16 and 32-64-64-3",
            "by_samples_per_ray": res, "train": volume_train(dev, rays)}


def volume_train(dev, rays, S=64, steps=10, warmup=3):
    """Training a field from ray colours (Sec. 6.2), one step = render, colour L2 loss, backward
    through the compositing, the colour network, the field head, the density network and the
    encoding, Adam on the touched table entries and on both networks (``VolumeTrainer.step``).
    Target colours are seeded uniform values: the step's work does not depend on them."""
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.render import VolumeTrainer
    R = rays[0].shape[0]
    target = torch.from_numpy(synth.rng(64).random((R, 3)).astype(np.float32)).to(dev)
    out = {"rays": R, "samples_per_ray": S, "targets": "seeded uniform colours"}
    for kind, mode in VARIANTS:
        enc = Encoder(3, 16, 2, 19, 16.0, 1.38, kind=kind, res_mode=mode, table_dtype="f16")
        vt = VolumeTrainer(enc, R, S, seed=63, device=dev)
        for _ in range(warmup):
            vt.step(*rays, target)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record()
        for _ in range(steps):
            vt.step(*rays, target)
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / steps
        out[vname(kind, mode)] = {"res_mode": mode, "ms_per_step": ms, "samples_per_s": R * S / (ms / 1e3),
                                  "table_layout": vt.tab.layout, "coarse_levels_on_second_stream": vt.tab.split_coarse}
        del vt
        torch.cuda.empty_cache()
    for m in ("raw", "equal_mem"):
        out["grid_over_simplex_time_" + m] = out["grid"]["ms_per_step"] / out[vname("simplex", m)]["ms_per_step"]
    return out


# Encode forward + backward of each configuration of the benchmark plan (the plain binary32 case,
# the image, SDF-style and volumetric workloads; the serving load is `serve`).
PER_CONFIG = [
    ("plain_fp32_2d_L8_T2^14_P2^16", dict(d=2, n_levels=8, n_features=2, log2_T=14, base_res=16.0, growth=1.5),
     "f32", 1 << 16, "uniform"),
    ("image_2d_L16_T2^22_fp16_P2^18", dict(CFG), "f16", 1 << 18, "uniform"),
    ("sdf_3d_L16_T2^19_bf16_P2^20", dict(d=3, n_levels=16, n_features=2, log2_T=19, base_res=16.0, growth=1.38),
     "bf16", 1 << 20, "sdf"),
    ("volume_3d_L16_T2^19_fp16_2^16rays_x1024", dict(d=3, n_levels=16, n_features=2, log2_T=19, base_res=16.0,
                                                      growth=1.38), "f16", 1 << 26, "rays"),
]

# ncu counters of the encoding kernels per configuration, encoder and stage, from one capture of
# ``bench.py --profile-encode`` (the volumetric configuration at 2^16 rays x 64 samples there):
# L2 sector throughput and DRAM throughput as a percentage of their peaks, L2 hit rate, DRAM bytes
# per point.  Reported only while the kernel sources hash to ENCODE_NCU_SHA.
ENCODE_NCU_SHA = 'b8bc06d238dec3bd0fd796c812d8e2ac3a899f34'
ENCODE_NCU = {
 "plain_fp32_2d_L8_T2^14_P2^16/simplex_raw/fwd": {
  "l2_throughput_pct": 21.8,
  "l2_sectors_pct": 9.4,
  "dram_throughput_pct": 1.4,
  "l2_hit_pct": 66.1,
  "dram_bytes_per_point": 14.0,
  "points_captured": 65536
 },
 "plain_fp32_2d_L8_T2^14_P2^16/simplex_raw/bwd": {
  "l2_throughput_pct": 16.6,
  "l2_sectors_pct": 7.9,
  "dram_throughput_pct": 4.9,
  "l2_hit_pct": 47.0,
  "dram_bytes_per_point": 150.1,
  "points_captured": 65536
 },
 "plain_fp32_2d_L8_T2^14_P2^16/simplex_equal_mem/fwd": {
  "l2_throughput_pct": 24.7,
  "l2_sectors_pct": 10.3,
  "dram_throughput_pct": 1.5,
  "l2_hit_pct": 69.5,
  "dram_bytes_per_point": 15.3,
  "points_captured": 65536
 },
 "plain_fp32_2d_L8_T2^14_P2^16/simplex_equal_mem/bwd": {
  "l2_throughput_pct": 16.2,
  "l2_sectors_pct": 7.7,
  "dram_throughput_pct": 4.7,
  "l2_hit_pct": 46.9,
  "dram_bytes_per_point": 151.4,
  "points_captured": 65536
 },
 "plain_fp32_2d_L8_T2^14_P2^16/grid/fwd": {
  "l2_throughput_pct": 24.9,
  "l2_sectors_pct": 10.3,
  "dram_throughput_pct": 1.4,
  "l2_hit_pct": 70.9,
  "dram_bytes_per_point": 14.9,
  "points_captured": 65536
 },
 "plain_fp32_2d_L8_T2^14_P2^16/grid/bwd": {
  "l2_throughput_pct": 20.7,
  "l2_sectors_pct": 9.2,
  "dram_throughput_pct": 4.8,
  "l2_hit_pct": 48.7,
  "dram_bytes_per_point": 151.0,
  "points_captured": 65536
 },
 "image_2d_L16_T2^22_fp16_P2^18/simplex_raw/fwd": {
  "l2_throughput_pct": 58.7,
  "l2_sectors_pct": 38.3,
  "dram_throughput_pct": 36.8,
  "l2_hit_pct": 51.4,
  "dram_bytes_per_point": 594.7,
  "points_captured": 262144
 },
 "image_2d_L16_T2^22_fp16_P2^18/simplex_raw/bwd": {
  "l2_throughput_pct": 23.6,
  "l2_sectors_pct": 11.9,
  "dram_throughput_pct": 33.2,
  "l2_hit_pct": 29.6,
  "dram_bytes_per_point": 1968.1,
  "points_captured": 262144
 },
 "image_2d_L16_T2^22_fp16_P2^18/simplex_equal_mem/fwd": {
  "l2_throughput_pct": 58.8,
  "l2_sectors_pct": 38.4,
  "dram_throughput_pct": 38.0,
  "l2_hit_pct": 51.0,
  "dram_bytes_per_point": 632.0,
  "points_captured": 262144
 },
 "image_2d_L16_T2^22_fp16_P2^18/simplex_equal_mem/bwd": {
  "l2_throughput_pct": 24.2,
  "l2_sectors_pct": 11.9,
  "dram_throughput_pct": 34.0,
  "l2_hit_pct": 28.9,
  "dram_bytes_per_point": 2062.9,
  "points_captured": 262144
 },
 "image_2d_L16_T2^22_fp16_P2^18/grid/fwd": {
  "l2_throughput_pct": 59.0,
  "l2_sectors_pct": 37.5,
  "dram_throughput_pct": 35.7,
  "l2_hit_pct": 52.1,
  "dram_bytes_per_point": 627.5,
  "points_captured": 262144
 },
 "image_2d_L16_T2^22_fp16_P2^18/grid/bwd": {
  "l2_throughput_pct": 26.6,
  "l2_sectors_pct": 12.6,
  "dram_throughput_pct": 32.1,
  "l2_hit_pct": 33.7,
  "dram_bytes_per_point": 2197.0,
  "points_captured": 262144
 },
 "sdf_3d_L16_T2^19_bf16_P2^20/simplex_raw/fwd": {
  "l2_throughput_pct": 64.6,
  "l2_sectors_pct": 23.4,
  "dram_throughput_pct": 3.6,
  "l2_hit_pct": 90.0,
  "dram_bytes_per_point": 54.5,
  "points_captured": 1048576
 },
 "sdf_3d_L16_T2^19_bf16_P2^20/simplex_raw/bwd": {
  "l2_throughput_pct": 70.9,
  "l2_sectors_pct": 25.7,
  "dram_throughput_pct": 11.5,
  "l2_hit_pct": 55.2,
  "dram_bytes_per_point": 329.8,
  "points_captured": 1048576
 },
 "sdf_3d_L16_T2^19_bf16_P2^20/simplex_equal_mem/fwd": {
  "l2_throughput_pct": 66.0,
  "l2_sectors_pct": 23.8,
  "dram_throughput_pct": 3.9,
  "l2_hit_pct": 90.3,
  "dram_bytes_per_point": 60.8,
  "points_captured": 1048576
 },
 "sdf_3d_L16_T2^19_bf16_P2^20/simplex_equal_mem/bwd": {
  "l2_throughput_pct": 76.7,
  "l2_sectors_pct": 27.0,
  "dram_throughput_pct": 7.2,
  "l2_hit_pct": 61.4,
  "dram_bytes_per_point": 193.8,
  "points_captured": 1048576
 },
 "sdf_3d_L16_T2^19_bf16_P2^20/grid/fwd": {
  "l2_throughput_pct": 65.1,
  "l2_sectors_pct": 22.8,
  "dram_throughput_pct": 2.2,
  "l2_hit_pct": 94.2,
  "dram_bytes_per_point": 59.3,
  "points_captured": 1048576
 },
 "sdf_3d_L16_T2^19_bf16_P2^20/grid/bwd": {
  "l2_throughput_pct": 74.1,
  "l2_sectors_pct": 25.9,
  "dram_throughput_pct": 6.3,
  "l2_hit_pct": 59.4,
  "dram_bytes_per_point": 335.5,
  "points_captured": 1048576
 },
 "volume_3d_L16_T2^19_fp16_2^16rays_x1024/simplex_raw/fwd": {
  "l2_throughput_pct": 58.3,
  "l2_sectors_pct": 21.0,
  "dram_throughput_pct": 5.4,
  "l2_hit_pct": 89.9,
  "dram_bytes_per_point": 70.7,
  "points_captured": 4194304
 },
 "volume_3d_L16_T2^19_fp16_2^16rays_x1024/simplex_raw/bwd": {
  "l2_throughput_pct": 63.9,
  "l2_sectors_pct": 23.1,
  "dram_throughput_pct": 9.4,
  "l2_hit_pct": 54.5,
  "dram_bytes_per_point": 293.1,
  "points_captured": 4194304
 },
 "volume_3d_L16_T2^19_fp16_2^16rays_x1024/simplex_equal_mem/fwd": {
  "l2_throughput_pct": 60.8,
  "l2_sectors_pct": 21.8,
  "dram_throughput_pct": 5.2,
  "l2_hit_pct": 90.8,
  "dram_bytes_per_point": 71.9,
  "points_captured": 4194304
 },
 "volume_3d_L16_T2^19_fp16_2^16rays_x1024/simplex_equal_mem/bwd": {
  "l2_throughput_pct": 77.8,
  "l2_sectors_pct": 27.3,
  "dram_throughput_pct": 5.9,
  "l2_hit_pct": 62.1,
  "dram_bytes_per_point": 153.7,
  "points_captured": 4194304
 },
 "volume_3d_L16_T2^19_fp16_2^16rays_x1024/grid/fwd": {
  "l2_throughput_pct": 60.3,
  "l2_sectors_pct": 21.1,
  "dram_throughput_pct": 3.3,
  "l2_hit_pct": 93.9,
  "dram_bytes_per_point": 71.8,
  "points_captured": 4194304
 },
 "volume_3d_L16_T2^19_fp16_2^16rays_x1024/grid/bwd": {
  "l2_throughput_pct": 76.0,
  "l2_sectors_pct": 26.5,
  "dram_throughput_pct": 5.9,
  "l2_hit_pct": 58.1,
  "dram_bytes_per_point": 297.8,
  "points_captured": 4194304
 }
}


def _sources_sha(files=("encode.cu", "encode_common.cuh", "lattice.cuh")):
    import hashlib
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2311_15439_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _config_points(dev, ea, P, pts):
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.render import vr_samples
    if pts == "uniform":
        return torch.from_numpy(synth.uniform_points(P, ea["d"], 78)).to(dev)
    if pts == "sdf":
        return torch.from_numpy(synth.sdf_points(P, 79)).to(dev)
    rays = [torch.from_numpy(a).to(dev) for a in synth.camera_rays(1 << 16, 60)]
    return vr_samples(*rays, P >> 16)[0]


def encode_bytes_per_point(ea, kind, tdt, odt):
    """Algorithmic bytes per point of the forward (point, one table entry per vertex and level, the
    encoding) and of the backward (point, dL/d(encoding) in binary32, one binary32 read-modify-write
    of each vertex's F gradients)."""
    d, L, F = ea["d"], ea["n_levels"], ea["n_features"]
    V = d + 1 if kind == "simplex" else 1 << d
    es = {"f32": 4, "f16": 2, "bf16": 2}
    return (4 * d + L * V * F * es[tdt] + L * F * es[odt], 4 * d + 4 * L * F + 2 * L * V * F * 4)


def per_config_encode(dev):
    """Per configuration: encode forward and backward points/s (each recorded once into a CUDA graph
    and replayed), for the simplex encoder in both res_modes and the 2^d grid on the same tables
    and points; each stage's algorithmic bytes over its time against the measured HBM copy peak,
    and the ncu L2 / DRAM throughput of the same kernels where the committed capture matches."""
    import torch
    from paper_2311_15439_gb300.api import Encoder
    dts = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    hbm, _ = _peaks()
    ncu_ok = ENCODE_NCU_SHA is not None and _sources_sha() == ENCODE_NCU_SHA
    gen = torch.Generator(device=dev).manual_seed(77)
    out = {}

    def graph_time(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        g.replay()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record()
        for _ in range(reps):
            g.replay()
        b.record()
        torch.cuda.synchronize(dev)
        del g
        return a.elapsed_time(b) / reps / 1e3

    for name, ea, tdt, P, pts in PER_CONFIG:
        x = _config_points(dev, ea, P, pts)
        n_out = ea["n_levels"] * ea["n_features"]
        dout = torch.randn((P, n_out), device=dev, generator=gen)
        reps = 1000 if P <= (1 << 16) else (3 if P >= (1 << 26) else 50)
        row = {"points": P, "table_dtype": tdt, "replays": reps}
        tab = None
        for kind, mode in VARIANTS:
            enc = Encoder(**ea, kind=kind, res_mode=mode, table_dtype=tdt, out_dtype=tdt)
            if tab is None:                        # the same tables for every encoder
                tab = (torch.rand(enc.table_shape(), device=dev, generator=gen) * 2 - 1).to(dts[tdt])
            grad = torch.zeros(enc.table_shape(), dtype=torch.float32, device=dev)
            o = torch.empty((P, n_out), dtype=dts[tdt], device=dev)
            tf = graph_time(lambda: enc.encode_fwd(x, tab, o), reps)
            tb = graph_time(lambda: enc.encode_bwd(x, dout, grad), reps)
            bf, bb = encode_bytes_per_point(ea, kind, tdt, tdt)
            rec = {"res_mode": mode, "fwd_bwd_points_per_s": P / (tf + tb), "fwd_ms": tf * 1e3, "bwd_ms": tb * 1e3,
                   "fwd_bytes_per_point": bf, "bwd_bytes_per_point": bb,
                   "fwd_hbm_frac": P * bf / tf / 1e9 / hbm, "bwd_hbm_frac": P * bb / tb / 1e9 / hbm}
            v = vname(kind, mode)
            if ncu_ok:
                for stage in ("fwd", "bwd"):
                    c = ENCODE_NCU.get("%s/%s/%s" % (name, v, stage))
                    if c:
                        rec["%s_ncu" % stage] = c
            row[v] = rec
            if kind == "simplex" and mode == "raw" and tdt == "f32":
                tpf = graph_time(lambda: enc.encode_plain_fwd(x, tab, o), reps)
                tpb = graph_time(lambda: enc.encode_plain_bwd(x, dout, grad), reps)
                row["simplex_plain_f32"] = {"res_mode": "raw", "fwd_bwd_points_per_s": P / (tpf + tpb),
                                            "fwd_ms": tpf * 1e3, "bwd_ms": tpb * 1e3}
            del enc, grad, o
        for m in ("raw", "equal_mem"):
            row["grid_over_simplex_time_" + m] = (row[vname("simplex", m)]["fwd_bwd_points_per_s"]
                                                  / row["grid"]["fwd_bwd_points_per_s"])
        out[name] = row
        del x, dout, tab
        torch.cuda.empty_cache()
    out["ceiling"] = ("fwd/bwd_hbm_frac: algorithmic bytes / time / measured HBM copy peak (%.1f GB/s); "
                      "*_ncu: ncu L2 sector and DRAM throughput as %% of peak, L2 hit rate, DRAM bytes per point "
                      "(%s)" % (hbm, "capture matches these sources" if ncu_ok else "no capture of these sources"))
    return out


def profile_mlp(dev, kernel):
    """Three launches of the image workload's network training pass (32 -> 64 -> 64 -> 3 fp16, L2
    loss, 2^18 points) on ``kernel``, for a one-kernel ncu capture (about 60 MB on the device)."""
    import torch
    from paper_2311_15439_gb300 import _lib, synth
    from paper_2311_15439_gb300.api import Mlp
    from paper_2311_15439_gb300.trainer import default_loss_scale
    _lib.check(_lib.lib().sxe_mlp_set_kernel(kernel), "sxe_mlp_set_kernel")
    mlp = Mlp(32, N_OUT, n_hidden=2, dtype="f16")
    W = torch.from_numpy(mlp.init_weights(1)).to(dev).half()
    x = torch.from_numpy(synth.rng(2).uniform(-1, 1, size=(BATCH, 32)).astype(np.float32)).to(dev).half()
    t = torch.from_numpy(synth.rng(3).random((BATCH, N_OUT)).astype(np.float32)).to(dev)
    dW = torch.zeros((mlp.n_params,), device=dev)
    din = torch.empty((BATCH, 32), device=dev)
    sq = torch.zeros((1,), device=dev)
    ws = mlp.workspace(BATCH, dev)
    for _ in range(3):
        mlp.mlp_train_l2(W, x, t, dW, sq, din=din, loss_scale=default_loss_scale(BATCH, N_OUT), workspace=ws)
    torch.cuda.synchronize(dev)
    print("network training pass x3 done, kernel %d" % kernel)


def profile_encode(dev):
    """One forward and one backward launch of every configuration and encoder of
    ``per_config_encode`` (the volumetric configuration at 2^16 rays x 64 samples, so that the
    capture holds a few GB), for an ncu capture of the encoding kernels; prints each launch's key."""
    import torch
    from paper_2311_15439_gb300.api import Encoder
    dts = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    gen = torch.Generator(device=dev).manual_seed(77)
    for name, ea, tdt, P, pts in PER_CONFIG:
        P = min(P, 1 << 22)
        x = _config_points(dev, ea, P, pts)
        n_out = ea["n_levels"] * ea["n_features"]
        dout = torch.randn((P, n_out), device=dev, generator=gen)
        tab = None
        for kind, mode in VARIANTS:
            enc = Encoder(**ea, kind=kind, res_mode=mode, table_dtype=tdt, out_dtype=tdt)
            if tab is None:
                tab = (torch.rand(enc.table_shape(), device=dev, generator=gen) * 2 - 1).to(dts[tdt])
            grad = torch.zeros(enc.table_shape(), dtype=torch.float32, device=dev)
            o = torch.empty((P, n_out), dtype=dts[tdt], device=dev)
            enc.encode_fwd(x, tab, o)
            nb = enc.bwd_kernel_count(P)
            enc.encode_bwd(x, dout, grad)
            torch.cuda.synchronize(dev)
            print("launch %s/%s fwd 1, bwd %s points %d" % (name, vname(kind, mode), nb, P), flush=True)
        del x, dout, tab
        torch.cuda.empty_cache()


def _replayed_step_ms(tr, xd, td, steps, warmup):
    """Time per step of ``steps`` replays of recorded training steps (one recording per resident
    batch, cycled; no timing events inside), after ``warmup`` eager steps."""
    import torch
    for i in range(warmup):
        tr.step(xd[i % len(xd)], td[i % len(td)])
    recs = []
    for i in range(len(xd)):
        tr.capture(xd[i], td[i], warmup=0)
        recs.append(tr.graph)
    for g in recs:                       # first launches outside the timed span
        tr.t += 1
        g.replay()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for i in range(steps):
        tr.t += 1
        recs[i % len(recs)].replay()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def image_step_variants(dev, xd, td, steps=100, warmup=5):
    """The headline training step with the simplex encoder in both res_modes and with the 2^d grid
    encoder (same L, F, T, table layout, network and batches), each timed the same way (replays of
    recorded steps without timing events): the comparison of Sec. 6.1's image-fitting run time, per
    res_mode of the simplex side."""
    import torch
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import Trainer
    out = {"timing": "%d replays of recorded steps per encoder (8 recordings, one per resident batch, cycled), "
                     "no timing events inside" % steps}
    for kind, mode in VARIANTS:
        enc = Encoder(**CFG, kind=kind, res_mode=mode, table_dtype="f16")
        tr = Trainer(enc, Mlp(CFG["n_levels"] * CFG["n_features"], N_OUT, n_hidden=2, dtype="f16"), BATCH, seed=0,
                     device=dev, table_layout="records")
        ms = _replayed_step_ms(tr, xd, td, steps, warmup)
        out[vname(kind, mode)] = {"res_mode": mode, "ms_per_step": ms, "points_per_s": BATCH / (ms / 1e3),
                                  "steps": steps}
        del tr
        torch.cuda.empty_cache()
    for m in ("raw", "equal_mem"):
        out["grid_over_simplex_time_" + m] = out["grid"]["ms_per_step"] / out[vname("simplex", m)]["ms_per_step"]
    return out


def _train_fixed_steps(dev, tr, steps, make_batch, chunk=100):
    """``steps`` eager training steps on batches made on the device ``chunk`` at a time outside the
    timed part; returns the summed CUDA-event time of the steps (s)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    total = 0.0
    for c0 in range(0, steps, chunk):
        batches = [make_batch() for _ in range(min(chunk, steps - c0))]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        for x, t in batches:
            tr.step(x, t)
        b.record(stream)
        torch.cuda.synchronize(dev)
        total += a.elapsed_time(b) / 1e3
        del batches
    return total


def _predict(tr, x):
    """The trained field at points x (device float32 [P, d]): encoding, then the network forward."""
    enc = tr.enc.encode_fwd(x, tr.tables)
    return tr.mlp.mlp_fwd(tr.W_lowp, enc)


def fit_quality(dev, image_steps=5000, sdf_steps=2000, repeats=5):
    """Quality at equal table size (Sec. 6.1): the image workload (L=16, F=2, T=2^22 fp16, network
    32-64-64-3, 2^18 points per step, Adam) trained for ``image_steps`` steps with each encoder, and
    the PSNR of its prediction (clipped to [0, 1]) over 2^18 held-out pixel centres against the FP64
    image; the SDF-style workload (d=3, T=2^19 bf16, network 32-64-1, 2^20 points per step) trained
    for ``sdf_steps`` steps, and its mean squared SDF error on 2^18 held-out points of the same
    distribution (half uniform, half within 0.01 of the surface).  Training batches are drawn on
    the device by torch from seeded generators; the step time excludes drawing them.  Each fit runs
    ``repeats`` times with different batch seeds (the same initial tables and network): the table
    gradients are summed by atomics in no fixed order, so runs diverge, and the final error of one
    run spreads by several dB; the record gives the median and the range."""
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import Trainer
    out = {}
    img = synth.ProceduralImage(seed=7, size=16384, n_waves=64)
    x_eval = synth.uniform_points(1 << 18, 2, 4242)
    t_eval = img.sample(x_eval).astype(np.float64)
    xe = torch.from_numpy(x_eval).to(dev)
    res = {"steps": image_steps, "points_per_step": BATCH, "eval_pixels": 1 << 18,
           "config": "d=2 L=16 F=2 T=2^22 fp16 base 16 growth 2.0, network 32-64-64-3 fp16"}
    for kind, mode in VARIANTS:
        runs = []
        for rep in range(repeats):
            enc = Encoder(**CFG, kind=kind, res_mode=mode, table_dtype="f16")
            tr = Trainer(enc, Mlp(32, N_OUT, n_hidden=2, dtype="f16"), BATCH, seed=0, device=dev,
                         table_layout="records")
            gen = torch.Generator(device=dev).manual_seed(2024 + rep)

            def batch():
                x = torch.rand((BATCH, 2), generator=gen, device=dev)
                return x, img.sample_torch(x)
            sec = _train_fixed_steps(dev, tr, image_steps, batch)
            y = np.clip(_predict(tr, xe).cpu().numpy().astype(np.float64), 0.0, 1.0)
            mse = float(np.mean((y - t_eval) ** 2))
            runs.append((10.0 * math.log10(1.0 / mse), sec, tr.loss()))
            del tr
            torch.cuda.empty_cache()
        psnr = [r[0] for r in runs]
        res[vname(kind, mode)] = {"res_mode": mode, "psnr_db": float(np.median(psnr)),
                                  "psnr_db_min": min(psnr), "psnr_db_max": max(psnr), "runs": repeats,
                                  "train_s": float(np.median([r[1] for r in runs])),
                                  "final_batch_loss": float(np.median([r[2] for r in runs]))}
    out["image"] = res
    scene = synth.SphereTorusScene(5)
    xs_eval = scene.sample(1 << 18, 4343)
    s_eval = scene.sdf(xs_eval).astype(np.float64)
    xse = torch.from_numpy(xs_eval).to(dev)
    P = 1 << 20
    res = {"steps": sdf_steps, "points_per_step": P, "eval_points": 1 << 18,
           "config": "d=3 L=16 F=2 T=2^19 bf16 base 16 growth 1.38, network 32-64-1 bf16"}
    for kind, mode in VARIANTS:
        runs = []
        for rep in range(repeats):
            enc = Encoder(3, 16, 2, 19, 16.0, 1.38, kind=kind, res_mode=mode, table_dtype="bf16")
            tr = Trainer(enc, Mlp(32, 1, n_hidden=1, dtype="bf16"), P, seed=6, device=dev)
            gen = torch.Generator(device=dev).manual_seed(2025 + rep)

            def batch():
                x = scene.sample_torch(P, gen)
                return x, scene.sdf_torch(x)
            sec = _train_fixed_steps(dev, tr, sdf_steps, batch)
            err = _predict(tr, xse).cpu().numpy().astype(np.float64) - s_eval
            near = np.abs(s_eval[:, 0]) < 0.01
            runs.append((float(np.mean(err ** 2)), float(np.mean(np.abs(err[near]))), sec, tr.loss()))
            del tr
            torch.cuda.empty_cache()
        mse = [r[0] for r in runs]
        res[vname(kind, mode)] = {"res_mode": mode, "eval_mse": float(np.median(mse)), "eval_mse_min": min(mse),
                                  "eval_mse_max": max(mse), "runs": repeats,
                                  "eval_mae_near_surface": float(np.median([r[1] for r in runs])),
                                  "train_s": float(np.median([r[2] for r in runs])),
                                  "final_batch_loss": float(np.median([r[3] for r in runs]))}
    out["sdf"] = res
    return out


def sdf_train(dev, P=1 << 20, steps=20, warmup=3, n_batches=4):
    """SDF-style training step (d = 3, L = 16, F = 2, T = 2^19 bf16 tables, network 32-64-1 bf16,
    2^20 points: half uniform in the unit cube, half within 0.01 of a seeded union of 32 spheres
    and tori, target their signed distance), Trainer with the table layout its size selects;
    simplex and the 8-corner grid, points/s."""
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import Trainer
    scene = synth.SphereTorusScene(5)
    xs = [synth.sdf_points(P, 300 + i) for i in range(n_batches)]
    batches = [(torch.from_numpy(x).to(dev), torch.from_numpy(scene.sdf(x)).to(dev)) for x in xs]
    out = {"points_per_step": P, "config": "d=3 L=16 F=2 T=2^19 bf16, network 32-64-1 bf16"}
    for kind, mode in VARIANTS:
        tr = Trainer(Encoder(3, 16, 2, 19, 16.0, 1.38, kind=kind, res_mode=mode, table_dtype="bf16"),
                     Mlp(32, 1, n_hidden=1, dtype="bf16"), P, seed=6, device=dev)
        for i in range(warmup):
            tr.step(*batches[i % n_batches])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record()
        for i in range(steps):
            tr.step(*batches[i % n_batches])
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / steps
        out[vname(kind, mode)] = {"res_mode": mode, "ms_per_step": ms, "points_per_s": P / (ms / 1e3),
                                  "table_layout": tr.tab.layout, "coarse_levels_on_second_stream": tr.tab.split_coarse,
                                  "loss": tr.loss()}
        del tr
        torch.cuda.empty_cache()
    for m in ("raw", "equal_mem"):
        out["grid_over_simplex_time_" + m] = out["grid"]["ms_per_step"] / out[vname("simplex", m)]["ms_per_step"]
    out["table_backward_roofline"] = dense_bwd_roofline(dev, xs[0])
    return out


def dense_bwd_roofline(dev, x_host, reps=20):
    """The SDF-style table backward of the levels that take the direct path, against the probe's
    rate of random float2 reductions over a footprint the size of the dense gradient array (which
    stays in L2): contributions / that rate over the CUDA-event time of the kernel."""
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.api import Encoder
    enc = Encoder(3, 16, 2, 19, 16.0, 1.38, table_dtype="bf16")
    P = x_host.shape[0]
    x = torch.from_numpy(x_host).to(dev)
    dout = torch.from_numpy(synth.normal_grads(P, enc.n_out, 301)).to(dev)
    grad = torch.zeros((enc.n_levels * enc.T, enc.n_features), dtype=torch.float32, device=dev)
    lc = enc.bwd_coarse_levels(P)
    st = torch.cuda.current_stream(dev).cuda_stream

    def timed(fn, n):
        for _ in range(3):
            fn(1)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        s.record()
        for r in range(n):
            fn(2 + r)
        e.record()
        torch.cuda.synchronize(dev)
        return s.elapsed_time(e) / n / 1e3

    sec = timed(lambda r: enc.encode_bwd(x, dout, grad, levels=(lc, enc.n_levels)), reps)
    n_ops, slots = 1 << 24, grad.numel() // 2
    sink = torch.zeros((1,), dtype=torch.float32, device=dev)
    probe_s = timed(lambda r: probe(0, grad.data_ptr(), slots, 2, n_ops, r, sink.data_ptr(), st), 5)
    contributions = P * (enc.n_levels - lc) * enc.n_vertices
    peak = n_ops / probe_s
    return {"kernel": "encode_bwd (levels %d-%d, dense binary32 gradient, %d MiB)" % (lc, enc.n_levels - 1,
                                                                                    grad.numel() * 4 >> 20),
            "contributions": contributions, "measured_ms": sec * 1e3, "achieved_ops_per_s": contributions / sec,
            "peak_ops_per_s": peak, "peak": "probe: random float2 reductions over the gradient array's footprint",
            "frac": contributions / sec / peak}


def serve_bench(dev, n_requests=800, rate_hz=1000.0, seed=5, repeats=3, sweep=(250.0, 500.0, 1000.0, 2000.0)):
    """Field queries of 4K..4M points (log-uniform), d uniform in 2..5, served by the continuous-
    batching loop (L=16, F=2, T=2^19, fp16): per encoder (simplex in both res_modes, 2^d grid)
    p50/p99 latency of ``repeats`` seeded Poisson runs at ``rate_hz`` (each run's figures and their
    median), p50/p99 at a rising offered rate, and the capacity: points/s of a closed-loop run in
    which every request of a stream is queued at once, so that the GPU never waits for arrivals."""
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.serve import FieldServer, NativeFieldServer, make_field, poisson_load, run_load
    sys.setswitchinterval(2e-4)          # let the scheduler thread take the GIL promptly
    dims = (2, 3, 4, 5)
    pools = {d: torch.from_numpy(synth.uniform_points(4 << 20, d, 900 + d)).pin_memory() for d in dims}
    out = {"load": "%d Poisson requests at %.0f/s per run, %d runs, sizes log-uniform 4K..4M points, d in {2,3,4,5}"
                   % (n_requests, rate_hz, repeats)}

    def one_run(srv, rate, n, s):
        arrivals, ds, sizes = poisson_load(rate, n, dims, 4096, 4 << 20, s)
        if rate == float("inf"):
            arrivals = np.zeros_like(arrivals)
        reqs, wall = run_load(srv, arrivals, ds, sizes, pools, s)
        lat = np.array([r.latency for r in reqs]) * 1e3
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "offered_points_per_s": float(sizes.sum() / arrivals[-1]) if arrivals[-1] > 0 else None,
                "served_points_per_s": float(sizes.sum() / wall),
                "errors": sum(r.error is not None for r in reqs)}

    for kind, mode in VARIANTS:
        fields = {d: make_field(d, kind=kind, res_mode=mode, seed=d, device=dev) for d in dims}
        srv = NativeFieldServer(fields, mem_budget_bytes=4 << 30, n_slots=4, max_batch_points=4 << 20,
                                device=dev).start()
        for d in dims:                   # warm-up: one request per d (allocator, pinned buffers, kernel load)
            if not srv.submit(d, pools[d][:65536]).wait(120.0):
                raise TimeoutError("serving warm-up request did not complete")
        runs = [one_run(srv, rate_hz, n_requests, seed + r) for r in range(repeats)]
        rising = {str(int(rt)): one_run(srv, rt, n_requests // 2, seed + 100 + k) for k, rt in enumerate(sweep)}
        closed = one_run(srv, float("inf"), n_requests, seed + 200)
        srv.stop()
        out[vname(kind, mode)] = {
            "res_mode": mode,
            "p50_ms": float(np.median([r["p50_ms"] for r in runs])),
            "p99_ms": float(np.median([r["p99_ms"] for r in runs])),
            "p50_ms_runs": [r["p50_ms"] for r in runs], "p99_ms_runs": [r["p99_ms"] for r in runs],
            "offered_points_per_s": float(np.median([r["offered_points_per_s"] for r in runs])),
            "capacity_points_per_s": closed["served_points_per_s"],
            "by_offered_rate_hz": rising, "batches": srv.n_batches,
            "errors": sum(r["errors"] for r in runs) + closed["errors"]}
        del srv, fields
        torch.cuda.empty_cache()
    for m in ("raw", "equal_mem"):
        out["simplex_over_grid_capacity_" + m] = (out[vname("simplex", m)]["capacity_points_per_s"]
                                                   / out["grid"]["capacity_points_per_s"])
    # the same load through the Python scheduler (simplex, raw), for comparison with the library's;
    # its forward passes on the kernel the library's loop takes (mma.sync) for the length of the run
    from paper_2311_15439_gb300 import _lib
    prev = _lib.lib().sxe_mlp_get_kernel()
    _lib.check(_lib.lib().sxe_mlp_set_kernel(_lib.SXE_MLP_KERNEL_MMA_SYNC), "sxe_mlp_set_kernel")
    try:
        fields = {d: make_field(d, seed=d, device=dev) for d in dims}
        srv = FieldServer(fields, mem_budget_bytes=4 << 30, n_slots=4, max_batch_points=4 << 20, device=dev).start()
        for d in dims:
            if not srv.submit(d, pools[d][:65536]).wait(120.0):
                raise TimeoutError("serving warm-up request did not complete")
        runs = [one_run(srv, rate_hz, n_requests, seed + r) for r in range(repeats)]
        srv.stop()
    finally:
        _lib.lib().sxe_mlp_set_kernel(prev)
    out["python_scheduler_simplex_raw"] = {"p50_ms": float(np.median([r["p50_ms"] for r in runs])),
                                           "p99_ms": float(np.median([r["p99_ms"] for r in runs]))}
    out["scheduler"] = ("library (sxe_server_*: C++ scheduler thread, 4 stream slots, batches of <= 2^20 points on "
                        "high-priority streams, host-callback completion; network forward on mma.sync); "
                        "python_scheduler_* is serve.FieldServer on the same kernels")
    return out


# ----------------------------------------------------------------------------------------
# CPU oracle arm (the reference of this benchmark)
# ----------------------------------------------------------------------------------------
def oracle_step(x, tgt, H, W, state, t):
    """One training step of the FP64 oracle: encode, network + L2 loss, backward, scatter,
    Adam on every table parameter (zero-gradient skip) and on the network."""
    from oracle import adam, encoding, mlp
    L, T, F = H.shape
    e = encoding.simplex_encode(x, H, base_res=CFG["base_res"], growth=CFG["growth"])
    y, acts = mlp.mlp_forward(W, e)
    loss, dy = mlp.l2_loss(y, tgt)
    dW, de = mlp.mlp_backward(W, acts, dy)
    g = encoding.simplex_encode_bwd(x, de, n_levels=L, log2_T=int(T).bit_length() - 1, n_features=F,
                                    base_res=CFG["base_res"], growth=CFG["growth"])
    hp = dict(lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15)
    for l in range(L):
        H[l], state["m"][l], state["v"][l] = adam.adam_step(H[l], g[l], state["m"][l], state["v"][l], t,
                                                            skip_zero_grad=True, **hp)
    for i in range(len(W)):
        W[i], state["mW"][i], state["vW"][i] = adam.adam_step(W[i], dW[i], state["mW"][i], state["vW"][i], t,
                                                              skip_zero_grad=False, **hp)
    return loss


# The same oracle step spread over host cores: a pool of worker processes (spawn) attached to the
# table, moment and gradient arrays in shared memory.  Phase 1 splits the points: each worker
# encodes its chunk, runs the network forward, the L2 loss and the backward (its loss gradient
# rescaled from its chunk's mean to the batch's); phase 2 splits the levels: each worker
# scatters dL/d(encoding) of all points into its levels of the gradient; phase 3 splits the table
# parameters: each worker runs Adam on its range.  Every phase calls the oracle's own functions.
_W = {}


def _shm_array(name, shape):
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=np.float64, buffer=shm.buf)


def _worker_init(names, shape):
    for key, name in names.items():
        _W[key] = _shm_array(name, shape)


def _w_points(x, tgt, W, P_total):
    from oracle import encoding, mlp
    H = _W["H"][1]
    e = encoding.simplex_encode(x, H, base_res=CFG["base_res"], growth=CFG["growth"])
    y, acts = mlp.mlp_forward(W, e)
    loss, dy = mlp.l2_loss(y, tgt)
    dy = dy * (x.shape[0] / P_total)                      # the batch mean's gradient
    dW, de = mlp.mlp_backward(W, acts, dy)
    return loss * x.shape[0], dW, de


def _w_levels(x, de, levels):
    from oracle import encoding
    H, g = _W["H"][1], _W["g"][1]
    L, T, F = H.shape
    grads = encoding.simplex_encode_bwd(x, de, n_levels=L, log2_T=int(T).bit_length() - 1, n_features=F,
                                        base_res=CFG["base_res"], growth=CFG["growth"], levels=levels)
    for l, gl in grads.items():
        g[l] = gl


def _w_adam(lo, hi, t):
    from oracle import adam
    H, m, v, g = (_W[k][1].reshape(-1) for k in ("H", "m", "v", "g"))
    H[lo:hi], m[lo:hi], v[lo:hi] = adam.adam_step(H[lo:hi], g[lo:hi], m[lo:hi], v[lo:hi], t, skip_zero_grad=True,
                                                  lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15)


class ParallelOracle:
    """The oracle's training step (encode, network + L2 loss, backward, scatter, Adam over every
    table parameter and the network) on ``n`` worker processes; the arrays of the full workload
    (L = 16, T = 2^22, F = 2, FP64) live in shared memory."""

    def __init__(self, n):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        from paper_2311_15439_gb300 import synth
        L, T, F = CFG["n_levels"], 1 << CFG["log2_T"], CFG["n_features"]
        self.shape, self.n = (L, T, F), n
        self.shm, self.arr = {}, {}
        for key in ("H", "m", "v", "g"):
            shm = shared_memory.SharedMemory(create=True, size=L * T * F * 8)
            self.shm[key] = shm
            self.arr[key] = np.ndarray(self.shape, dtype=np.float64, buffer=shm.buf)
            self.arr[key][:] = 0.0
        self.arr["H"][:] = synth.uniform_tables(L, T, F, 0, dtype="f32", scale=1e-4)[0]
        g = np.random.Generator(np.random.PCG64(1))
        self.W = [g.uniform(-math.sqrt(6 / fi), math.sqrt(6 / fi), size=(fo, fi)) for fo, fi in
                  [(64, 32), (64, 64), (3, 64)]]
        self.mW = [np.zeros_like(w) for w in self.W]
        self.vW = [np.zeros_like(w) for w in self.W]
        self.pool = mp.get_context("spawn").Pool(n, initializer=_worker_init,
                                                 initargs=({k: v.name for k, v in self.shm.items()}, self.shape))

    def step(self, x, tgt, t):
        from oracle import adam
        P, n = x.shape[0], self.n
        cuts = np.linspace(0, P, n + 1).astype(int)
        parts = self.pool.starmap(_w_points, [(x[a:b], tgt[a:b], self.W, P) for a, b in zip(cuts[:-1], cuts[1:])
                                              if b > a])
        loss = sum(p[0] for p in parts) / P
        dW = [sum(p[1][i] for p in parts) for i in range(len(self.W))]
        de = np.concatenate([p[2] for p in parts])
        L = self.shape[0]
        self.pool.starmap(_w_levels, [(x, de, list(range(k, L, n))) for k in range(min(n, L))])
        N = int(np.prod(self.shape))
        cuts = np.linspace(0, N, n + 1).astype(np.int64)
        self.pool.starmap(_w_adam, [(int(a), int(b), t) for a, b in zip(cuts[:-1], cuts[1:])])
        for i in range(len(self.W)):
            self.W[i], self.mW[i], self.vW[i] = adam.adam_step(self.W[i], dW[i], self.mW[i], self.vW[i], t,
                                                               skip_zero_grad=False, lr=1e-2, beta1=0.9, beta2=0.99,
                                                               eps=1e-15)
        return loss

    def close(self):
        self.pool.close()
        self.pool.join()
        for shm in self.shm.values():
            shm.close()
            shm.unlink()


def host_cores():
    """Host cores this process may run on (the count ``nproc`` prints)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle(sample_points, steps, seconds_cap, cores=1):
    """Points/s of the oracle's training step on ``sample_points``-point batches of the image
    workload (full tables), on one core (the plain oracle step) or ``cores`` worker processes."""
    from paper_2311_15439_gb300 import synth
    img = synth.ProceduralImage(seed=7, size=16384, n_waves=64)
    par = ParallelOracle(cores) if cores > 1 else None
    if par is None:
        L, T, F = CFG["n_levels"], 1 << CFG["log2_T"], CFG["n_features"]
        H = synth.uniform_tables(L, T, F, 0, dtype="f32", scale=1e-4)[0].astype(np.float64)
        g = np.random.Generator(np.random.PCG64(1))
        dims = [(64, 32), (64, 64), (3, 64)]
        W = [g.uniform(-math.sqrt(6 / fi), math.sqrt(6 / fi), size=(fo, fi)) for fo, fi in dims]
        state = {"m": np.zeros_like(H), "v": np.zeros_like(H), "mW": [np.zeros_like(w) for w in W],
                 "vW": [np.zeros_like(w) for w in W]}
    done, t0 = 0, time.perf_counter()
    times = []
    try:
        for k in range(steps):
            x = synth.uniform_points(sample_points, 2, 5000 + k)
            tgt = img.sample(x)
            s = time.perf_counter()
            if par is None:
                oracle_step(x, tgt, H, W, state, k + 1)
            else:
                par.step(x, tgt, k + 1)
            times.append(time.perf_counter() - s)
            done += 1
            if time.perf_counter() - t0 > seconds_cap:
                break
    finally:
        if par is not None:
            par.close()
    return sample_points * done / sum(times), done, times


def cpu_baseline_subprocess(seconds):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-only", "--cpu-seconds", str(seconds)]
    try:
        res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
        return json.loads(res.stdout.strip().splitlines()[-1])
    except Exception as exc:  # report, do not fail the GPU line
        return {"value": None, "error": repr(exc)[:200]}


def cpu_baseline_only(seconds):
    """The oracle's training step on all host cores (the reported value) and on one core, each
    for about ``seconds`` of wall time."""
    sample = 1 << 13
    n = host_cores()
    v1, d1, _ = time_oracle(sample, 1000, seconds / 2, cores=1)
    vn, dn, _ = time_oracle(sample, 1000, seconds / 2, cores=n) if n > 1 else (v1, d1, None)
    what = ("oracle steps of %d points each on the full workload tables (L=16, T=2^22, F=2; Adam over all "
            "134M table parameters)" % sample)
    print(json.dumps({"value": vn, "unit": "points/s", "cores": n, "kind": "oracle",
                      "sample": "%d %s, %d worker processes (points, levels and parameter ranges split)"
                                % (dn, what, n),
                      "single_core": {"value": v1, "cores": 1, "sample": "%d %s" % (d1, what)}}))


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")                     # one thread per worker process
    sample = 1 << 13
    n = host_cores()
    _, done, times = time_oracle(sample, args.warmup + args.steps, 1e9, cores=n)
    t = times[args.warmup:]
    value = sample * len(t) / sum(t)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
        "steps": len(t), "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": n, "kind": "oracle",
                         "sample": "%d-point steps of the full workload (tables L=16, T=2^22), %d worker processes"
                                   % (sample, n)},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kind", default="simplex", choices=["simplex", "grid"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-volume", action="store_true")
    ap.add_argument("--mlp-kernel", default="auto", choices=["auto", "mma_sync", "tcgen05", "tcgen05_pipelined", "tcgen05_3tile"],
                    help="kernel of the network training pass")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--split-batch", type=int, default=1,
                    help="parts of the step's batch: each part's table backward beside the next part's network pass")
    ap.add_argument("--quality-steps", type=int, default=5000,
                    help="training steps of the image quality runs (the SDF runs take 2/5 of it); 0 skips them")
    ap.add_argument("--profile-mlp", action="store_true",
                    help="three launches of the network training pass on --mlp-kernel (for an ncu capture)")
    ap.add_argument("--profile-encode", action="store_true",
                    help="one launch of each encoding kernel per configuration and encoder (for an ncu capture)")
    ap.add_argument("--cpu-baseline-only", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile_mlp:
        import torch
        from paper_2311_15439_gb300 import _lib
        from paper_2311_15439_gb300 import build as B
        B.build()
        profile_mlp(torch.device("cuda", 0), {"auto": _lib.SXE_MLP_KERNEL_AUTO, "mma_sync": _lib.SXE_MLP_KERNEL_MMA_SYNC,
                                              "tcgen05": _lib.SXE_MLP_KERNEL_TCGEN05,
                                              "tcgen05_pipelined": _lib.SXE_MLP_KERNEL_TCGEN05_PIPELINED,
                                              "tcgen05_3tile": _lib.SXE_MLP_KERNEL_TCGEN05_3TILE}[args.mlp_kernel])
    elif args.profile_encode:
        import torch
        from paper_2311_15439_gb300 import build as B
        B.build()
        profile_encode(torch.device("cuda", 0))
    elif args.cpu_baseline_only:
        cpu_baseline_only(args.cpu_seconds)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
