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
METRIC = "simplex encode fwd+bwd training-step throughput"
N_POOL = 8   # distinct resident batches cycled through the timed steps

# DRAM traffic of one step's launch of a stage (dram__bytes_read.sum + dram__bytes_write.sum of its
# kernels in one ncu capture of this workload), with the SHA-1 of the kernel sources it was taken
# on: the figure is reported only while those sources are unchanged.
TRAFFIC = {
    "encode_bwd": (35.82e6 + 755.55e6, "6db9b692110c81022350715653cfadf71ada9d02",
                   ("encode.cu", "encode_common.cuh", "sxe_internal.cuh")),
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
                                              "tcgen05": _lib.SXE_MLP_KERNEL_TCGEN05}[args.mlp_kernel]),
               "sxe_mlp_set_kernel")
    enc = Encoder(**CFG, kind=args.kind, table_dtype="f16")
    mlp = Mlp(CFG["n_levels"] * CFG["n_features"], N_OUT, n_hidden=2, dtype="f16")
    tr = Trainer(enc, mlp, BATCH, seed=rank, device=dev, table_layout="records")
    xs, ts = make_batches(N_POOL, seed0=1000 + 100 * rank)
    xd = [torch.from_numpy(x).to(dev) for x in xs]
    td = [torch.from_numpy(t).to(dev) for t in ts]
    stream = torch.cuda.current_stream(dev)

    for i in range(args.warmup):
        tr.step(xd[i % N_POOL], td[i % N_POOL])
    torch.cuda.synchronize(dev)

    # ---- device-timed region: K steps, per-stage events on the launching stream
    names = ["encode_fwd", "mlp_train_l2", "encode_bwd", "adam_tables", "adam_mlp"]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(args.steps)]
    F = enc.n_features
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        for k in range(args.steps):
            x, t = xd[k % N_POOL], td[k % N_POOL]
            e = ev[k]
            tr.t += 1
            tr.adam_tables.advance(tr.t_dev, tr.corrections)
            e[0].record(stream)
            tr.enc.encode_fwd(x, tr.tables, tr.enc_out)
            e[1].record(stream)
            tr.mlp.mlp_train_l2(tr.W_lowp, tr.enc_out, t, tr.dW, tr.sq_sum, din=tr.d_enc, loss_scale=tr.loss_scale,
                                workspace=tr.ws)
            e[2].record(stream)
            tr.enc.encode_bwd(x, tr.d_enc, tr.state, grad_stride=4 * F, grad_offset=3 * F, touched=tr.touched)
            e[3].record(stream)
            tr.adam_tables.step_touched_dev(tr.corrections, tr.state, tr.touched, tr.tables, F)
            e[4].record(stream)
            tr.adam_mlp.step_dev(tr.corrections, tr.W, tr.mW, tr.vW, tr.dW, lowp=tr.W_lowp)
            e[5].record(stream)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
    ms = start.elapsed_time(stop)
    per_kernel = {n: float(np.mean([ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps)]))
                  for i, n in enumerate(names)}
    ms = max_over_ranks(ms, world, dev)
    loss = tr.loss()
    n_touched, n_sectors = count_touched(tr, xd[0])

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
    grid_img = image_grid_step(dev, xd, td, ms / args.steps) if (rank == 0 and not args.no_sweep and
                                                                  args.kind == "simplex") else None
    per_cfg = per_config_encode(dev) if (rank == 0 and not args.no_sweep) else None

    if rank == 0:
        value = job_throughput(BATCH, args.steps, world, ms)
        work = _stage_work(n_touched)
        dom = max(work, key=lambda n: per_kernel[n])
        bound, amount = work[dom]
        hbm_peak, peak_src = _peaks()
        if bound == "hbm":
            achieved = amount / (per_kernel[dom] / 1e3) / 1e9
            peak, unit = hbm_peak, "GB/s"
        else:
            achieved = amount / (per_kernel[dom] / 1e3) / 1e12
            peak, unit = _tensor_peak(), "TFLOP/s"
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "kind": args.kind, "mlp_kernel": {"auto": "auto (two-tile tcgen05 kernel for this network)", "mma_sync": "mma_sync",
                                      "tcgen05": "tcgen05"}[args.mlp_kernel],
                       "global_batch": BATCH * world,
                       "points_per_step_per_gpu": BATCH, "parallelism": "replicas (one per GPU)",
                       "l2": "working set > L2: 256 MiB fp16 tables + 2 GiB fp32 table state records, no flush",
                       "batches": "%d resident distinct batches cycled" % N_POOL},
            "e2e": {"value": job_throughput(BATCH, e2e_steps, world, ms_e2e), "unit": "points/s",
                    "h2d_bytes_per_step": BATCH * (2 + N_OUT) * 4, "d2h_bytes_per_step": 4,
                    "api": "trainer.HostFeed.step (double-buffered copies on a copy stream, recorded step "
                           "replayed, loss read one step behind)"},
            "roofline": {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                         "frac": achieved / peak, "traffic": _traffic(dom), "peak_source": peak_src,
                         "work_per_step": amount, "touched_entries_per_step": n_touched},
            "per_kernel_ms": per_kernel,
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
        gathers = contrib
        pred_fwd = n_sectors / peaks_ra["gather_4B_table"] + (gathers - n_sectors) / peaks_ra["gather_4B_l2"]
        line["gather_roofline"] = {
            "kernel": "encode_fwd", "gathers": gathers, "table_sectors_touched": n_sectors,
            "achieved_gathers_per_s": gathers / (per_kernel["encode_fwd"] / 1e3),
            "achieved_over_random_gather_peak": gathers / (per_kernel["encode_fwd"] / 1e3) / peaks_ra["gather_4B_table"],
            "predicted_ms": pred_fwd * 1e3, "measured_ms": per_kernel["encode_fwd"],
            "frac": pred_fwd * 1e3 / per_kernel["encode_fwd"],
            "model": "first gather from a 32-byte table sector = one random 4-byte gather missing L2 "
                     "(probe over the fp16 tables); later ones hit (probe over 8 MiB)"}
        if comparators is not None:
            line["comparators"] = comparators
        if volume is not None:
            line["volume"] = volume
        if sdf is not None:
            line["sdf_train"] = sdf
        if grid_img is not None:
            line["image_grid_step"] = grid_img
        if per_cfg is not None:
            line["per_config_encode"] = per_cfg
        if serving is not None:
            line["serve"] = serving
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline_subprocess(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def encode_sweep(dev, reps=20):
    """Encode forward+backward points/s of the simplex encoder vs the 2^d grid at d = 2..5
    (L = 16, F = 2, T = 2^19, fp16 tables, 2^20 points), and the binary32 path."""
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.api import Encoder
    P = 1 << 20
    out = {}
    for d in (2, 3, 4, 5):
        x = torch.from_numpy(synth.uniform_points(P, d, 50 + d)).to(dev)
        dout = torch.randn((P, 32), device=dev)
        row = {}
        for kind, tdt in (("simplex", "f16"), ("grid", "f16"), ("simplex", "f32")):
            enc = Encoder(d, 16, 2, 19, 16.0, 1.38, kind=kind, table_dtype=tdt, out_dtype=tdt)
            tab = torch.zeros(enc.table_shape(), dtype=torch.float16 if tdt == "f16" else torch.float32, device=dev)
            grad = torch.zeros(enc.table_shape(), dtype=torch.float32, device=dev)
            o = torch.empty((P, 32), dtype=tab.dtype, device=dev)
            for _ in range(3):
                enc.encode_fwd(x, tab, o)
                enc.encode_bwd(x, dout, grad)
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            s.record()
            for _ in range(reps):
                enc.encode_fwd(x, tab, o)
                enc.encode_bwd(x, dout, grad)
            e.record()
            torch.cuda.synchronize(dev)
            row["%s_%s" % (kind, tdt)] = P * reps / (s.elapsed_time(e) / 1e3)
            if kind == "simplex" and tdt == "f32":       # the plain binary32 path on the same tables
                for _ in range(2):
                    enc.encode_plain_fwd(x, tab, o)
                    enc.encode_plain_bwd(x, dout, grad)
                torch.cuda.synchronize(dev)
                s.record()
                for _ in range(reps):
                    enc.encode_plain_fwd(x, tab, o)
                    enc.encode_plain_bwd(x, dout, grad)
                e.record()
                torch.cuda.synchronize(dev)
                row["simplex_plain_f32"] = P * reps / (s.elapsed_time(e) / 1e3)
        out["d%d" % d] = row
    return {"encode_fwd_bwd_points_per_s": out, "config": "L=16 F=2 T=2^19 base 16 growth 1.38, 2^20 points"}


def random_access_peaks(dev, state_bytes, table, n_ops=1 << 24, reps=5):
    """Peak rates of the scattered patterns that bound the table kernels, measured on this GPU
    with the library's probe: float2 reductions into random 32-byte records of a footprint the
    size of the table state (L2 misses) and of 8 MiB (L2 hits), and 4-byte gathers from the
    fp16 tables.  Returns ops/s."""
    import torch
    from paper_2311_15439_gb300 import _lib as L
    lib = L.lib()
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
    for kind in ("simplex", "grid"):
        enc = Encoder(3, 16, 2, 19, 16.0, 1.38, kind=kind, table_dtype="f16")
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
            res.setdefault(str(S), {})[kind] = {"render_ms": ev[0].elapsed_time(ev[1]) / reps,
                                                "encode_ms": ev[2].elapsed_time(ev[3]) / reps}
            del rr
            torch.cuda.empty_cache()
    for S, r in res.items():
        r["grid_over_simplex_render"] = r["grid"]["render_ms"] / r["simplex"]["render_ms"]
        r["grid_over_simplex_encode"] = r["grid"]["encode_ms"] / r["simplex"]["encode_ms"]
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
    for kind in ("simplex", "grid"):
        enc = Encoder(3, 16, 2, 19, 16.0, 1.38, kind=kind, table_dtype="f16")
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
        out[kind] = {"ms_per_step": ms, "samples_per_s": R * S / (ms / 1e3), "table_layout": vt.tab.layout,
                     "coarse_levels_on_second_stream": vt.tab.split_coarse}
        del vt
        torch.cuda.empty_cache()
    out["grid_over_simplex"] = out["grid"]["ms_per_step"] / out["simplex"]["ms_per_step"]
    return out


# Encode forward + backward of each configuration of the benchmark plan (the plain binary32 case,
# the image, SDF-style and volumetric workloads; the serving load is `serve`), simplex and grid.
PER_CONFIG = [
    ("plain_fp32_2d_L8_T2^14_P2^16", dict(d=2, n_levels=8, n_features=2, log2_T=14, base_res=16.0, growth=1.5),
     "f32", 1 << 16, "uniform"),
    ("image_2d_L16_T2^22_fp16_P2^18", dict(CFG), "f16", 1 << 18, "uniform"),
    ("sdf_3d_L16_T2^19_bf16_P2^20", dict(d=3, n_levels=16, n_features=2, log2_T=19, base_res=16.0, growth=1.38),
     "bf16", 1 << 20, "sdf"),
    ("volume_3d_L16_T2^19_fp16_2^16rays_x1024", dict(d=3, n_levels=16, n_features=2, log2_T=19, base_res=16.0,
                                                      growth=1.38), "f16", 1 << 26, "rays"),
]


def per_config_encode(dev):
    """Per configuration: encode forward and backward points/s (each recorded once into a CUDA graph
    and replayed), simplex and grid on the same tables, and the forward's achieved random gathers/s
    over the probe's random 4-byte gather rate on that configuration's own tables (the fraction of
    the gather roofline; above 1 where tables or reuse sit in L2)."""
    import torch
    from paper_2311_15439_gb300 import _lib as L
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.api import Encoder
    from paper_2311_15439_gb300.render import vr_samples
    lib = L.lib()
    st = torch.cuda.current_stream(dev).cuda_stream
    sink = torch.zeros((1,), dtype=torch.float32, device=dev)
    dts = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    gen = torch.Generator(device=dev).manual_seed(77)
    out = {}
    for name, ea, tdt, P, pts in PER_CONFIG:
        if pts == "uniform":
            x = torch.from_numpy(synth.uniform_points(P, ea["d"], 78)).to(dev)
        elif pts == "sdf":
            x = torch.from_numpy(synth.sdf_points(P, 79)).to(dev)
        else:
            rays = [torch.from_numpy(a).to(dev) for a in synth.camera_rays(1 << 16, 60)]
            x = vr_samples(*rays, P >> 16)[0]
        n_out = ea["n_levels"] * ea["n_features"]
        dout = torch.randn((P, n_out), device=dev, generator=gen)
        reps = 1000 if P <= (1 << 16) else (3 if P >= (1 << 26) else 50)
        row = {"points": P, "table_dtype": tdt, "replays": reps}
        for kind in ("simplex", "grid"):
            enc = Encoder(**ea, kind=kind, table_dtype=tdt, out_dtype=tdt)
            tab = (torch.rand(enc.table_shape(), device=dev, generator=gen) * 2 - 1).to(dts[tdt])
            grad = torch.zeros(enc.table_shape(), dtype=torch.float32, device=dev)
            o = torch.empty((P, n_out), dtype=dts[tdt], device=dev)
            times = {}
            for stage, fn in (("fwd", lambda: enc.encode_fwd(x, tab, o)), ("bwd", lambda: enc.encode_bwd(x, dout, grad))):
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
                times[stage] = a.elapsed_time(b) / reps / 1e3
                del g
            gathers = P * ea["n_levels"] * enc.n_vertices
            words = tab.view(torch.float32).reshape(-1) if tab.element_size() == 4 else tab.view(torch.float32)
            slots = 1 << int(math.log2(words.numel() // 2))
            n_ops = 1 << 24
            probe(1, words.data_ptr(), slots, 2, n_ops, 1, sink.data_ptr(), st)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for r in range(3):
                probe(1, words.data_ptr(), slots, 2, n_ops, 2 + r, sink.data_ptr(), st)
            b.record()
            torch.cuda.synchronize(dev)
            peak = 3 * n_ops / (a.elapsed_time(b) / 1e3)
            row[kind] = {"fwd_bwd_points_per_s": P / (times["fwd"] + times["bwd"]),
                         "fwd_ms": times["fwd"] * 1e3, "bwd_ms": times["bwd"] * 1e3,
                         "fwd_gathers_per_s": gathers / times["fwd"], "random_gather_peak_per_s": peak,
                         "gather_roofline_frac": gathers / times["fwd"] / peak}
            if kind == "simplex" and tdt == "f32":
                times_p = {}
                for stage, fn in (("fwd", lambda: enc.encode_plain_fwd(x, tab, o)),
                                  ("bwd", lambda: enc.encode_plain_bwd(x, dout, grad))):
                    fn()
                    torch.cuda.synchronize(dev)
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g):
                        fn()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize(dev)
                    a.record()
                    for _ in range(reps):
                        g.replay()
                    b.record()
                    torch.cuda.synchronize(dev)
                    times_p[stage] = a.elapsed_time(b) / reps / 1e3
                    del g
                row["simplex_plain_f32"] = {"fwd_bwd_points_per_s": P / (times_p["fwd"] + times_p["bwd"])}
            del enc, tab, grad, o
        row["grid_over_simplex"] = row["simplex"]["fwd_bwd_points_per_s"] / row["grid"]["fwd_bwd_points_per_s"]
        out[name] = row
        del x, dout
        torch.cuda.empty_cache()
    return out


def image_grid_step(dev, xd, td, simplex_ms, steps=100, warmup=5):
    """The headline training step with the 2^d grid encoder instead of the simplex one (same
    L, F, T, tables, network, batches): the comparison of Sec. 6.1's image-fitting run time."""
    import torch
    from paper_2311_15439_gb300.api import Encoder, Mlp
    from paper_2311_15439_gb300.trainer import Trainer
    enc = Encoder(**CFG, kind="grid", table_dtype="f16")
    tr = Trainer(enc, Mlp(CFG["n_levels"] * CFG["n_features"], N_OUT, n_hidden=2, dtype="f16"), BATCH, seed=0,
                 device=dev, table_layout="records")
    for i in range(warmup):
        tr.step(xd[i % len(xd)], td[i % len(td)])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    a.record()
    for i in range(steps):
        tr.step(xd[i % len(xd)], td[i % len(td)])
    b.record()
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    del tr
    torch.cuda.empty_cache()
    return {"grid_ms_per_step": ms, "grid_points_per_s": BATCH / (ms / 1e3), "simplex_ms_per_step": simplex_ms,
            "grid_over_simplex": ms / simplex_ms, "steps": steps,
            "note": "grid: 4 corners per level against the simplex's 3 vertices, same tables and network"}


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
    for kind in ("simplex", "grid"):
        tr = Trainer(Encoder(3, 16, 2, 19, 16.0, 1.38, kind=kind, table_dtype="bf16"),
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
        out[kind] = {"ms_per_step": ms, "points_per_s": P / (ms / 1e3), "table_layout": tr.tab.layout,
                     "coarse_levels_on_second_stream": tr.tab.split_coarse, "loss": tr.loss()}
        del tr
        torch.cuda.empty_cache()
    out["grid_over_simplex"] = out["grid"]["ms_per_step"] / out["simplex"]["ms_per_step"]
    out["table_backward_roofline"] = dense_bwd_roofline(dev, xs[0])
    return out


def dense_bwd_roofline(dev, x_host, reps=20):
    """The SDF-style table backward of the levels that take the direct path, against the probe's
    rate of random float2 reductions over a footprint the size of the dense gradient array (which
    stays in L2): contributions / that rate over the CUDA-event time of the kernel."""
    import torch
    from paper_2311_15439_gb300 import _lib as L
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
    lib = L.lib()
    probe_s = timed(lambda r: probe(0, grad.data_ptr(), slots, 2, n_ops, r, sink.data_ptr(), st), 5)
    contributions = P * (enc.n_levels - lc) * enc.n_vertices
    peak = n_ops / probe_s
    return {"kernel": "encode_bwd (levels %d-%d, dense binary32 gradient, %d MiB)" % (lc, enc.n_levels - 1,
                                                                                    grad.numel() * 4 >> 20),
            "contributions": contributions, "measured_ms": sec * 1e3, "achieved_ops_per_s": contributions / sec,
            "peak_ops_per_s": peak, "peak": "probe: random float2 reductions over the gradient array's footprint",
            "frac": contributions / sec / peak}


def serve_bench(dev, n_requests=800, rate_hz=1000.0, seed=5):
    """Poisson-arriving field queries of 4K..4M points (log-uniform), d uniform in 2..5, served
    by the continuous-batching loop; simplex fields vs 2^d grid fields (L=16, F=2, T=2^19, fp16)."""
    import torch
    from paper_2311_15439_gb300 import synth
    from paper_2311_15439_gb300.serve import FieldServer, make_field, poisson_load, run_load
    sys.setswitchinterval(2e-4)          # let the scheduler thread take the GIL promptly
    arrivals, ds, sizes = poisson_load(rate_hz, n_requests, (2, 3, 4, 5), 4096, 4 << 20, seed)
    pools = {d: torch.from_numpy(synth.uniform_points(4 << 20, d, 900 + d)).pin_memory() for d in (2, 3, 4, 5)}
    out = {"load": "%d Poisson requests at %.0f/s, sizes log-uniform 4K..4M points, d in {2,3,4,5}" % (n_requests, rate_hz)}
    for kind in ("simplex", "grid"):
        fields = {d: make_field(d, kind=kind, seed=d, device=dev) for d in (2, 3, 4, 5)}
        srv = FieldServer(fields, mem_budget_bytes=4 << 30, n_slots=4, max_batch_points=4 << 20, device=dev).start()
        # warm-up: one request per d (allocator, pinned buffers, kernel load)
        for d in (2, 3, 4, 5):
            if not srv.submit(d, pools[d][:65536]).wait(120.0):
                raise TimeoutError("serving warm-up request did not complete")
        reqs, wall = run_load(srv, arrivals, ds, sizes, pools, seed)
        srv.stop()
        lat = np.array([r.latency for r in reqs]) * 1e3
        out[kind] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "points_per_s": float(sizes.sum() / wall), "batches": srv.n_batches,
                     "errors": sum(r.error is not None for r in reqs)}
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


def time_oracle(sample_points, steps, seconds_cap):
    from paper_2311_15439_gb300 import synth
    L, T, F = CFG["n_levels"], 1 << CFG["log2_T"], CFG["n_features"]
    H = synth.uniform_tables(L, T, F, 0, dtype="f32", scale=1e-4)[0].astype(np.float64)
    g = np.random.Generator(np.random.PCG64(1))
    dims = [(64, 32), (64, 64), (3, 64)]
    W = [g.uniform(-math.sqrt(6 / fi), math.sqrt(6 / fi), size=(fo, fi)) for fo, fi in dims]
    state = {"m": np.zeros_like(H), "v": np.zeros_like(H), "mW": [np.zeros_like(w) for w in W],
             "vW": [np.zeros_like(w) for w in W]}
    img = synth.ProceduralImage(seed=7, size=16384, n_waves=64)
    done, t0 = 0, time.perf_counter()
    times = []
    for k in range(steps):
        x = synth.uniform_points(sample_points, 2, 5000 + k)
        tgt = img.sample(x)
        s = time.perf_counter()
        oracle_step(x, tgt, H, W, state, k + 1)
        times.append(time.perf_counter() - s)
        done += 1
        if time.perf_counter() - t0 > seconds_cap:
            break
    return sample_points * done / sum(times), done, times


def cpu_baseline_subprocess(seconds):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-only", "--cpu-seconds", str(seconds)]
    try:
        res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
        return json.loads(res.stdout.strip().splitlines()[-1])
    except Exception as exc:  # report, do not fail the GPU line
        return {"value": None, "error": repr(exc)[:200]}


def cpu_baseline_only(seconds):
    sample = 1 << 13
    v, done, _ = time_oracle(sample, 1000, seconds)
    print(json.dumps({"value": v, "unit": "points/s", "cores": 1, "kind": "oracle",
                      "sample": "%d oracle steps of %d points each on the full workload tables "
                               "(L=16, T=2^22, F=2; Adam over all 134M table parameters)" % (done, sample)}))


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    sample = 1 << 12
    _, done, times = time_oracle(sample, args.warmup + args.steps, 1e9)
    t = times[args.warmup:]
    value = sample * len(t) / sum(t)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
        "steps": len(t), "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": "%d-point steps of the full workload (tables L=16, T=2^22)" % sample},
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
    ap.add_argument("--mlp-kernel", default="auto", choices=["auto", "mma_sync", "tcgen05"],
                    help="kernel of the network training pass")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--cpu-baseline-only", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.cpu_baseline_only:
        cpu_baseline_only(args.cpu_seconds)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
