#!/usr/bin/env python
"""Throughput of the forest-of-octrees raycaster: ray segments per second.

One step = one whole render of the adaptive cube workload: 2,053,451 leaves
(levels 2-8, 2:1 balanced, trilinear FP32 data from 16 seeded Gaussians),
perspective 45-degree camera at 1920x1080, Dormand-Prince 5(4) at tolerance
1e-6 inside the midpoint bisection (c_RK = 1/2): pruning, per-leaf segments
and the merge of every ray's segments into its pixel.  The metric is the
number of ray segments the render integrates divided by its device time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torchrun; each rank renders its own copy of the
workload (independent replicas, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-segments/s"
UNIT = "segments/s"
WORKLOAD = ("adaptive unit cube, levels 2-8 (2,053,451 leaves, 2:1 balanced, trilinear FP32), "
            "perspective 45deg 1920x1080, DOPRI5 tol 1e-6, c_RK 0.5")
# Algorithmic FP32 operations (FADD/FMUL/FFMA/FMNMX, one each) of the render
# path, counted from the kernel source: per (node, ray) visit of the subtree
# descent (the node's corner, per axis its three faces, their crossings and
# the two halves' min / max, then the 8 children's max / min chains sharing
# their x and y prefixes), per segment set-up
# (slab interval, reference coordinates, the field's cubic along the segment,
# the first medium evaluation) and per Dormand-Prince step (five medium
# evaluations, seven stages on (A, B_r, B_g, B_b), the embedded error, the
# split test and the Eq. 2.14 fold).
FP32_OPS_VISIT = 67
FP32_OPS_SEGMENT = 128
FP32_OPS_DOPRI_STEP = 234
# The same for the shell's per-ray kernel: per segment the ray / leaf
# intersection (four planes, two spheres), the field's set-up and its first
# medium evaluation; per Dormand-Prince step five medium evaluations (each the
# inverse map: two ratios and their arctangent series, the radius; 26 FMAs of
# the monomial polynomial; the transfer function) and the same stage, error,
# split and fold work as the cube.  Reciprocals and square roots (MUFU) are
# not counted.
FP32_OPS_SHELL_SEGMENT = 160
FP32_OPS_SHELL_DOPRI_STEP = 499
FP32_LANES_PER_SM = 128
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-row-stride", type=int, default=1,
                   help="CPU baseline renders every n-th image row")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    p.add_argument("--no-backward", action="store_true", help="skip the adjoint measurement")
    p.add_argument("--batch-cameras", type=int, default=64,
                   help="cameras of the batched (CUDA graph) measurement; 0 skips it")
    p.add_argument("--no-shell", action="store_true",
                   help="skip the cubed-sphere shell measurements (render and adjoint)")
    p.add_argument("--only-shell", action="store_true",
                   help="run the shell measurements alone (profiling captures)")
    p.add_argument("--shell-image", default="2048x2048",
                   help="image size WxH of the shell render (smaller sizes only for profiling)")
    p.add_argument("--shell-bwd-image", default="1024x1024",
                   help="image size WxH of the shell adjoint (smaller sizes only for profiling)")
    p.add_argument("--image", default="1920x1080",
                   help="image size WxH (smaller sizes only for profiling captures)")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over the ranks (the job's time is its slowest
    rank's); world == 1 returns x."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of independent replicas: every rank processes the
    same number of units; the job takes as long as its slowest rank."""
    return world * units_per_rank / (ms_max * 1e-3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_fma_peak(local: int) -> dict:
    """The FP32 FMA throughput of this GPU, measured: independent FFMA chains
    (paper_1809_01334_gb300/csrc/ocr_fp32_peak.cu), seven launches of about
    40 ms after a warm-up, CUDA events, SM clock sampled meanwhile.  The
    rate counts lane-FMA instructions per second (one FMA = one operation,
    as the kernels' algorithmic counts do)."""
    import ctypes
    from paper_1809_01334_gb300 import build as B
    B.build()
    lib = ctypes.CDLL(B.PEAK_LIB)
    fn = lib.ocr_fp32_fma_peak
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)]
    best, med, ms = ctypes.c_double(), ctypes.c_double(), ctypes.c_float()
    blocks_per_sm, trips, reps = 4, 60000, 7
    with ClockSampler(local) as clk:
        rc = fn(blocks_per_sm, trips, reps, ctypes.byref(best), ctypes.byref(med),
                ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError(f"FP32 FMA microbenchmark failed ({rc})")
    return {"fma_per_s_best": best.value, "fma_per_s_median": med.value, "ms_best": ms.value,
            "launch": f"{blocks_per_sm} CTAs of 256 threads per SM, 8 independent FFMA chains "
                      f"per thread, {trips} x 16 steps each",
            "clocks": clk.summary()}


def subtree_traffic():
    """DRAM bytes per launch of the subtree pass from the committed ncu capture
    (profiles/subtree_kernel_traffic.json), or None when the kernel's sources
    have changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "subtree_kernel_traffic.json")) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for f in rec["sources"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        return rec["dram_bytes_per_launch"] if h.hexdigest() == rec["sources_sha256"] else None
    except (OSError, ValueError, KeyError):
        return None


def cpu_baseline(forest, tf, cam, integ, stride: int):
    """The FP64 oracle, as it stands, on this host's cores: every stride-th row."""
    import numpy as np
    import oracle as O
    rows = np.arange(0, cam.h, stride, dtype=np.int32)
    O.build()
    t0 = time.perf_counter()
    r = O.render(forest, tf, cam, integ, rows=rows)
    dt = time.perf_counter() - t0
    cores = os.cpu_count()
    return {"value": r["segments"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"every {stride}th row of the 1920x1080 image ({len(rows)} rows, "
                      f"{r['segments']} segments, {dt:.1f} s)"}


def run_batch(args, forest, tf, integ, dev, flush):
    """Many cameras of uneven sizes (log-uniform 256^2 .. 2048^2) rendered by one
    CUDA-graph launch, against the same cameras rendered one view at a time
    (each: set the camera, render, as a single-view user would)."""
    import torch
    from paper_1809_01334_gb300 import Renderer
    from paper_1809_01334_gb300 import inputs as I
    cams = I.batch_cameras(args.batch_cameras)
    npix = sum(c.w * c.h for c in cams)
    r = Renderer(forest, tf, integ, device=dev)
    r.set_cameras(cams)
    tune = r.autotune(reps=1)
    out = torch.empty((npix, 4), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    reps = 3

    def graph_ms():
        """Device time of one replay of the batch captured in a CUDA graph."""
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            r.render_batch(out, stream=s)  # warm-up outside the capture
        torch.cuda.current_stream(dev).wait_stream(s)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            r.render_batch(out, stream=torch.cuda.current_stream(dev))
        ms = []
        for k in range(1 + reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            torch.cuda.synchronize(dev)
            if k:
                ms.append(a.elapsed_time(b))
        del g
        return sum(ms) / len(ms)

    # the best decomposition of each kind: the persistent kernel and the
    # per-camera kernel chains on the internal streams
    best = {}
    for t in tune["tried"]:
        kind = "persistent" if t["persistent"] and not t["merge"] else "streams"
        if kind not in best or t["ms"] < best[kind]["ms"]:
            best[kind] = t
    modes = {}
    for kind in ("streams", "persistent"):
        if kind in best:
            t = best[kind]
            r.set_tuning(t["tile_depth"], t["streams"], t["shell_warps"], t["merge"],
                         1 if kind == "persistent" else 0, t["chunks_per_item"], t["ctas_per_sm"])
            modes[kind] = {"graph_ms": graph_ms(), "tuning": t}
    win = min(modes, key=lambda k: modes[k]["graph_ms"])
    t = modes[win]["tuning"]
    r.set_tuning(t["tile_depth"], t["streams"], t["shell_warps"], t["merge"],
                 1 if win == "persistent" else 0, t["chunks_per_item"], t["ctas_per_sm"])
    _, _, st = r.render_batch(out, with_index=True)
    segments = st["segments"]
    gms = [modes[win]["graph_ms"]]
    # one view at a time: the same planned cameras (planning is outside the
    # timed region for both arms), each view rendered alone on the stream
    # after the previous one, device time
    views = [torch.empty((c.h, c.w, 4), dtype=torch.float32, device=dev) for c in cams]
    seq = []
    for k in range(1 + reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for v in range(len(cams)):
            r.render_view(v, views[v], stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        if k:
            seq.append(a.elapsed_time(b))
    r.close()
    gm = sum(gms) / len(gms)
    sq = sum(seq) / len(seq)
    return {"cameras": len(cams), "pixels": npix, "segments": segments,
            "graph_ms": gm, "sequential_ms": sq, "speedup_vs_sequential": sq / gm,
            "decomposition": win, "launches_per_batch": st["launches"],
            "persistent_graph_ms": modes.get("persistent", {}).get("graph_ms"),
            "streams_graph_ms": modes.get("streams", {}).get("graph_ms"),
            "segments_per_s": segments / (gm * 1e-3), "mpixel_per_s": npix / (gm * 1e-3) / 1e6,
            "autotune": {"best": tune["best"], "tried": tune["tried"]},
            "sequential": "the same planned cameras, one ocr_render_view per view in "
                          "order on one stream, device time (L2 flushed before each arm)",
            "sizes": "square, side round(256 * 8**u), u ~ U[0,1], seeded"}


def _timed(fn, stream, flush, warmup, steps):
    """Mean device time (ms) of fn() over steps runs after warmup runs, L2
    flushed before each (outside the timed interval)."""
    import torch
    ms = []
    for k in range(warmup + steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        if k >= warmup:
            ms.append(a.elapsed_time(b))
    return sum(ms) / len(ms)


def run_shell(args, dev, flush):
    """Cubed-sphere shell render: 6 trees, levels 4-7 (5,001,233 leaves),
    degree-2 data, 2048x2048, DOPRI5 tol 1e-5; and the adjoint of an L2 loss
    on the levels 4-6 shell (1,082,535 leaves) at 1024x1024."""
    import numpy as np
    import torch
    from paper_1809_01334_gb300 import Renderer
    from paper_1809_01334_gb300 import inputs as I
    stream = torch.cuda.current_stream(dev)
    sw, sh = (int(x) for x in args.shell_image.split("x"))
    forest, tf, cam, integ = I.preset_c3(w=sw, h=sh)
    r = Renderer(forest, tf, integ, device=dev)
    r.set_camera(cam)
    out = torch.empty((cam.h, cam.w, 4), dtype=torch.float32, device=dev)
    _, st = r.render(out, fill_counters=True)
    phases = []

    def fwd():
        phases.append(r.render(out, time_phases=True)[1])
    ms = _timed(fwd, stream, flush, 2, 5)
    rays_ms = sum(p["ms_subtree"] for p in phases[2:]) / len(phases[2:])
    shell_ops = FP32_OPS_SHELL_SEGMENT * st["segments"] + FP32_OPS_SHELL_DOPRI_STEP * st["rk_steps"]
    shell_peak = args.fp32_peak["fma_per_s_best"] / 1e12
    c3 = {"workload": "cubed-sphere shell, 6 trees, levels 4-7 (%d leaves, degree-2 FP32 "
                      "data), perspective 45deg %dx%d, DOPRI5 tol 1e-5" % (forest.nleaves, sw, sh),
          "ms_per_render": ms, "segments": st["segments"], "rk_steps": st["rk_steps"],
          "pair_tests": st["leaf_tests"], "segments_per_s": st["segments"] / (ms * 1e-3),
          "mpixel_per_s": cam.w * cam.h / (ms * 1e-3) / 1e6, "ms_rays_kernel": rays_ms,
          "launches": st["launches"],
          "roofline": {"bound": "alu", "kernel": "shell_rays_kernel",
                       "achieved": shell_ops / (rays_ms * 1e-3) / 1e12, "peak": shell_peak,
                       "unit": "TFP32op/s",
                       "frac": shell_ops / (rays_ms * 1e-3) / 1e12 / shell_peak,
                       "fp32_ops_per_launch": shell_ops,
                       "peak_source": "measured (FP32 FMA microbenchmark)"}}
    r.close()
    del out
    # differentiation on the levels 4-6 shell
    bw, bh = (int(x) for x in args.shell_bwd_image.split("x"))
    forest, tf, cam, integ = I.preset_c5(w=bw, h=bh)
    r = Renderer(forest, tf, integ, device=dev)
    r.set_camera(cam)
    out = torch.empty((cam.h, cam.w, 4), dtype=torch.float32, device=dev)
    pert = forest.nodal * (1 + 0.05 * np.random.default_rng(1809).uniform(-1, 1, forest.nodal.shape))
    base = r.nodal
    r.set_data(torch.from_numpy(pert.astype(np.float32)).to(dev), r.tf)
    target = r.render(out)[0].clone()
    r.set_data(base, r.tf)
    img = r.render(out)[0]
    grad_img = (2.0 * (img - target)).contiguous()
    _, st = r.render(out, fill_counters=True)
    fms = _timed(lambda: r.render(out), stream, flush, 2, 5)
    bms = _timed(lambda: r.backward(grad_img, check=False), stream, flush, 2, 5)
    r.sync()  # device errors of the stream-ordered adjoint
    c5 = {"workload": "cubed-sphere shell, levels 4-6 (%d leaves, degree-2 FP32 data), "
                      "%dx%d, DOPRI5 tol 1e-5; L2 loss against a render of a seeded 5%% "
                      "nodal perturbation" % (forest.nleaves, bw, bh),
          "ms_forward": fms, "ms_backward": bms, "fwd_bwd_over_fwd": (fms + bms) / fms,
          "segments": st["segments"], "grads": "27 nodal values per leaf and the 32 knot values"}
    r.close()
    return c3, c5


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step renders a bounded sample of rows."""
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    from paper_1809_01334_gb300 import inputs as I
    O.build()
    forest, tf, cam, integ = I.preset_c2()
    nrows = cam.h // 8  # every 8th row per step (the oracle's per-call set-up is then a small part)
    times, segs = [], []
    for k in range(args.warmup + args.steps):
        rows = np.arange(k % 8, cam.h, 8, dtype=np.int32)[:nrows]
        t0 = time.perf_counter()
        r = O.render(forest, tf, cam, integ, rows=rows)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            segs.append(r["segments"])
    value = sum(segs) / sum(times)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{nrows} rows per step"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": f"{nrows} image rows per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1809_01334_gb300 import Renderer
    from paper_1809_01334_gb300 import inputs as I

    torch.cuda.set_device(local)
    args.fp32_peak = fp32_fma_peak(local)
    if args.only_shell:
        dev = torch.device("cuda", local)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        with ClockSampler(local) as clk:
            c3, c5 = run_shell(args, dev, flush)
        if rank == 0:
            print(json.dumps({"shell_render": c3, "shell_backward": c5,
                              "fp32_peak": args.fp32_peak, "clocks": clk.summary()}), flush=True)
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    w, h = (int(x) for x in args.image.split("x"))
    forest, tf, cam, integ = I.preset_c2(w=w, h=h)
    r = Renderer(forest, tf, integ, device=dev)
    r.set_camera(cam)
    out = torch.empty((cam.h, cam.w, 4), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # the segment count of this workload is deterministic: take it once
    _, st0 = r.render(out, fill_counters=True)
    segments, launches = st0["segments"], st0["launches"]

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    for _ in range(args.warmup):
        flush.zero_()
        r.render(out)
    torch.cuda.synchronize(dev)

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    merge_ms, prune_ms, sub_ms = [], [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()  # outside the timed interval of the step
            evs[k][0].record(stream)
            _, st = r.render(out, time_phases=True)
            evs[k][1].record(stream)
            merge_ms.append(st["ms_merge"])
            prune_ms.append(st["ms_prune"])
            sub_ms.append(st["ms_subtree"])
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    ms_max = max_over_ranks(ms, world, dev)

    # end to end through the C ABI with host buffers (ocr_render_host): the
    # nodal data and knots copied in from pinned host memory, the image copied
    # out, every step
    nodal_h = torch.from_numpy(np.ascontiguousarray(forest.nodal, np.float32)).pin_memory()
    tf_h = torch.from_numpy(np.ascontiguousarray(tf.knots, np.float32)).pin_memory()
    out_h = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    e2e_ms = []
    for k in range(0 if args.no_e2e else args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r.render_host(nodal_h, tf_h, out_h, stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        if k >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    e2e = sum(e2e_ms) / len(e2e_ms) if e2e_ms else float("nan")
    e2e_max = max_over_ranks(e2e, world, dev)

    # differentiation: dL/d(nodal, knots) of an L2 loss against a target rendered
    # from a seeded 5% perturbation of the nodal data (segments recomputed)
    bwd_ms = []
    if not args.no_backward:
        pert = forest.nodal * (1 + 0.05 * np.random.default_rng(5).uniform(-1, 1, forest.nodal.shape))
        r.set_data(torch.from_numpy(pert.astype(np.float32)).to(dev), r.tf)
        target = r.render(out)[0].clone()
        r.set_data(torch.from_numpy(np.ascontiguousarray(forest.nodal, np.float32)).to(dev), r.tf)
        img = r.render(out)[0]
        grad_img = (2.0 * (img - target)).contiguous()
        for k in range(args.warmup + max(3, args.steps // 4)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r.backward(grad_img, check=False)  # stream-ordered
            b.record(stream)
            torch.cuda.synchronize(dev)
            if k >= args.warmup:
                bwd_ms.append(a.elapsed_time(b))
        r.sync()  # device errors of the stream-ordered adjoint

    batch = run_batch(args, forest, tf, integ, dev, flush) if args.batch_cameras > 0 else None
    shell = run_shell(args, dev, flush) if not args.no_shell else None

    if rank == 0:
        peaks, src = measured_peaks()
        mm = sum(merge_ms) / len(merge_ms)
        sm = sum(sub_ms) / len(sub_ms)
        # the dominant kernel is the subtree pass: FP32-ALU bound (its DRAM
        # traffic is a few percent of peak); peak = SMs x FP32 lanes x clock
        ops = (FP32_OPS_VISIT * st0["subtree_node_visits"] +
               FP32_OPS_SEGMENT * st0["subtree_segments"] +
               FP32_OPS_DOPRI_STEP * st0["subtree_rk_steps"])
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        nominal = nsm * FP32_LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6
        peak_ops = args.fp32_peak["fma_per_s_best"]
        achieved = ops / (sm * 1e-3)
        line = {
            "metric": METRIC, "value": job_throughput(segments, world, ms_max), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if (w, h) == (1920, 1080) else
                       WORKLOAD.replace("1920x1080", f"{w}x{h}"),
                       "image": [cam.w, cam.h], "leaves": forest.nleaves,
                       "segments_per_step": segments, "rk_steps_per_step": st0["rk_steps"],
                       "slots_per_step": st0["slots"], "slab_tests_per_step": st0["leaf_tests"],
                       "subtree_node_visits_per_step": st0["subtree_node_visits"],
                       "mpixel_per_s": world * cam.w * cam.h / (ms_max * 1e-3) / 1e6,
                       "l2": "flushed (512 MB write) before every timed step",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": launches * args.steps,
            "e2e": {"value": job_throughput(segments, world, e2e_max), "unit": UNIT,
                    "h2d_bytes_per_step": int(nodal_h.numel() * 4 + tf_h.numel() * 4),
                    "d2h_bytes_per_step": int(out_h.numel() * 4),
                    "api": "ocr_render_host (pinned host buffers; the copy in overlaps pruning)"},
            "roofline": {"bound": "alu", "kernel": "subtree_kernel",
                         "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "TFP32op/s", "frac": achieved / peak_ops,
                         "traffic": subtree_traffic(), "traffic_unit": "bytes per launch (ncu)",
                         "fp32_ops_per_launch": ops, "ms_per_launch": sm,
                         "peak_source": "measured (FP32 FMA microbenchmark, this run)",
                         "peak_measurement": args.fp32_peak,
                         "nominal_peak": nominal / 1e12,
                         "nominal_source": f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                           f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({src})",
                         "ms_merge": mm, "ms_prune": sum(prune_ms) / len(prune_ms),
                         # the same operations over the whole render's step
                         "render_frac": ops / (ms_max * 1e-3) / peak_ops},
            "clocks": clk.summary(),
        }
        if batch:
            line["batch"] = batch
        if shell:
            line["shell_render"], line["shell_backward"] = shell
        if bwd_ms:
            mb = sum(bwd_ms) / len(bwd_ms)
            line["backward"] = {"ms_backward": mb, "ms_forward": ms_max,
                                "fwd_bwd_over_fwd": (ms_max + mb) / ms_max,
                                "loss": "L2 against a render of a seeded 5% nodal perturbation",
                                "grads": "nodal values and transfer-function knots"}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(forest, tf, cam, integ, args.cpu_row_stride)
        print(json.dumps(line), flush=True)
    r.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
