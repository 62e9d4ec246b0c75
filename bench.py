"""Benchmark: plane extraction on organized point clouds, one frame per step.

Default workload: the 480x640 synthetic depth-camera frame (12 boxes, 15-degree ramp, 5 mm
noise, 1% outliers, 3% NaN; Laplacian 5 iterations, bilateral 3 iterations, K = 4). A step is
one pass of the whole path (Laplacian, normals, bilateral, mask, groups, segments) over one
frame already resident in HBM. The frame (3.7 MB) is smaller than L2, so L2 is flushed by
writing a 256 MB buffer before every timed step, outside the step's CUDA events.

Prints one JSON line. `value` is Mtri/s over all ranks (triangles = 2(H-1)(W-1) per frame),
`e2e` repeats the measurement from page-locked host buffers through the pipelined entry point
(pl3d_pipeline_*: every frame's points copied in and its mask, normals and labels copied out
inside the timed region, the copies of one frame beside the kernels of the next; the synchronous
one-frame call pl3d_extract_planes_host is reported beside it as `e2e.sync_call`), `roofline` describes
the kernel with the largest share of
device time, `cpu_baseline` times the FP64 oracle on the host cores on a bounded sample.

--impl reference times the FP64 oracle itself (the paper has no code to run) on the same
workload and prints the same line with "impl": "reference".

Multi-GPU (torchrun): frames are independent, so each rank runs its own frame (seeded by rank)
with no collective on the data path; only the timing uses a barrier and a max over ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Mtri/s smoothed+segmented and HBM roofline fraction; served p50/p99 frame latency"
E2E_DEPTH = 3          # frames in flight in the end-to-end pipeline
E2E_HOST_SETS = 8      # page-locked host input/output sets the end-to-end frames rotate through
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        rows = []
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((t, parts))
        inside = [r for r in rows if t0 <= r[0] <= t1] or [r for r in rows if t0 - 0.25 <= r[0] <= t1 + 0.25]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sm = [float(p[1]) for _, p in inside if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for _, p in inside if p[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, p in inside for i in range(4) if p[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


# ----------------------------------------------------------------------------- algorithmic work per launch


# FLOP per unit of work, from the operation lists of the method's arithmetic (Eq. 1-6, Algorithm 4)
# counted the way the FP32 peak counts them: an add, sub or mul is 1 FLOP, an FMA 2, an exp or
# rsqrt 1 (a count of one per listed operation, with "3 FMA" for a squared norm, gives smaller
# totals; the table below spells every operation out at FMA = 2, the unit of the peak).
FLOP_PER_UNIT = {
    # per point, iteration and window neighbour: difference 3 sub (3), squared norm 1 mul + 2 FMA
    # (5), 1/sqrt (1), weighted sum 3 FMA (6), weight sum 1 add (1)
    "laplacian_neighbour": 16.0,
    # per triangle, iteration and window triangle: centroid difference 3 sub + squared norm 5, normal
    # difference 3 sub + squared norm 5, exponent 2 adds + 1 mul (3), exp (1), weighted sum 3 FMA (6)
    "bilateral_window_triangle": 26.0,
    # per triangle: 2 edges (6 sub), cross product 3 mul + 3 FMA (9), unit length 1 mul + 2 FMA +
    # rsqrt + 3 mul (9), centroid 6 add + 3 mul (9) = 33, rounded down to 30 (edges shared in a quad)
    "geometry_triangle": 30.0,
    # per triangle and dominant normal: dot 1 mul + 2 FMA (5)
    "group_dot": 5.0,
}


def algorithmic_flop(H: int, W: int, prm: dict, K: int) -> dict:
    """FP32 FLOP per frame the method defines, phase by phase, from FLOP_PER_UNIT: Laplacian (Eq. 1-2)
    per point, iteration and window neighbour (k^2 - 1 of them); bilateral (Eq. 3-6) per triangle,
    iteration and window triangle (2 k^2 of them); geometry per triangle; group assignment per
    triangle and dominant normal. The unit counts are returned with them (`units`)."""
    npx = H * W
    ntri = 2 * (H - 1) * (W - 1)
    kl, kb = prm["lap_kernel"], prm["bil_kernel"]
    units = {"laplacian_neighbour": (kl * kl - 1) * npx * prm["lap_iters"],
             "bilateral_window_triangle": 2 * kb * kb * ntri * prm["bil_iters"],
             "geometry_triangle": ntri, "group_dot": K * ntri}
    f = {k: FLOP_PER_UNIT[k] * float(u) for k, u in units.items()}
    lap = f["laplacian_neighbour"]
    bil = f["bilateral_window_triangle"] + f["geometry_triangle"] + f["group_dot"]
    return {"laplacian": lap, "bilateral": bil, "total": lap + bil, "units": units, "flop_per_unit": FLOP_PER_UNIT}


def algorithmic_bytes(H: int, W: int) -> float:
    """HBM bytes the fully fused path must move per frame: read points 12 B/px; write normals
    12 B, mask 1 B and labels 4 B per triangle (about 46 B/px)."""
    return 12.0 * H * W + 17.0 * 2 * (H - 1) * (W - 1)


KERNEL_SOURCES = ["frame_kernels.cuh", "pl3d_internal.cuh", "sync.cuh", "df32.cuh", "uf.cuh", "f32x2.cuh"]


def kernel_source_hash() -> str:
    """sha256 over the sources the persistent kernels are compiled from."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2007_12065_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary of this kernel and workload, or None
    when the kernel sources changed since that capture (the summary records their hash)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        for key in ("traffic_bytes_per_launch:", "kernel_sources_sha256:"):
            if line.strip().startswith(key):
                vals[key] = line.strip()[len(key):].strip()
    if vals.get("kernel_sources_sha256:") != kernel_source_hash():
        return None
    try:
        return float(vals["traffic_bytes_per_launch:"])
    except (KeyError, ValueError):
        return None


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP32 CUDA-core peak: 128 lanes per SM, an FMA = 2 FLOP."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


# ----------------------------------------------------------------------------- oracle timing


def _cpu_name() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def time_oracle(frame, seconds_budget: float, threads: int, max_frames: int = 50) -> dict:
    """The oracle's method path on whole frames (its sensitivity reruns, test instrumentation, off)."""
    import oracle
    oracle.set_threads(threads)
    p = oracle.OracleParams(**frame.params)
    runs = []
    t_end = time.perf_counter() + seconds_budget
    while True:
        t0 = time.perf_counter()
        oracle.extract_planes(frame.points, p, frame.dominant_normals, sensitivity=False)
        runs.append(time.perf_counter() - t0)
        if time.perf_counter() >= t_end or len(runs) >= max_frames:
            break
    sec = statistics.median(runs)
    return {"seconds_per_frame": sec, "frames": len(runs), "threads": threads,
            "mtri_s": frame.n_triangles / sec / 1e6}


# ----------------------------------------------------------------------------- batched and served workloads

SERVED_SENSORS = [(240, 320)] * 3 + [(480, 640)] * 2 + [(720, 1280)] + [(128, 2048)] * 2


def _gen_frame(task):
    H, W, seed = task
    return synth.mixed_frame(H, W, seed=seed)


def generate_frames(tasks, procs: int):
    """Synthetic frames (H, W, seed) from the scene generators, made in a spawn pool (safe with
    CUDA initialised in this process)."""
    if procs <= 1 or len(tasks) <= 1:
        return [_gen_frame(t) for t in tasks]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(procs, len(tasks))) as pool:
        return pool.map(_gen_frame, tasks)


def batch_frames(bases: dict, n: int, seed: int):
    """n frames with sizes drawn uniformly from synth.MIXED_SIZES; each is one of the generated
    scenes of its size seen with fresh range noise (1e-3 relative, per pixel)."""
    rng = np.random.default_rng(seed)
    picks = rng.integers(0, len(synth.MIXED_SIZES), n)
    out = []
    for i, k in enumerate(picks):
        variants = bases[synth.MIXED_SIZES[int(k)]]
        base = variants[i % len(variants)]
        r = np.random.default_rng(seed * 7919 + i)
        pts = base.points * (1.0 + r.normal(0.0, 1e-3, base.points.shape[:2] + (1,))).astype(np.float32)
        out.append((np.ascontiguousarray(pts, dtype=np.float32), base))
    return out


def run_batched(pl3d, torch, dev, frames, reps: int) -> dict:
    """One batch of all frames (one persistent launch from a CUDA graph, autotuned launch shape)
    against one plain launch per frame, both timed with CUDA events on one stream."""
    stream = torch.cuda.current_stream(dev)
    ctx = pl3d.pl3d_create(dev.index or 0)
    b = pl3d.Batch()
    keep = []
    tris = 0
    for pts, base in frames:
        H, W = pts.shape[:2]
        n = 2 * (H - 1) * (W - 1)
        tris += n
        d = torch.from_numpy(pts).to(dev)
        o = (torch.empty(n, dtype=torch.uint8, device=dev), torch.empty((n, 3), device=dev),
             torch.empty(n, dtype=torch.int32, device=dev))
        p = pl3d.make_params(**base.params)
        keep.append((d, o, p, base.dominant_normals))
        b.add(d, H, W, p, base.dominant_normals, *o)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, n_rep):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(n_rep):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    batched = lambda: pl3d.pl3d_extract_planes_batched(ctx, b, stream)  # noqa: E731

    def per_frame():
        for (d, o, p, nd), (pts, base) in zip(keep, frames):
            pl3d.pl3d_extract_planes(ctx, d, pts.shape[0], pts.shape[1], p, nd, nd.shape[0], *o, stream)

    ms_default = timed(batched, reps)
    tun, tune_ms = pl3d.pl3d_autotune_batched(ctx, b, stream, reps=2)
    ms_batched = timed(batched, reps)
    pl3d.pl3d_set_tuning(ctx, None)
    ms_loop = timed(per_frame, reps)
    stats = pl3d.pl3d_batch_stats(ctx)
    smoothing = one_iteration_smoothing(pl3d, torch, ctx, keep, frames, stream)
    pl3d.pl3d_destroy(ctx)
    sizes = {}
    for pts, _ in frames:
        k = f"{pts.shape[0]}x{pts.shape[1]}"
        sizes[k] = sizes.get(k, 0) + 1
    return {"frames": len(frames), "sizes": sizes, "triangles": tris, "inputs_mb": sum(p.nbytes for p, _ in frames) / 1e6,
            "ms_batched": ms_batched, "mtri_s_batched": tris / ms_batched / 1e3,
            "ms_batched_default_tuning": ms_default, "tuning": tun.as_dict(),
            "ms_per_frame_launches": ms_loop, "mtri_s_per_frame_launches": tris / ms_loop / 1e3,
            "speedup_vs_per_frame": ms_loop / ms_batched, "graph_launches": stats["graph_launches"],
            "one_iteration_smoothing": smoothing,
            "l2": "inputs (about 450 MB) larger than L2; no flush"}


def one_iteration_work(name: str, px: int, tri: int) -> tuple[float, float]:
    """(algorithmic bytes, FLOP) of one filter iteration over px points and tri triangles with
    3 x 3 windows. Laplacian: read the points, write the displacement (12 + 12 B per point);
    8 window neighbours at FLOP_PER_UNIT. Bilateral pass: read points and displacement (24 B per
    point), write normal, mask, group and label (12 + 1 + 1 + 4 B per triangle); 18 window
    triangles at FLOP_PER_UNIT. Bilateral iteration alone (the filter step of Eq. 3-6 without
    geometry, groups, outputs and labels): read normal and centroid, write normal (36 B per
    triangle), the same 18 window triangles."""
    if name == "laplacian":
        return 24.0 * px, FLOP_PER_UNIT["laplacian_neighbour"] * 8 * px
    if name == "bilateral":
        return 24.0 * px + 18.0 * tri, FLOP_PER_UNIT["bilateral_window_triangle"] * 18 * tri
    if name == "bilateral_iteration":
        return 36.0 * tri, FLOP_PER_UNIT["bilateral_window_triangle"] * 18 * tri
    raise ValueError(name)


def one_iteration_smoothing(pl3d, torch, ctx, keep, frames, stream) -> dict:
    """The smoothing filters at one iteration per pass over the whole batch (inputs far larger
    than L2), as an HBM-roofline figure: the Laplacian phase reads the points (12 B/px) and writes
    the displacement (12 B/px); the bilateral phase reads points and displacement (24 B/px) and
    writes normals, mask, groups and labels (18 B/tri). Phase times come from the kernel's own
    %globaltimer stamps; alu_floor_us is the arithmetic of the pass at full FP32 issue (16 FLOP
    per Laplacian neighbour, 26 per bilateral window triangle, FMA = 2)."""
    peaks, src = _peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32 = fp32_peak_tflops(sms, float(peaks.get("sm_max_mhz", 2070.0))) * 1e12
    px = sum(p.shape[0] * p.shape[1] for p, _ in frames)
    tri = sum(2 * (p.shape[0] - 1) * (p.shape[1] - 1) for p, _ in frames)
    out = {}
    for name, lap, bil in (("laplacian", 1, 0), ("bilateral", 0, 1)):
        b = pl3d.Batch()
        for (d, o, p, nd), (pts, base) in zip(keep, frames):
            prm = dict(base.params, lap_iters=lap, bil_iters=bil, min_dot=1.5)
            b.add(d, pts.shape[0], pts.shape[1], pl3d.make_params(**prm), nd, *o)
        pl3d.pl3d_extract_planes_batched(ctx, b, stream)
        torch.cuda.synchronize()
        pl3d.pl3d_set_timing(ctx, True)
        pl3d.pl3d_read_timing(ctx, reset=True)
        for _ in range(3):
            pl3d.pl3d_extract_planes_batched(ctx, b, stream)
        t = pl3d.pl3d_read_timing(ctx, reset=True)
        pl3d.pl3d_set_timing(ctx, False)
        us = t[name][0] / t[name][1] * 1e3
        nbytes, flop = one_iteration_work(name, px, tri)
        gbs = nbytes / (us * 1e-6) / 1e9
        out[name] = {"us": us, "algorithmic_bytes": nbytes, "achieved_gbs": gbs,
                     "hbm_frac": gbs / float(peaks["hbm_gbs"]), "hbm_floor_us": nbytes / float(peaks["hbm_gbs"]) / 1e3,
                     "alu_floor_us": flop / fp32 * 1e6, "peak_source": f"{src} hbm_gbs"}
        if name == "bilateral":
            # the phase split by the tiles' stage totals (CTA time): its shares apply to the phase
            stages = {k: t[f"bil_{k}_cta"][0] for k in ("staging", "geometry", "iterations", "finish", "labels")}
            total = sum(stages.values()) or 1.0
            out[name]["stages_us"] = {k: us * v / total for k, v in stages.items()}
            it_us = us * stages["iterations"] / total
            ib, iflop = one_iteration_work("bilateral_iteration", px, tri)
            floor_us = max(ib / float(peaks["hbm_gbs"]) / 1e3, iflop / fp32 * 1e6)
            out["bilateral_iteration"] = {"us": it_us, "algorithmic_bytes": ib, "flop": iflop,
                                          "hbm_floor_us": ib / float(peaks["hbm_gbs"]) / 1e3,
                                          "alu_floor_us": iflop / fp32 * 1e6, "floor_us": floor_us,
                                          "frac_of_floor": floor_us / it_us,
                                          "tflops": iflop / (it_us * 1e-6) / 1e12}
    return out


def run_served(pl3d, torch, sensor_frames, rate: float, seconds: float, max_inflight: int, max_batch: int,
               seed: int) -> dict:
    """Replays a Poisson trace (total `rate` frames/s over the sensors, the sensor of each arrival
    uniform) against a server through the library's own trace driver (pl3d_server_replay: the
    submissions at their scheduled times and the collection of results run in native code);
    latency = end of the result's copy-out - scheduled arrival (the driver's submit lag included)."""
    ring = 8
    srv = pl3d.pl3d_server_create(0, max_inflight=max_inflight, max_batch_frames=max_batch, hbm_bytes=24 << 30)
    sources = []
    for fs in sensor_frames:
        H, W = fs[0].points.shape[:2]
        n = 2 * (H - 1) * (W - 1)
        sources.append(dict(points=[torch.from_numpy(f.points).pin_memory() for f in fs],
                            params=pl3d.make_params(**fs[0].params), dominant_normals=fs[0].dominant_normals,
                            outputs=[(torch.empty(n, dtype=torch.uint8).pin_memory(), torch.empty((n, 3)).pin_memory(),
                                      torch.empty(n, dtype=torch.int32).pin_memory()) for _ in range(ring)]))
    rng = np.random.default_rng(seed)
    n = max(1, int(rate * seconds))
    t_arr = np.cumsum(rng.exponential(1.0 / rate, n))
    which = rng.integers(0, len(sensor_frames), n)
    try:
        rep = pl3d.pl3d_server_replay(srv, sources, t_arr, which)
    finally:
        pl3d.pl3d_server_destroy(srv)
    return {"rate_fps": rate, "seconds": seconds, "requests": n, "p50_ms": rep["p50_ms"], "p90_ms": rep["p90_ms"],
            "p99_ms": rep["p99_ms"], "max_ms": rep["max_ms"], "mean_ms": rep["mean_ms"], "mtri_s": rep["mtri_s"],
            "achieved_fps": rep["achieved_fps"], "mean_batch_frames": rep["mean_batch_frames"],
            "max_batch_frames": rep["max_batch_frames"], "batches": rep["batches"],
            "max_inflight": rep["max_inflight"], "submit_lag_p99_ms": rep["submit_lag_p99_ms"],
            "all_ok": rep["failed"] == 0 and rep["completed"] == n, "driver": "pl3d_server_replay (native)"}


def served_sensor_frames(procs: int, seed: int = 105):
    tasks = [(H, W, seed * 100 + 10 * i + j) for i, (H, W) in enumerate(SERVED_SENSORS) for j in range(2)]
    fr = generate_frames(tasks, procs)
    return [fr[2 * i:2 * i + 2] for i in range(len(SERVED_SENSORS))]


# ----------------------------------------------------------------------------- arms


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_frame(workload: str, rank: int):
    """Rank 0 runs the named workload's own seed; other ranks run the same scene recipe with
    their own seed (frames are independent units: weak scaling, no data exchange)."""
    base = synth.WORKLOADS[workload]
    return base() if rank == 0 else base(seed=1000 + rank)


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The slowest rank's time: the job finishes when its last rank does."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mtri_s(triangles_per_rank: int, world: int, ms_per_step_max: float) -> float:
    """Whole-job throughput: every rank's triangles over the slowest rank's step time."""
    return triangles_per_rank * world / (ms_per_step_max / 1e3) / 1e6


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    frame = synth.WORKLOADS[args.workload]()
    cores = os.cpu_count() or 1
    import oracle
    oracle.set_threads(cores)
    p = oracle.OracleParams(**frame.params)
    for _ in range(args.warmup):
        oracle.extract_planes(frame.points, p, frame.dominant_normals, sensitivity=False)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.extract_planes(frame.points, p, frame.dominant_normals, sensitivity=False)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = frame.n_triangles / (ms / 1e3) / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mtri/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "H": frame.H, "W": frame.W, "triangles": frame.n_triangles},
        "cpu_baseline": {"value": value, "unit": "Mtri/s", "cores": cores, "kind": "oracle",
                         "sample": f"whole {frame.H}x{frame.W} frame per step, FP64 C oracle, OpenMP {cores} threads "
                                   "(sensitivity reruns off)"},
        "e2e": {"value": value, "unit": "Mtri/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_pl3d(args):
    import torch
    import paper_2007_12065_gb300 as pl3d
    from paper_2007_12065_gb300 import build as pl3d_build

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    pl3d_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    frame = rank_frame(args.workload, rank)
    H, W, ntri = frame.H, frame.W, frame.n_triangles
    params = pl3d.make_params(**frame.params)
    nd = frame.dominant_normals
    K = nd.shape[0]
    ctx = pl3d.pl3d_create(local)
    stream = torch.cuda.current_stream(dev)

    pts = torch.from_numpy(frame.points).to(dev)
    mask = torch.empty(ntri, dtype=torch.uint8, device=dev)
    normals = torch.empty((ntri, 3), dtype=torch.float32, device=dev)
    labels = torch.empty(ntri, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        pl3d.pl3d_extract_planes(ctx, pts, H, W, params, nd, K, mask, normals, labels, stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    # keep the GPU busy ~0.3 s before timing so that clocks settle and the sampler sees load
    t_warm = time.perf_counter()
    while time.perf_counter() - t_warm < 0.3:
        flush.fill_(0.5)
        step()
    torch.cuda.synchronize()

    # ---------------- timed region (device)
    def timed_region(timing: bool):
        n0 = pl3d.pl3d_launch_count(ctx)
        if timing:
            pl3d.pl3d_set_timing(ctx, True)
            pl3d.pl3d_read_timing(ctx, reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        t_b = time.perf_counter()
        per_kernel = None
        if timing:
            pl3d.pl3d_set_timing(ctx, False)
            per_kernel = pl3d.pl3d_read_timing(ctx, reset=True)
        return (pl3d.pl3d_launch_count(ctx) - n0, per_kernel, [a.elapsed_time(b) for a, b in ev], t_a, t_b)

    # The measured region runs the calls as a user makes them, without the library's per-phase
    # instrumentation; a second region with it on gives the kernel's own launch time and the
    # phase and stage times of the roofline.
    launches, _, step_ms, t0, t1 = timed_region(False)
    # A step far above the median means the stream ran dry while the host thread stalled (its
    # start event recorded, its launch late): re-measure once and say so, as for clock events.
    host_stall = None
    if max(step_ms) > 20 * statistics.median(step_ms):
        host_stall = {"max_step_ms": max(step_ms), "median_step_ms": statistics.median(step_ms)}
        launches, _, step_ms, t0, t1 = timed_region(False)
    _, per_kernel, instrumented_ms, _, _ = timed_region(True)
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    value = aggregate_mtri_s(ntri, world, ms)

    # ---------------- end to end: host buffers through the pipelined entry point
    # A stream of frames, each copied in from page-locked host memory, run, and copied back out;
    # the copies of one frame overlap the kernels of the others (pl3d_pipeline_*). The host
    # timer runs from the first submit to the last frame's outputs in host memory.
    step()
    torch.cuda.synchronize()
    ref = (mask.cpu(), normals.cpu(), labels.cpu())
    h_pts = [torch.from_numpy(frame.points).pin_memory() for _ in range(E2E_HOST_SETS)]
    h_out = [(torch.empty(ntri, dtype=torch.uint8).pin_memory(), torch.empty((ntri, 3), dtype=torch.float32).pin_memory(),
              torch.empty(ntri, dtype=torch.int32).pin_memory()) for _ in range(E2E_HOST_SETS)]
    e2e_steps = max(10 * args.steps, 200)
    pipe = pl3d.pl3d_pipeline_create(local, max_points=H * W, depth=E2E_DEPTH)

    def e2e_run(n):
        tickets = []
        for k in range(n):
            b = k % E2E_HOST_SETS
            if k >= E2E_HOST_SETS:
                pl3d.pl3d_pipeline_wait(pipe, tickets[k - E2E_HOST_SETS])   # host set b free again
            tickets.append(pl3d.pl3d_pipeline_submit(pipe, h_pts[b], H, W, params, nd, K, *h_out[b]))
        for t in tickets[-E2E_HOST_SETS:]:
            pl3d.pl3d_pipeline_wait(pipe, t)
        return (n - 1) % E2E_HOST_SETS

    e2e_run(max(args.warmup, 3) * E2E_HOST_SETS)
    barrier()
    t_a = time.perf_counter()
    last = e2e_run(e2e_steps)
    e2e_s = time.perf_counter() - t_a
    barrier()
    e2e_match = all(torch.equal(a.view(torch.uint8), b.view(torch.uint8)) for a, b in zip(h_out[last], ref))
    pl3d.pl3d_pipeline_destroy(pipe)
    e2e_ms = max_over_ranks(1e3 * e2e_s / e2e_steps, world, dev)

    # the synchronous host-buffer call, one frame at a time (latency of a lone frame)
    hs_pts, (hs_mask, hs_normals, hs_labels) = h_pts[0], h_out[0]
    for _ in range(3):
        pl3d.pl3d_extract_planes_host(ctx, hs_pts, H, W, params, nd, K, hs_mask, hs_normals, hs_labels, stream)
    torch.cuda.synchronize()
    sync_s = []
    for k in range(max(args.steps // 2, 10)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t_s = time.perf_counter()
        pl3d.pl3d_extract_planes_host(ctx, hs_pts, H, W, params, nd, K, hs_mask, hs_normals, hs_labels, stream)
        sync_s.append(time.perf_counter() - t_s)
    sync_ms = max_over_ranks(1e3 * sum(sync_s) / len(sync_s), world, dev)
    sampler.stop()
    clocks = sampler.summary(t0, t1)

    if rank != 0:
        pl3d.pl3d_destroy(ctx)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    # ---------------- explicit mesh and segment lists of the frame (pl3d_extract_mesh)
    mesh = None
    if world == 1:
        i32 = dict(dtype=torch.int32, device=dev)
        mo = [torch.empty(3 * ntri, **i32), torch.empty(ntri, **i32), torch.empty(3 * ntri, **i32),
              torch.zeros(3, dtype=torch.int64, device=dev), torch.empty(ntri, **i32), torch.empty(ntri + 1, **i32),
              torch.empty(ntri, **i32), torch.empty(ntri, dtype=torch.uint8, device=dev)]
        step()                                           # labels of this frame
        for _ in range(3):
            pl3d.pl3d_extract_mesh(ctx, pts, labels, H, W, *mo, stream=stream)
        m_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(50)]
        for e_a, e_b in m_ev:
            flush.fill_(0.25)
            e_a.record(stream)
            pl3d.pl3d_extract_mesh(ctx, pts, labels, H, W, *mo, stream=stream)
            e_b.record(stream)
        torch.cuda.synchronize()
        m_us = statistics.median(a.elapsed_time(b) for a, b in m_ev) * 1e3
        nT, nS, nL = (int(x) for x in mo[3].cpu())
        # algorithmic bytes: read points 12 B/px and labels 4 B/tri; write T_map 4 B/tri, T and HE
        # 12 B per kept triangle each, border 1 B per kept triangle, segment lists 4 B per listed one
        m_bytes = 12.0 * H * W + 8.0 * ntri + 25.0 * nT + 4.0 * nL + 8.0 * nS
        peaks_m, src_m = _peaks()
        mesh = {"us": m_us, "triangles": nT, "segments": nS, "in_segments": nL, "algorithmic_bytes": m_bytes,
                "achieved_gbs": m_bytes / (m_us * 1e-6) / 1e9, "peak_gbs": float(peaks_m["hbm_gbs"]),
                "frac": m_bytes / (m_us * 1e-6) / 1e9 / float(peaks_m["hbm_gbs"]),
                "peak_source": f"{src_m} hbm_gbs", "l2": "flushed before every launch"}

    # ---------------- Gaussian accumulator of the frame's filtered normals (pl3d_fastga, level 4)
    fastga = None
    if world == 1:
        ga_counts = torch.empty(5120, dtype=torch.int32, device=dev)
        step()
        for _ in range(3):
            pl3d.pl3d_fastga(ctx, normals, mask, ntri, 4, 1, ga_counts, None, stream)
        g_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(50)]
        for e_a, e_b in g_ev:
            flush.fill_(0.75)
            e_a.record(stream)
            pl3d.pl3d_fastga(ctx, normals, mask, ntri, 4, 1, ga_counts, None, stream)
            e_b.record(stream)
        torch.cuda.synchronize()
        g_us = statistics.median(a.elapsed_time(b) for a, b in g_ev) * 1e3
        n_in = int(ga_counts.sum().item())
        g_bytes = 13.0 * ntri                            # normal 12 B + mask 1 B per triangle
        peaks_g, src_g = _peaks()
        fastga = {"us": g_us, "level": 4, "cells": 5120, "triangles": ntri, "integrated": n_in,
                  "mnormals_s": n_in / (g_us * 1e-6) / 1e6, "algorithmic_bytes": g_bytes,
                  "achieved_gbs": g_bytes / (g_us * 1e-6) / 1e9, "hbm_frac": g_bytes / (g_us * 1e-6) / 1e9 /
                  float(peaks_g["hbm_gbs"]), "peak_source": f"{src_g} hbm_gbs", "l2": "flushed before every launch"}

    # ---------------- batched (256 mixed frames, one launch) and served (Poisson trace) workloads
    batched = served = None
    if world == 1 and not args.no_batched:
        tasks = [(H_, W_, 104_000 + 10 * i + j) for i, (H_, W_) in enumerate(synth.MIXED_SIZES) for j in range(2)]
        gen = generate_frames(tasks, os.cpu_count() or 1)
        bases = {hw: gen[2 * i:2 * i + 2] for i, hw in enumerate(synth.MIXED_SIZES)}
        batched = run_batched(pl3d, torch, dev, batch_frames(bases, 256, 104), reps=5)
        batched["config"] = "256 frames, sizes uniform over " + ", ".join(f"{a}x{b}" for a, b in synth.MIXED_SIZES)
    if world == 1 and not args.no_served:
        sf = served_sensor_frames(os.cpu_count() or 1)
        served = {"sensors": ", ".join(f"{a}x{b}" for a, b in SERVED_SENSORS),
                  "continuous_batching": run_served(pl3d, torch, sf, args.served_rate, args.served_seconds, 2, 64,
                                                    105),
                  "sequential_fifo": run_served(pl3d, torch, sf, args.served_rate, args.served_seconds, 1, 1, 105)}
        # the low and the saturating end of the swept range, both modes on the same traces
        served["rates"] = [{"mode": mode, **run_served(pl3d, torch, sf, r, args.served_seconds, mi, mb, 105)}
                           for r in args.served_rates if r != args.served_rate
                           for mode, mi, mb in (("continuous_batching", 2, 64), ("sequential_fifo", 1, 1))]
        if args.served_sweep:
            served["sweep"] = [{"mode": mode, **run_served(pl3d, torch, sf, r, 10.0, mi, mb, 105)}
                               for r in (200, 500, 1000, 2000, 5000)
                               for mode, mi, mb in (("continuous_batching", 2, 64), ("sequential_fifo", 1, 1))]

    # ---------------- roofline of the frame kernel (the only kernel: one launch per frame)
    peaks, peak_src = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    k_ms, k_n = per_kernel["frame_kernel"]
    avg_launch_s = k_ms / k_n / 1e3
    flop = algorithmic_flop(H, W, frame.params, K)
    nbytes = algorithmic_bytes(H, W)
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = fp32_peak_tflops(sm_count, mhz)
    achieved = flop["total"] / avg_launch_s / 1e12
    phases = {}
    for name in ("laplacian", "bilateral", "label_merge", "label_flatten"):
        p_ms, p_n = per_kernel[name]
        phases[name] = {"us": p_ms / max(p_n, 1) * 1e3}
    phases["laplacian"]["tflops"] = flop["laplacian"] / (phases["laplacian"]["us"] * 1e-6) / 1e12
    phases["bilateral"]["tflops"] = flop["bilateral"] / (phases["bilateral"]["us"] * 1e-6) / 1e12
    # the bilateral phase split by its tiles' stage totals (CTA time; the shares apply to the phase)
    st = {k: per_kernel.get(f"bil_{k}_cta", (0.0, 0))[0] for k in ("staging", "geometry", "iterations", "finish",
                                                                   "labels")}
    st_total = sum(st.values())
    if st_total > 0:
        phases["bilateral"]["stages_us"] = {k: phases["bilateral"]["us"] * v / st_total for k, v in st.items()}
    roofline = {"bound": "alu", "kernel": "frame_kernel", "achieved": achieved, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "traffic": recorded_traffic("frame_kernel", args.workload),
                "peak_source": f"FP32 CUDA-core peak: {sm_count} SMs x 128 lanes x 2 FLOP x {mhz} MHz",
                "avg_launch_us": avg_launch_s * 1e6, "work_per_launch": flop["total"], "work_unit": "FLOP",
                "work_units": flop["units"], "flop_per_unit": flop["flop_per_unit"],
                "hbm": {"algorithmic_bytes": nbytes, "achieved_gbs": nbytes / avg_launch_s / 1e9,
                        "peak_gbs": float(peaks["hbm_gbs"]), "peak_source": f"{peak_src} hbm_gbs"},
                "phases_us": phases}

    # ---------------- CPU baseline (oracle on the host cores, bounded sample)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        r = time_oracle(frame, args.cpu_seconds, cores)
        r1 = time_oracle(frame, 6.0, 1, max_frames=10)   # medians of 10 frames (fewer past the budget)
        r4 = time_oracle(frame, 3.0, 4, max_frames=10)
        cpu = {"value": r["mtri_s"], "unit": "Mtri/s", "cores": cores, "kind": "oracle",
               "sample": f"{r['frames']} whole {H}x{W} frames, median wall time, FP64 C oracle with OpenMP "
                         f"on {cores} threads (its sensitivity reruns, test instrumentation, off)",
               "single_thread": {"value": r1["mtri_s"], "frames": r1["frames"]},
               "four_threads": {"value": r4["mtri_s"], "frames": r4["frames"]},
               "cpu": _cpu_name()}

    line = {
        "metric": METRIC, "value": value, "unit": "Mtri/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "H": H, "W": W, "triangles_per_frame": ntri,
                   "frames_per_step_per_gpu": 1, "lap_iters": frame.params["lap_iters"],
                   "bil_iters": frame.params["bil_iters"], "K": K,
                   "l2": f"flushed before every timed step ({L2_FLUSH_BYTES >> 20} MB write, outside the step events)",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks,
        "e2e": {"value": aggregate_mtri_s(ntri, world, e2e_ms), "unit": "Mtri/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(h_pts[0].numel() * 4),
                "d2h_bytes_per_step": int(sum(t.numel() * t.element_size() for t in h_out[0])),
                "api": f"pl3d_pipeline_submit / pl3d_pipeline_wait, depth {E2E_DEPTH}: {e2e_steps} frames back to "
                       f"back from {E2E_HOST_SETS} page-locked host buffer sets; points copied in, mask, normals and "
                       "labels copied out, every frame, inside the host-timed region",
                "l2": "not flushed: every frame's points arrive over the host link inside the step",
                "outputs_match_device_path": bool(e2e_match),
                "sync_call": {"api": "pl3d_extract_planes_host (synchronous; L2 flushed before each call)",
                              "ms_per_frame": sync_ms, "mtri_s": aggregate_mtri_s(ntri, world, sync_ms)}},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "mesh": mesh,
        "fastga": fastga,
        "batched": batched,
        "served": served,
        "remeasured_after_host_stall": host_stall,
        "step_ms_p50": statistics.median(step_ms),
        "step_ms_min": min(step_ms),
        "step_ms_with_phase_timing": statistics.mean(instrumented_ms),
        "wall_s_timed_region": t1 - t0,
    }
    print(json.dumps(line), flush=True)
    pl3d.pl3d_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="pl3d", choices=["pl3d", "reference"])
    ap.add_argument("--workload", default="rgbd_480x640", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-frame batched workload")
    ap.add_argument("--no-served", action="store_true", help="skip the served (Poisson trace) workload")
    ap.add_argument("--served-rate", type=float, default=2000.0, help="frames/s of the served trace")
    ap.add_argument("--served-seconds", type=float, default=5.0, help="seconds of every served trace")
    ap.add_argument("--served-rates", type=float, nargs="*", default=[500.0, 5000.0],
                    help="further served rates (frames/s), each run in both modes")
    ap.add_argument("--served-sweep", action="store_true", help="also sweep 200..5000 frames/s, 10 s each")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_pl3d(args)


if __name__ == "__main__":
    main()
