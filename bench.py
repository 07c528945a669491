"""Benchmark: Mrays/s of the Schwarzschild renderer on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--form mixed|fp32|fp64] [--size 4096]

One step = one bh_render of the whole hot path over the workload: pinhole
camera rays, orbital-plane reduction, Dormand-Prince 5(4) with event location
(disk, spheres, capture, escape), shading and the SoA stores.  The default
workload is the 4096 x 4096 mixed-precision frame (r_obs = 50M, inclination
75 deg, disk [6M, 30M], 8 seeded spheres, FP32 stepping with FP64 for the
periastron reset and for |b - 3 sqrt(3) M| < 0.05M).  Rank 0 prints one JSON
line.  `--impl reference` times the CPU oracle instead (the FP64 plain
renderer on the host cores, a bounded pixel sample per step).

Multi-GPU: the path has no exchange step; N ranks render N independent
frames (replicas, weak scaling) and the value is the total over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2507_16165_gb300 import workloads as W  # noqa: E402

METRIC = "Mrays/s at 4096^2 (FP64 / FP32 / MLP surrogate) at stated exit-dir error"
UNIT = "Mrays/s"
# Algorithmic work of one attempted Dormand-Prince 5(4) step on (u, u') in
# the tableau's first-order form: 26 MUL + 59 FMA in the stages, error
# estimate, norm and scales, plus 4 in the step controller (89 FMA-pipe
# operations; an FMA counts as two floating-point operations).  The kernels
# take the same step in its second-order form with 57 operations, so the
# achieved rate counts the work of the method, not of that rewrite.
FLOP_PER_STEP = 2 * 59 + 26 + 4
SM_COUNT = 152
FP32_LANES_PER_SM = 128
# FP64 fused multiply-adds per SM and cycle on GB300 (the peak ncu reports for
# sm__sass_thread_inst_executed_op_dfma_pred_on: 2 per SM per cycle)
FP64_LANES_PER_SM = 2
# Algorithmic work of one classical Runge-Kutta step of the paper's own
# stepping mode: 4 right-hand sides (FMA + MUL), 6 stage arguments (FMA),
# the two weighted sums (2 x (3 ADD + MUL + FMA)) and h/6: 37 FLOP.
FLOP_PER_RK4_STEP = 4 * 3 + 6 * 2 + 2 * 6 + 1
STATED_ERROR = {"mixed": 1e-4, "fp32": 1e-4, "fp64": 1e-9, "surrogate": 1e-3,
                "paper": 1e-4, "paper_fp32": 1e-4}
# kernels one render launches: coherent + long-ray passes, and in MIXED the
# band pre-pass and the FP64 band pass
KERNELS_PER_RENDER = {"mixed": 4, "fp32": 2, "fp64": 2, "surrogate": 4, "paper": 1,
                      "paper_fp32": 1}


def workload(form: str, size: int, name: str = "c3"):
    """c3: the 4096^2 frame of one camera (the surrogate form renders the same
    scene: config 4); c5: the 64-camera orbit sequence (resolutions
    256^2..2048^2, about 9e7 rays) rendered by one graph replay."""
    if name == "c5":
        from dataclasses import replace
        return replace(W.config5(64), mode=form)
    if form == "surrogate":
        return W.config4(size)
    if form in ("paper", "paper_fp32"):
        # the paper's own fixed-step polyline on the config-3 scene
        from dataclasses import replace
        return replace(W.config3(size, "fp64"), mode=form, name=f"c3_{form}_{size}")
    return W.config3(size, form)


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2507_16165_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def profile_traffic(form: str) -> float | None:
    """DRAM bytes per launch of the coherent kernel from a committed ncu
    summary, or None when absent or taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except OSError:
        return None
    e = t.get(form)
    if not e or e.get("source_sha") != source_hash():
        return None
    return float(e["dram_bytes_per_launch"])


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over all ranks (x itself for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(rays_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job Mrays/s: each rank renders its own replica of the workload,
    and the job takes as long as its slowest rank."""
    return world * rays_per_rank * steps / seconds / 1e6


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, seconds: float = 10.0, seed: int = 0) -> dict:
    """The CPU oracle, as it stands, on a seeded random pixel sample of the
    workload, with every host core (OpenMP).  Test infrastructure: this leg is
    the only part of the GPU benchmark that runs the oracle."""
    import numpy as np

    import oracle
    lib = oracle.load()
    cores = oracle.threads(os.cpu_count() or 1, lib=lib)
    cam = w.cameras[0]
    rng = np.random.default_rng(seed)
    o = oracle.opts(rtol=1e-10, atol=1e-10)

    def run(n):
        idx = rng.integers(0, cam.w * cam.h, n)
        t0 = time.perf_counter()
        oracle.render_pixels(w.scene, w.cameras, np.zeros(n, np.int32), idx % cam.w,
                             idx // cam.w, o, nthreads=cores, lib=lib)
        return time.perf_counter() - t0

    probe = 1 << 14
    dt = run(probe)
    n = int(min(1 << 24, max(probe, probe * seconds / max(dt, 1e-6))))
    dt = run(n)
    return {"value": n / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} seeded random pixels of the {cam.w}x{cam.h} frame, FP64 oracle "
                      f"(rtol = atol = 1e-10), OpenMP dynamic schedule over the pixel list, "
                      f"{dt:.1f} s"}


def run_reference(args) -> None:
    """The CPU oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle
    w = workload(args.form, args.size)
    lib = oracle.load()
    cores = oracle.threads(os.cpu_count() or 1, lib=lib)
    cam = w.cameras[0]
    rng = np.random.default_rng(1)
    n = args.ref_pixels
    o = oracle.opts(rtol=1e-10, atol=1e-10)

    def step():
        idx = rng.integers(0, cam.w * cam.h, n)
        oracle.render_pixels(w.scene, w.cameras, np.zeros(n, np.int32), idx % cam.w,
                             idx // cam.w, o, nthreads=cores, lib=lib)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = n * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{w.name} (oracle on a {n}-pixel sample per step)",
                   "rays_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} seeded random pixels per step of the {cam.w}x{cam.h} "
                                   "frame, FP64 rtol = atol = 1e-10"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    import paper_2507_16165_gb300 as bh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world,
                                device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            t = torch.ones(1, device="cuda")
            dist.all_reduce(t)
        torch.cuda.synchronize()

    w = workload(args.form, args.size, args.workload)
    if args.sky_image:
        from dataclasses import replace
        w = replace(w, scene=replace(w.scene, sky_texture=W.sky_texture(0, 2048, 1024)))
    n = w.n_rays
    sc = bh.Scene(w.scene)
    cams = sc.cameras(w.cameras)
    wv = [c.w for c in w.cameras]
    hv = [c.h for c in w.cameras]
    stream = torch.cuda.Stream()
    f64 = args.form in ("fp64", "paper")
    paper = args.form in ("paper", "paper_fp32")
    dirs = torch.empty(2 * n, dtype=torch.float64 if f64 else torch.float32, device="cuda")
    flags = torch.empty(n, dtype=torch.int16, device="cuda")
    rgba = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    opts = bh.render_opts(args.form, stream, rtol=w.rtol, atol=w.atol, band=w.band,
                          paper_eps=args.paper_eps, spp=args.spp, doppler=int(args.doppler))
    # rays traced per pixel: n x n samples plus the centre ray when anti-aliased
    rays_per_pixel = args.spp + 1 if args.spp > 1 else 1

    surrogate = None
    if args.form == "surrogate":
        # trained weights of the project (train_surrogate.py); training time
        # is reported separately and is not part of the timed region
        path = os.path.join(ROOT, "paper_2507_16165_gb300", "data", "surrogate_m1.bin")
        bh.bh_surrogate_load(sc.handle, path)
        try:
            with open(os.path.splitext(path)[0] + ".json") as f:
                surrogate = json.load(f)
        except OSError:
            surrogate = {"weights": path}
    graph = None
    tuned = None
    if args.workload == "c5":
        # autotune the launch shape on this workload, then capture the whole
        # multi-camera render once and replay it
        tuned = bh.bh_autotune(sc.handle, cams, wv, hv, dirs, flags, rgba, opts)
        graph = bh.bh_graph_create(sc.handle, cams, wv, hv, dirs, flags, rgba, opts)

    def render():
        if graph:
            bh.bh_graph_launch(graph, stream)
        else:
            bh.bh_render(sc.handle, cams, wv, hv, dirs, flags, rgba, opts)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            render()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms, steps32, steps_all = [], 0, 0
    barrier()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 255)                 # L2 flush, outside the events
                starts[k].record(stream)
                render()
                ends[k].record(stream)
            st = bh.bh_render_stats(sc.handle)       # syncs the stream, outside the events
            kernel_ms.append(st["kernel_ms"])
            steps_all += st["steps"]
            steps32 += st["steps"] - st["steps_fp64"]
        barrier()
        t_wall = time.perf_counter() - t_wall
    bh.bh_scene_sync(sc.handle)
    ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), world, "cuda")
    ms_per_step = ms / args.steps
    value = job_rate(n * rays_per_pixel, args.steps, world, ms * 1e-3)

    # roofline: the integrator kernels (coherent + long-ray passes) against
    # the FP32 pipe, or the FP64 pipe in the FP64 form
    int_ms = sum(km[0] + km[1] for km in kernel_ms)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    lanes = FP64_LANES_PER_SM if f64 else FP32_LANES_PER_SM
    peak_tflops = SM_COUNT * lanes * 2 * sm_max * 1e6 / 1e12
    n_steps = steps_all if f64 else steps32
    flop_step = FLOP_PER_RK4_STEP if paper else FLOP_PER_STEP
    achieved = n_steps * flop_step / (int_ms * 1e-3) / 1e12 if int_ms > 0 else None
    prec = "FP64" if f64 else "FP32"
    method = f"fixed-step Runge-Kutta 4, eps {args.paper_eps}" if paper else "Dormand-Prince"
    roofline = {
        "bound": "alu",
        "achieved": achieved,
        "peak": peak_tflops,
        "unit": "TFLOP/s",
        "frac": (achieved / peak_tflops) if achieved is not None else None,
        # DRAM bytes per launch from the ncu capture of this exact workload
        # (the 4096^2 config-3 frame, default shading, one sample per pixel)
        "traffic": profile_traffic(args.form) if (args.workload == "c3" and args.size == 4096
                                                  and args.spp <= 1 and not args.sky_image
                                                  and not args.doppler) else None,
        "kernel": ("k_paper" if paper else "k_coherent + k_longrays") + f" ({prec} {method} steps)",
        "peak_source": f"derived: {SM_COUNT} SMs x {lanes} {prec} FMA lanes x 2 FLOP x "
                       f"{sm_max:.0f} MHz (max SM clock)",
        "algorithmic": f"{flop_step} FLOP per attempted {prec} step x "
                       f"{n_steps / args.steps:.0f} steps per frame",
        "integrator_ms_per_step": int_ms / args.steps,
    }

    # end to end through the C-ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        hd = torch.empty(2 * n, dtype=dirs.dtype, pin_memory=True)
        hf = torch.empty(n, dtype=torch.int16, pin_memory=True)
        hr = torch.empty(n, dtype=torch.int32, pin_memory=True)
        for _ in range(max(1, args.warmup)):
            bh.bh_render_host(sc.handle, cams, wv, hv, hd, hf, hr, opts)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            bh.bh_render_host(sc.handle, cams, wv, hv, hd, hf, hr, opts)
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        import ctypes
        from paper_2507_16165_gb300 import _capi
        e2e = {"value": job_rate(n * rays_per_pixel, args.steps, world, dt), "unit": UNIT,
               "h2d_bytes_per_step": len(cams) * (ctypes.sizeof(_capi.bh_camera) + 8),
               "d2h_bytes_per_step": n * (dirs.element_size() * 2 + 2 + 4)}

    stats = bh.bh_render_stats(sc.handle)
    if graph:
        bh.bh_graph_destroy(graph)
    sc.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None if (args.no_cpu or world > 1 or args.workload != "c3") else \
        cpu_baseline(w, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if f64 else ("f32" if paper else "f32+f64"),
        "data": "synthetic",
        "config": {"workload": w.name, "form": args.form, "rays_per_step": n,
                   "size": (f"{args.size}x{args.size}" if args.workload == "c3"
                            else f"{len(w.cameras)} cameras, 256^2..2048^2"),
                   "r_obs": 50.0 if args.workload == "c3" else "15..100 (log-uniform)",
                   "inclination_deg": 75.0 if args.workload == "c3" else "0..89",
                   "disk": list(w.scene.disk), "spheres": len(w.scene.spheres),
                   "rtol": w.rtol, "atol": w.atol,
                   "band": w.band, "stated_exit_dir_error_rad": STATED_ERROR[args.form],
                   "paper_eps": args.paper_eps if paper else None,
                   "spp": args.spp if args.spp > 1 else None,
                   "disk_shading": "keplerian doppler" if args.doppler else "temperature ramp",
                   "sky": "2048x1024 image, bilinear" if args.sky_image else "procedural checker",
                   "mpixels_per_s": job_rate(n, args.steps, world, ms * 1e-3),
                   "parallelism": f"replicas x{world}",
                   "l2": "256 MB buffer written between timed steps (outside the events)",
                   "launch": ("autotuned shape, one CUDA-graph replay per step: " + json.dumps(tuned))
                   if tuned else "bh_render per step, default launch shape"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": KERNELS_PER_RENDER[args.form] * args.steps,
        "clocks": clk.summary(),
        "surrogate_training": (dict({k: surrogate.get(k) for k in
                                     ("samples", "n_valid", "epochs", "steps", "wall_s",
                                      "train_ms", "label_ms", "val_rmse")},
                                    calib_samples=surrogate["calibration"]["samples"],
                                    calib_served_fraction=surrogate["calibration"]["served_fraction"],
                                    served_bins=surrogate["calibration"]["served_bins"],
                                    served_rays_fraction=stats["n_surrogate"] / n)
                               if surrogate else None),
        "steps_per_ray": steps_all / args.steps / (n * rays_per_pixel),
        "wall_s": t_wall,
        "stats_last": {k: stats[k] for k in ("rays", "n_band", "n_long", "periastron", "n_capt",
                                             "n_disk", "n_sphere", "n_esc", "n_surrogate",
                                             "n_fallback")},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--form", choices=("mixed", "fp32", "fp64", "surrogate", "paper", "paper_fp32"),
                    default="mixed")
    ap.add_argument("--sky-image", action="store_true",
                    help="a 2048x1024 synthetic sky image in place of the checker")
    ap.add_argument("--doppler", action="store_true",
                    help="Keplerian disk with Doppler and gravitational shift")
    ap.add_argument("--spp", type=int, default=1,
                    help="samples per pixel (a square; fp32 and fp64 forms)")
    ap.add_argument("--paper-eps", type=float, default=0.01,
                    help="fixed step of the paper's own stepping forms (rad)")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--workload", choices=("c3", "c5"), default="c3")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-pixels", type=int, default=1 << 18)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)   # timing rule: at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
