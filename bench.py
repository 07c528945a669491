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
# kernels one render launches: tile + long-ray passes, and in MIXED the band
# pre-pass and the FP64 band pass; the surrogate: band pre-pass, FP64 band
# pass, surrogate pass, lock-step pass over its fallback list, long-ray pass
KERNELS_PER_RENDER = {"mixed": 4, "fp32": 2, "fp64": 2, "surrogate": 5, "paper": 1,
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


# The NVML poller, run as its own process so that it never competes with
# the timed loop for the interpreter: it reads (never sets) the SM clock and
# the clock-event reason bits of one GPU every millisecond and writes them to
# a file, after printing "ready" once polling has begun.
_NVML_POLLER = r"""
import ctypes, signal, sys, time
ident, out = sys.argv[1], sys.argv[2]
lib = ctypes.CDLL("libnvidia-ml.so.1")
if lib.nvmlInit_v2() != 0:
    sys.exit(1)
dev = ctypes.c_void_p()
if ident.startswith("GPU-"):
    ok = lib.nvmlDeviceGetHandleByUUID(ident.encode(), ctypes.byref(dev)) == 0
else:
    n = ctypes.c_uint()
    lib.nvmlDeviceGetCount_v2(ctypes.byref(n))
    ok = lib.nvmlDeviceGetHandleByIndex_v2(0 if n.value == 1 else int(ident), ctypes.byref(dev)) == 0
if not ok:
    sys.exit(1)
reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
    lib.nvmlDeviceGetCurrentClocksThrottleReasons
mx, clk, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
lib.nvmlDeviceGetMaxClockInfo(dev, 1, ctypes.byref(mx))
stop = []
signal.signal(signal.SIGTERM, lambda *a: stop.append(1))
rows = []
print("ready", flush=True)
t_end = time.time() + 900
while not stop and time.time() < t_end:
    if lib.nvmlDeviceGetClockInfo(dev, 1, ctypes.byref(clk)) == 0 and reasons(dev, ctypes.byref(rs)) == 0:
        rows.append("%d %d %d" % (clk.value, mx.value, rs.value))
    time.sleep(0.001)
with open(out, "w") as f:
    f.write("\n".join(rows))
"""


class NvmlPoller:
    """SM clock and clock-event reasons of one GPU, read through NVML (the
    driver's libnvidia-ml) every millisecond by a separate process; raises
    OSError when NVML or the device cannot be found."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    def __init__(self, cuda_index: int):
        import tempfile
        ident = str(cuda_index)
        try:
            import torch
            uuid = getattr(torch.cuda.get_device_properties(cuda_index), "uuid", None)
            if uuid is not None:
                ident = "GPU-" + str(uuid)
        except Exception:
            pass
        fd, self.path = tempfile.mkstemp(prefix="bh_clocks_")
        os.close(fd)
        self.proc = subprocess.Popen([sys.executable, "-c", _NVML_POLLER, ident, self.path],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        # polling has begun once "ready" arrives (NVML found), else the process exits
        line = self.proc.stdout.readline()
        if line.strip() != "ready":
            self.proc.wait(timeout=5)
            os.unlink(self.path)
            raise OSError("NVML poller unavailable")

    def finish(self) -> dict | None:
        self.proc.terminate()
        try:
            self.proc.wait(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            return None
        try:
            with open(self.path) as f:
                rows = [tuple(int(x) for x in ln.split()) for ln in f if ln.strip()]
        finally:
            os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[0]) for r in rows)
        bits = 0
        for r in rows:
            bits |= r[2]
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(max(r[1] for r in rows)),
                "reasons": sorted(n for b, n in self.REASONS.items() if bits & b),
                "samples": len(sm), "source": "NVML every 1 ms (separate process)"}


class ClockSampler:
    """Clock and throttle-reason samples while the timed region runs: NVML
    polled every millisecond by a separate process where the driver's library
    loads (so that a region of a few tens of milliseconds holds many samples),
    and nvidia-smi at 50 ms beside it (the summary's fallback)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None
        self.nvml = None
        self.nvml_summary = None

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
        try:
            self.nvml = NvmlPoller(self.index)
        except (OSError, subprocess.SubprocessError):
            self.nvml = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.nvml:
            self.nvml_summary = self.nvml.finish()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self) -> dict:
        if self.nvml_summary:
            return self.nvml_summary
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
                "samples": len(sm), "source": "nvidia-smi every 50 ms"}


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


# Forms of the metric measured beside the headline, each on its own workload
# and options: (bh mode, workload, extra bh_render_opts, test asserting its
# stated error).  c5 is the 64-camera orbit sequence in one graph replay with
# the autotuned launch shape.
FORMS = {
    "fp64": ("fp64", "c3", {}, "tests/test_gpu_fullsize.py::c3_fp64_4096"),
    "fp32": ("fp32", "c3", {}, "tests/test_gpu_fullsize.py::c3_fp32_4096"),
    "mixed": ("mixed", "c3", {}, "tests/test_gpu_fullsize.py::c3_mixed_4096"),
    "mixed_literal": ("mixed", "c3", {"periastron_reset": 2},
                      "tests/test_gpu_fullsize.py::c3_mixed_literal_4096"),
    "surrogate": ("surrogate", "c3", {}, "tests/test_gpu_fullsize.py::c4_surrogate_4096"),
    "c5_fp32": ("fp32", "c5", {}, "tests/test_gpu_batch.py::test_batch64_full_size_sampled_parity[fp32]"),
    "c5_surrogate": ("surrogate", "c5", {},
                     "tests/test_gpu_batch.py::test_batch64_full_size_sampled_parity[surrogate]"),
}
# MLP work per evaluated ray (mlp_tc.cuh): per 128 rays, 18 tcgen05.mma of
# M = 128, N = 64, K = 16 (the high and low halves of the inputs of layers
# 1-3, four K blocks for layers 2 and 3) and 8 of N = 16 (layer 4), 2 FLOP a
# multiply-add; and one tanh.approx (one MUFU operation) per hidden
# activation, 3 x 64.
MLP_FLOP_PER_RAY = 2 * (18 * 64 * 16 + 8 * 16 * 16)
MLP_MUFU_PER_RAY = 3 * 64
# special-function (MUFU) operations per SM and cycle on Blackwell: 4 per
# SM sub-partition
MUFU_PER_SM = 16


class FormRun:
    """One form of the renderer set up on its workload: scene, device
    buffers, options and, for the 64-camera workload, the autotuned shape
    captured in a CUDA graph."""

    def __init__(self, bh, torch, form, wname, size, extra, stream, args):
        self.bh, self.torch = bh, torch
        self.form = form
        self.w = workload(form, size, wname)
        if args.sky_image:
            from dataclasses import replace
            self.w = replace(self.w, scene=replace(self.w.scene, sky_texture=W.sky_texture(0, 2048, 1024)))
        w = self.w
        self.n = w.n_rays
        self.sc = bh.Scene(w.scene)
        self.cams = self.sc.cameras(w.cameras)
        self.wv = [c.w for c in w.cameras]
        self.hv = [c.h for c in w.cameras]
        self.stream = stream
        self.f64 = form in ("fp64", "paper")
        self.paper = form in ("paper", "paper_fp32")
        n = self.n
        self.dirs = torch.empty(2 * n, dtype=torch.float64 if self.f64 else torch.float32, device="cuda")
        self.flags = torch.empty(n, dtype=torch.int16, device="cuda")
        self.rgba = torch.empty(n, dtype=torch.int32, device="cuda")
        self.extra = dict(extra)
        self.opts = bh.render_opts(form, stream, rtol=w.rtol, atol=w.atol, band=w.band,
                                   paper_eps=args.paper_eps, spp=args.spp,
                                   doppler=int(args.doppler), **self.extra)
        self.rays_per_pixel = args.spp + 1 if args.spp > 1 else 1
        self.surrogate = None
        if form == "surrogate":
            # trained weights of the project (train_surrogate.py); training
            # is reported separately and is not part of the timed region
            path = os.path.join(ROOT, "paper_2507_16165_gb300", "data", "surrogate_m1.bin")
            bh.bh_surrogate_load(self.sc.handle, path)
            try:
                with open(os.path.splitext(path)[0] + ".json") as f:
                    self.surrogate = json.load(f)
            except OSError:
                self.surrogate = {"weights": path}
        self.graph = None
        self.tuned = None
        if wname == "c5":
            # autotune the launch shape on this workload, then capture the
            # whole multi-camera render once and replay it
            self.tuned = bh.bh_autotune(self.sc.handle, self.cams, self.wv, self.hv, self.dirs,
                                        self.flags, self.rgba, self.opts)
            self.graph = bh.bh_graph_create(self.sc.handle, self.cams, self.wv, self.hv, self.dirs,
                                            self.flags, self.rgba, self.opts)

    def render(self):
        if self.graph:
            self.bh.bh_graph_launch(self.graph, self.stream)
        else:
            self.bh.bh_render(self.sc.handle, self.cams, self.wv, self.hv, self.dirs, self.flags,
                              self.rgba, self.opts)

    def timed(self, steps, warmup, flush, barrier=None):
        """Warm-up renders, then `steps` renders each bracketed by CUDA events
        on the render stream (L2 flushed before each, outside the events).
        Returns (total ms, per-render kernel times, statistics summed)."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            for _ in range(warmup):
                self.render()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        kernel_ms, tot = [], {}
        if barrier:
            barrier()
        for k in range(steps):
            with torch.cuda.stream(self.stream):
                flush.fill_(k & 255)
                starts[k].record(self.stream)
                self.render()
                ends[k].record(self.stream)
            st = self.bh.bh_render_stats(self.sc.handle)  # syncs the stream, outside the events
            kernel_ms.append(st["kernel_ms"])
            for key in ("steps", "steps_fp64", "mlp_rays", "n_surrogate"):
                tot[key] = tot.get(key, 0) + st[key]
        if barrier:
            barrier()
        self.bh.bh_scene_sync(self.sc.handle)
        ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
        return ms, kernel_ms, tot

    def roofline(self, kernel_ms, tot, steps, peaks):
        """Roofline of the dominant kernel: the integrator (coherent +
        long-ray passes) against the FP32 pipe (FP64 pipe in the FP64 form),
        or the surrogate pass against the special-function unit that one
        tanh per hidden activation loads, with its tensor-pipe work beside."""
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        if self.form == "surrogate":
            # kernel_ms[0]: the band pre-pass and the surrogate pass
            t_ms = sum(km[0] for km in kernel_ms)
            mufu = tot["mlp_rays"] * MLP_MUFU_PER_RAY
            peak = SM_COUNT * MUFU_PER_SM * sm_max * 1e6 / 1e12
            achieved = mufu / (t_ms * 1e-3) / 1e12 if t_ms > 0 else None
            flops = tot["mlp_rays"] * MLP_FLOP_PER_RAY / (t_ms * 1e-3) / 1e12 if t_ms > 0 else None
            bf16 = peaks.get("bf16_tflops")
            return {
                "bound": "xu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "kernel": "k_surrogate (set-up, MLP by tcgen05 FP16 into tensor memory, shading of the served rays)",
                "peak_source": f"derived: {SM_COUNT} SMs x {MUFU_PER_SM} MUFU ops per cycle x "
                               f"{sm_max:.0f} MHz (max SM clock)",
                "algorithmic": f"{MLP_MUFU_PER_RAY} tanh per network evaluation x "
                               f"{tot['mlp_rays'] / steps:.0f} evaluations per frame",
                "tensor": {"achieved": flops, "peak": bf16, "unit": "TFLOP/s",
                           "frac": flops / bf16 if (flops and bf16) else None,
                           "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst) of measured",
                           "algorithmic": f"{MLP_FLOP_PER_RAY} FLOP per evaluated ray"},
                "surrogate_pass_ms": t_ms / steps,
            }
        int_ms = sum(km[0] + km[1] for km in kernel_ms)
        lanes = FP64_LANES_PER_SM if self.f64 else FP32_LANES_PER_SM
        peak = SM_COUNT * lanes * 2 * sm_max * 1e6 / 1e12
        n_steps = tot["steps"] if self.f64 else tot["steps"] - tot["steps_fp64"]
        flop_step = FLOP_PER_RK4_STEP if self.paper else FLOP_PER_STEP
        achieved = n_steps * flop_step / (int_ms * 1e-3) / 1e12 if int_ms > 0 else None
        prec = "FP64" if self.f64 else "FP32"
        return {
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved is not None else None, "traffic": None,
            "kernel": ("k_paper" if self.paper else "k_coherent + k_longrays") + f" ({prec} steps)",
            "peak_source": f"derived: {SM_COUNT} SMs x {lanes} {prec} FMA lanes x 2 FLOP x "
                           f"{sm_max:.0f} MHz (max SM clock)",
            "algorithmic": f"{flop_step} FLOP per attempted {prec} step x "
                           f"{n_steps / steps:.0f} steps per frame",
            "integrator_ms_per_step": int_ms / steps,
        }

    def close(self):
        if self.graph:
            self.bh.bh_graph_destroy(self.graph)
            self.graph = None
        self.bh.bh_autotune_reset()
        self.sc.close()


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

    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    peaks = measured_peaks()
    extra = {"periastron_reset": 2} if args.periastron_reset == 2 else {}
    fr = FormRun(bh, torch, args.form, args.workload, args.size, extra, stream, args)
    w, n = fr.w, fr.n
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        ms, kernel_ms, tot = fr.timed(args.steps, args.warmup, flush, barrier)
        t_wall = time.perf_counter() - t_wall
    ms = max_over_ranks(ms, world, "cuda")
    ms_per_step = ms / args.steps
    value = job_rate(n * fr.rays_per_pixel, args.steps, world, ms * 1e-3)
    roofline = fr.roofline(kernel_ms, tot, args.steps, peaks)
    # DRAM bytes per launch from the ncu capture of this exact workload
    # (the 4096^2 config-3 frame, default shading, one sample per pixel)
    if (args.workload == "c3" and args.size == 4096 and args.spp <= 1 and not args.sky_image
            and not args.doppler and not extra):
        roofline["traffic"] = profile_traffic(args.form)

    # end to end through the C-ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        hd = torch.empty(2 * n, dtype=fr.dirs.dtype, pin_memory=True)
        hf = torch.empty(n, dtype=torch.int16, pin_memory=True)
        hr = torch.empty(n, dtype=torch.int32, pin_memory=True)
        for _ in range(max(1, args.warmup)):
            bh.bh_render_host(fr.sc.handle, fr.cams, fr.wv, fr.hv, hd, hf, hr, fr.opts)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            bh.bh_render_host(fr.sc.handle, fr.cams, fr.wv, fr.hv, hd, hf, hr, fr.opts)
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        import ctypes
        from paper_2507_16165_gb300 import _capi
        e2e = {"value": job_rate(n * fr.rays_per_pixel, args.steps, world, dt), "unit": UNIT,
               "h2d_bytes_per_step": len(fr.cams) * (ctypes.sizeof(_capi.bh_camera) + 8),
               "d2h_bytes_per_step": n * (fr.dirs.element_size() * 2 + 2 + 4)}

    stats = bh.bh_render_stats(fr.sc.handle)
    tuned, surrogate = fr.tuned, fr.surrogate
    fr.close()

    # every form of the metric, each on its own workload, after the headline
    forms = None
    if not args.no_forms:
        forms = {}
        with ClockSampler(local) as fclk:
            for name, (form, wname, fextra, test) in FORMS.items():
                f = FormRun(bh, torch, form, wname, 4096, fextra, stream, args)
                k = 3 if form == "fp64" else max(3, min(args.steps, 10))
                fms, fkm, ftot = f.timed(k, 3, flush, barrier)
                fms = max_over_ranks(fms, world, "cuda")
                forms[name] = {
                    "workload": f.w.name, "rays_per_frame": f.n,
                    "mrays_per_s": job_rate(f.n, k, world, fms * 1e-3),
                    "ms_per_frame": fms / k, "steps": k,
                    "steps_per_ray": ftot["steps"] / k / f.n,
                    "stated_exit_dir_error_rad": STATED_ERROR[form],
                    "error_asserted_by": test,
                    "options": fextra or None,
                    "roofline": f.roofline(fkm, ftot, k, peaks),
                    "launch": ("autotuned shape in one CUDA-graph replay: " + json.dumps(f.tuned))
                    if f.tuned else "bh_render, default launch shape",
                    "served_fraction": ftot["n_surrogate"] / k / f.n if form == "surrogate" else None,
                }
                f.close()
        base = forms["fp64"]["mrays_per_s"]
        for name, e in forms.items():
            e["speedup_vs_fp64_gpu"] = e["mrays_per_s"] / base if name.startswith(("fp", "mixed", "surr")) else None
        forms["clocks"] = fclk.summary()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None if (args.no_cpu or world > 1 or args.workload != "c3") else \
        cpu_baseline(w, args.cpu_seconds)
    c5 = args.workload == "c5"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if fr.f64 else ("f32" if (fr.paper or args.form == "fp32") else "f32+f64"),
        "data": "synthetic",
        "config": {"workload": w.name, "form": args.form, "rays_per_step": n,
                   "size": (f"{len(w.cameras)} cameras, 256^2..2048^2" if c5
                            else f"{args.size}x{args.size}"),
                   "r_obs": "15..100 (log-uniform)" if c5 else 50.0,
                   "inclination_deg": "0..89" if c5 else 75.0,
                   "disk": list(w.scene.disk), "spheres": len(w.scene.spheres),
                   "rtol": fr.opts.rtol, "atol": fr.opts.atol,
                   "rtol_far": 10 * fr.opts.rtol if not fr.f64 else fr.opts.rtol,
                   "h_max": 0.3 if not fr.f64 else None,
                   "h_max_far": 0.5 if not fr.f64 else None,
                   "far_rays": "|b - 3 sqrt(3) M| >= 2M take rtol_far and h_max_far",
                   "band": w.band,
                   "band_rtol": 1e-8 if args.form in ("mixed", "surrogate") else None,
                   "periastron_reset": (("FP64 turning point for every ray (b from the FP64 image "
                                         "radius)" if extra else
                                         "FP64 turning point for |b - 3 sqrt(3) M| < 2M")
                                        if args.form in ("mixed", "surrogate") else None),
                   "rtol_near": (fr.opts.rtol / 100 if args.form == "fp32" else None),
                   "stated_exit_dir_error_rad": STATED_ERROR[args.form],
                   "paper_eps": args.paper_eps if fr.paper else None,
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
        "forms": forms,
        "surrogate_training": (dict({k: surrogate.get(k) for k in
                                     ("samples", "n_valid", "epochs", "steps", "wall_s",
                                      "train_ms", "label_ms", "val_rmse")},
                                    calib_samples=surrogate["calibration"]["samples"],
                                    calib_served_fraction=surrogate["calibration"]["served_fraction"],
                                    served_bins=surrogate["calibration"]["served_bins"],
                                    served_rays_fraction=stats["n_surrogate"] / n)
                               if surrogate else None),
        "steps_per_ray": tot["steps"] / args.steps / (n * fr.rays_per_pixel),
        "wall_s": t_wall,
        "stats_last": {k: stats[k] for k in ("rays", "n_band", "n_long", "periastron", "n_capt",
                                             "n_disk", "n_sphere", "n_esc", "n_surrogate",
                                             "n_fallback", "mlp_rays")},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
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
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the other forms of the metric (measured after the headline)")
    ap.add_argument("--periastron-reset", type=int, default=1, choices=(1, 2),
                    help="mixed form: FP64 turning point for near-critical rays (1) or all (2)")
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
