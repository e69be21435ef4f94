#!/usr/bin/env python3
"""Benchmark: 3D C2C FFT (forward + backward) of a 256^3 PME-shaped complex64 grid.

One step = one forward and one backward transform of the whole grid through
the C ABI (libcroft.so), i.e. every pass of the hot path.  Metric: GFLOP/s with
the nominal count 5 N log2 N per direction.

Timing: plan outside the timed region; W warm-up steps; then K steps, each
preceded by an L2 flush (a write of a buffer twice the L2 size, outside the
timed events); each transform is bracketed by CUDA events on the stream it runs
on and the step time is the sum of the two.  The dominant pass kernel is timed
by the plan's own per-pass events inside the same steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl croft|reference]

With N > 1 (torchrun) every rank runs an independent replica of the workload
(the single-grid transform has no data-parallel shard on one box) and value is
the sum over ranks; the time is the max over ranks.

--impl reference times the FP64 CPU oracle (the only reference this method has)
on the host cores, on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (256, 256, 256)
WORKLOAD = "pme256: 256x256x256 complex64 C2C forward+backward, 200k +-1 charges spread by order-4 B-splines, seed 1"
METRIC = "3D C2C FFT GFLOP/s (5N log2 N), % of HBM roofline, TC vs FP32 at fixed error"
HBM_FALLBACK_GBS = 6800.0


def nominal_flops(shape) -> float:
    n = math.prod(shape)
    return 5.0 * n * math.log2(n)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return HBM_FALLBACK_GBS, "fallback"


# The sources that decide the pass kernels' code and launch shape: a DRAM-traffic figure
# taken with ncu stays valid while these files are unchanged.
PASS_KERNEL_SOURCES = ("croft_butterflies.cuh", "croft_fft_core.cuh", "croft_internal.h", "croft_kernels.cu",
                       "croft_pass_kernel.cuh", "croft_passes.cu", "croft_row_layouts.h",
                       "croft_sched.h", "croft_sizes.h")


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2002_04896_gb300", "csrc")
    for name in PASS_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "ncu_dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:  # noqa: BLE001
        return None
    ent = d.get(kernel_key)
    if not ent or ent.get("src_sha") != kernel_source_sha():
        return None
    return float(ent["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:  # noqa: BLE001
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(torch, value: float, device) -> float:
    """The largest of every rank's `value` (an all-reduce, so also a barrier); `value` itself
    when no process group is initialised.  Times are aggregated this way: the job takes as
    long as its slowest rank."""
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(world: int, flops_per_rank_step: float, ms_step: float) -> float:
    """Whole-job throughput: every rank runs its own replica of the step (weak scaling)."""
    return world * flops_per_rank_step / (ms_step * 1e-3) / 1e9


def cpu_oracle_step(x, sample_planes=None):
    """Forward + backward with the FP64 oracle; optionally on a sample of the pencils of each axis.

    sample_planes = s: the z and y passes run on x-slabs [0, s) and the x pass on
    y-slabs [0, s): s/nx of the 1D DFTs of every axis (a bounded sample of the step).
    Returns the nominal flops the sample covers.
    """
    import numpy as np

    import oracle

    if sample_planes is None:
        y = oracle.forward(x)
        oracle.backward(y.astype(np.complex64))
        return 2 * nominal_flops(x.shape)
    s = sample_planes
    frac = s / x.shape[0]
    for sign in (oracle.FORWARD, oracle.BACKWARD):
        a = x[:s].astype(np.complex128)
        a = oracle.dft_along_axis(a, 2, sign)
        a = oracle.dft_along_axis(a, 1, sign)
        b = x[:, :s].astype(np.complex128)
        oracle.dft_along_axis(b, 0, sign)
    return 2 * nominal_flops(x.shape) * frac


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import synthetic_inputs as S

    x = S.config_input("pme256")
    cores = os.cpu_count()
    # the whole step unless (steps + warmup) full steps would exceed ~3 minutes; then a
    # fixed fraction of the pencils of every axis per step
    t0 = time.perf_counter()
    cpu_oracle_step(x, None)
    t_full = time.perf_counter() - t0
    sample = None
    if t_full * (args.steps + args.warmup) > 180.0:
        sample = max(1, int(SHAPE[0] * 180.0 / (t_full * (args.steps + args.warmup))))
    for _ in range(args.warmup - 1):
        cpu_oracle_step(x, sample)
    t0 = time.perf_counter()
    fl = 0.0
    for _ in range(args.steps):
        fl += cpu_oracle_step(x, sample)
    dt = time.perf_counter() - t0
    val = fl / dt / 1e9
    part = "all" if sample is None else f"{sample}/{SHAPE[0]}"
    desc = (f"FP64 oracle (numpy matmul per-axis DFT), forward+backward on {part} of the pencils "
            f"of each axis of the pme256 grid per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": list(SHAPE)},
        "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _flush(flush):
    flush.fill_(1.0)


def time_transform(croft, torch, stream, flush, plan, run_fwd, run_bwd, reps=5, warm=2):  # noqa: PLR0913
    """Median device ms of forward and backward (L2 flushed before each, no events between the passes),
    then the mean per-pass ms from `reps` further runs with per-pass events.  (An event recorded
    between two passes stops the next pass from launching early, so the whole-transform times
    are taken without them.)"""
    def once(fn, per_pass):
        with torch.cuda.stream(stream):
            _flush(flush)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
        pt = croft.croft_plan_pass_times(plan) if per_pass else []
        stream.synchronize()
        return a.elapsed_time(b), pt

    if plan:
        croft.croft_plan_set_timing(plan, False)
    fw, bw = [], []
    for i in range(warm + reps):
        tf, _ = once(run_fwd, False)
        tb, _ = once(run_bwd, False)
        if i >= warm:
            fw.append(tf)
            bw.append(tb)
    passes = []
    if plan:
        croft.croft_plan_set_timing(plan, True)
        for _ in range(reps):
            passes.append(once(run_fwd, True)[1])
            passes.append(once(run_bwd, True)[1])
        croft.croft_plan_set_timing(plan, False)
    np_ = len(passes[0]) if passes and passes[0] else 0
    pass_ms = [statistics.mean(p[i] for p in passes) for i in range(np_)]
    return statistics.median(fw), statistics.median(bw), pass_ms


ROW_NAMES = ("pme480_fp32", "pme384x360x320_fp32", "pme512_fp32", "pme512_tc_bf16x3", "pme256_convolve",
             "f64_128", "f64_1024", "batch96")


def measure_rows(croft, torch, dev, stream, flush, peak, only=None):  # noqa: PLR0915
    """The other hot-path rows, timed on device-generated data (timing does not depend on values):
    non-power-of-two meshes, FP32 vs tensor-core 512^3 (with the round-trip error of each),
    and the 96-grid batch (one persistent launch vs per-grid plans)."""
    import numpy as np

    import synthetic_inputs as S

    rows = {}
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)

    def grid(shape):
        return torch.complex(torch.rand(shape, device=dev, generator=gen) * 2 - 1,
                             torch.rand(shape, device=dev, generator=gen) * 2 - 1)

    def want(name):
        return only is None or name in only

    for name, shape, dtype in (("pme480_fp32", (480, 480, 480), 0), ("pme384x360x320_fp32", (384, 360, 320), 0),
                               ("pme512_fp32", (512, 512, 512), 0), ("pme512_tc_bf16x3", (512, 512, 512), 1)):
        if not want(name):
            continue
        x = grid(shape)
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        n = math.prod(shape)
        with croft.Plan(*shape, dtype=dtype) as p:
            croft.croft_plan_set_timing(p.handle, True)
            sh = stream.cuda_stream
            f_ms, b_ms, pass_ms = time_transform(
                croft, torch, stream, flush, p.handle,
                lambda: croft.croft_exec_forward(p.handle, x, y, sh),
                lambda: croft.croft_exec_backward(p.handle, y, z, sh))
            desc = p.describe()
        stream.synchronize()
        rt = float(torch.linalg.vector_norm((z - n * x).flatten()) / torch.linalg.vector_norm((n * x).flatten()))
        t = f_ms + b_ms
        cufft = None
        if dtype == 0:  # library context: cuFFT through torch.fft, same protocol
            del z
            cf, cb, _ = time_transform(croft, torch, stream, flush, None,
                                       lambda: torch.fft.fftn(x, norm="backward", out=y),
                                       lambda: torch.fft.ifftn(y, norm="forward"))
            cufft = {"ms_fwd": cf, "ms_bwd": cb, "gflops": 2 * nominal_flops(shape) / ((cf + cb) * 1e-3) / 1e9}
            z = None
        dom = max(range(len(pass_ms)), key=lambda i: pass_ms[i])
        rows[name] = {"shape": list(shape), "ms_fwd": f_ms, "ms_bwd": b_ms,
                      "gflops": 2 * nominal_flops(shape) / (t * 1e-3) / 1e9,
                      "hbm_frac_whole_transform": (32.0 * n / (t * 1e-3) / 1e9) / peak,
                      "pass_ms": pass_ms, "dominant_pass_gbs": 16.0 * n / (pass_ms[dom] * 1e-3) / 1e9,
                      "dominant_pass_frac": (16.0 * n / (pass_ms[dom] * 1e-3) / 1e9) / peak,
                      "roundtrip_rel_l2": rt, "plan": desc, "cufft_torch_fftn_context": cufft}
        del x, y, z
    if want("pme256_convolve"):
        # PME reciprocal-space convolution B(G * F(x)) on 256^3 with the smooth-PME influence function:
        # croft_exec_convolve (last-axis forward * G * backward fused) vs forward, a torch multiply, backward
        shape = (256, 256, 256)
        n = math.prod(shape)
        x = grid(shape)
        y = torch.empty_like(x)
        y2 = torch.empty_like(x)
        g = torch.from_numpy(S.pme_influence(shape)).to(dev)
        with croft.Plan(*shape) as p:
            sh = stream.cuda_stream
            t_conv, t_sep, pts = [], [], []
            for i in range(2 + 5 + 5):
                per_pass = i >= 7  # the last runs: per-pass events (kept out of the whole-pipeline times)
                croft.croft_plan_set_timing(p.handle, per_pass)
                for kind in ("conv", "sep"):
                    with torch.cuda.stream(stream):
                        _flush(flush)
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        if kind == "conv":
                            croft.croft_exec_convolve(p.handle, x, y, g, sh)
                        else:
                            croft.croft_exec_forward(p.handle, x, y2, sh)
                            y2.mul_(g)
                            croft.croft_exec_backward(p.handle, y2, y2, sh)
                        b.record(stream)
                    pt = croft.croft_plan_pass_times(p.handle, 16) if (kind == "conv" and per_pass) else None
                    stream.synchronize()
                    if 2 <= i < 7:
                        (t_conv if kind == "conv" else t_sep).append(a.elapsed_time(b))
                    if pt:
                        pts.append(pt)
            desc = p.describe()
        stream.synchronize()
        diff = float(torch.linalg.vector_norm((y - y2).flatten()) / torch.linalg.vector_norm(y2.flatten()))
        tc_ms, ts_ms = statistics.median(t_conv), statistics.median(t_sep)
        pass_ms = [statistics.mean(q[i] for q in pts) for i in range(len(pts[0]))] if pts else []
        rows["pme256_convolve"] = {
            "shape": list(shape), "ms": tc_ms, "gflops": 2 * nominal_flops(shape) / (tc_ms * 1e-3) / 1e9,
            "pass_ms": pass_ms,
            "fused_pass_ms": pass_ms[len(pass_ms) // 2] if pass_ms else None,
            "fused_pass_frac": ((20.0 * n / (pass_ms[len(pass_ms) // 2] * 1e-3) / 1e9) / peak) if pass_ms else None,
            "hbm_frac_compulsory": (20.0 * n / (tc_ms * 1e-3) / 1e9) / peak,
            "hbm_frac_passes": (84.0 * n / (tc_ms * 1e-3) / 1e9) / peak,
            "separate_ms": ts_ms, "speedup_vs_separate": ts_ms / tc_ms, "rel_diff_vs_separate": diff,
            "plan": desc,
            "notes": "fused: 4 plain passes (16N B each) + 1 fused pass (20N B: grid in/out + G); "
                     "separate: 6 passes + torch's multiply (20N B)"}
        del x, y, y2, g
    # complex128 at the paper's sizes (its Tables 1 and 3 time one double-complex forward transform)
    paper = {128: {"croft_best_s": 0.014, "croft_best_cores": 32, "fftw3_best_s": 0.019, "fftw3_best_cores": 32,
                   "source": "Table 1"},
             1024: {"croft_best_s": 1.2722, "croft_best_cores": 512, "fftw3_best_s": 4.7209, "fftw3_best_cores": 256,
                    "source": "Table 3"}}
    for n in (128, 1024):
        if not want(f"f64_{n}"):
            continue
        shape = (n, n, n)
        x = torch.complex(torch.rand(shape, device=dev, dtype=torch.float64, generator=gen) * 2 - 1,
                          torch.rand(shape, device=dev, dtype=torch.float64, generator=gen) * 2 - 1)
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        with croft.Plan(*shape, dtype=croft.CROFT_C2C_F64) as p:
            croft.croft_plan_set_timing(p.handle, True)
            sh = stream.cuda_stream
            f_ms, b_ms, pass_ms = time_transform(
                croft, torch, stream, flush, p.handle,
                lambda: croft.croft_exec_forward(p.handle, x, y, sh),
                lambda: croft.croft_exec_backward(p.handle, y, z, sh), reps=3 if n > 512 else 5, warm=1)
        stream.synchronize()
        nn = n ** 3
        rt = float(torch.linalg.vector_norm((z - nn * x).flatten()) / torch.linalg.vector_norm((nn * x).flatten()))
        rows[f"f64_{n}"] = {"shape": list(shape), "dtype": "f64", "ms_fwd": f_ms, "ms_bwd": b_ms,
                            "gflops_fwd": nominal_flops(shape) / (f_ms * 1e-3) / 1e9, "pass_ms": pass_ms,
                            "roundtrip_rel_l2": rt,
                            "paper_context": dict(paper[n], speedup_vs_croft_best=paper[n]["croft_best_s"] / (f_ms * 1e-3),
                                                  speedup_vs_fftw3_best=paper[n]["fftw3_best_s"] / (f_ms * 1e-3))}
        del x, y, z
    if want("batch96"):
        # the batch of 96 uneven PME meshes (seed-3 sizes), one persistent launch vs per-grid plans
        rng = np.random.default_rng(3)
        dims = [tuple(int(v) for v in r) for r in rng.choice(np.asarray(S.BATCH_AXIS_CHOICES), size=(96, 3))]
        xs = [grid(d) for d in dims]
        ys = [torch.empty_like(x) for x in xs]
        zs = [torch.empty_like(x) for x in xs]
        total = sum(math.prod(d) for d in dims)
        fl = sum(2 * nominal_flops(d) for d in dims)
        brow = {"grids": 96, "points": total, "bytes_per_grid_set": 8 * total}
        for mode, key in ((croft.CROFT_BATCH_ONE_LAUNCH, "one_launch"), (croft.CROFT_BATCH_PER_PASS, "per_pass"),
                          (croft.CROFT_BATCH_PER_GRID, "per_grid"), (croft.CROFT_BATCH_GROUPED, "grouped")):
            with croft.BatchPlan(dims, mode=mode) as bp:
                croft.croft_plan_set_timing(bp.handle, True)
                sh = stream.cuda_stream
                f_ms, b_ms, _ = time_transform(
                    croft, torch, stream, flush, bp.handle,
                    lambda: croft.croft_exec_batched_forward(bp.handle, xs, ys, sh),
                    lambda: croft.croft_exec_batched_backward(bp.handle, ys, zs, sh))
                launches = croft.croft_plan_num_launches(bp.handle)
            t = f_ms + b_ms
            brow[key] = {"ms_fwd": f_ms, "ms_bwd": b_ms, "gflops": fl / (t * 1e-3) / 1e9,
                         "hbm_frac_whole_transform": (32.0 * total / (t * 1e-3) / 1e9) / peak,
                         "launches_per_direction": launches}
        stream.synchronize()
        err = max(float(torch.linalg.vector_norm((z - math.prod(d) * x).flatten()) /
                        torch.linalg.vector_norm((math.prod(d) * x).flatten())) for d, x, z in zip(dims, xs, zs))
        brow["roundtrip_rel_l2_max"] = err
        # the autotuned plan (CROFT_BATCH_AUTO): times the four schedules on scratch buffers at
        # creation (a fresh cache file, so it measures) and keeps the fastest
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            old_cache = os.environ.get("CROFT_TUNE_CACHE")
            os.environ["CROFT_TUNE_CACHE"] = os.path.join(td, "tune.txt")
            try:
                t0 = time.perf_counter()
                bp = croft.BatchPlan(dims)
                t_tune = time.perf_counter() - t0
                with bp:
                    sh = stream.cuda_stream
                    f_ms, b_ms, _ = time_transform(
                        croft, torch, stream, flush, bp.handle,
                        lambda: croft.croft_exec_batched_forward(bp.handle, xs, ys, sh),
                        lambda: croft.croft_exec_batched_backward(bp.handle, ys, zs, sh))
                    desc = bp.describe()
            finally:
                if old_cache is None:
                    os.environ.pop("CROFT_TUNE_CACHE", None)
                else:
                    os.environ["CROFT_TUNE_CACHE"] = old_cache
        t = f_ms + b_ms
        brow["autotuned"] = {"ms_fwd": f_ms, "ms_bwd": b_ms, "gflops": fl / (t * 1e-3) / 1e9,
                             "plan_creation_s": t_tune, "plan": desc}
        rows["batch96"] = brow
    return rows


def library_context(torch, x, flush, stream, x_h, flops_step, skip_cpu):
    """cuFFT (torch.fft.fftn / ifftn, both unnormalised) forward+backward on the device grid, timed
    like the croft steps (L2 flushed, events at the ends); scipy.fft on the host cores."""
    out = {}
    times = []
    for i in range(8):
        with torch.cuda.stream(stream):
            _flush(flush)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            yf = torch.fft.fftn(x, norm="backward")
            torch.fft.ifftn(yf, norm="forward")
            b.record(stream)
        stream.synchronize()
        if i >= 3:
            times.append(a.elapsed_time(b))
    ms = statistics.median(times)
    out["cufft_torch_fftn"] = {"ms_per_step": ms, "gflops": flops_step / (ms * 1e-3) / 1e9,
                               "note": "torch.fft.fftn + ifftn(norm='forward') on the same 256^3 complex64 grid"}
    if not skip_cpu:
        try:
            import numpy as np
            import scipy.fft as sfft
            for name, dt in (("complex64", np.complex64), ("complex128", np.complex128)):
                xc = x_h.astype(dt)
                sfft.ifftn(sfft.fftn(xc, workers=os.cpu_count()), norm="forward", workers=os.cpu_count())
                t0 = time.perf_counter()
                reps = 0
                while True:
                    sfft.ifftn(sfft.fftn(xc, workers=os.cpu_count()), norm="forward", workers=os.cpu_count())
                    reps += 1
                    if time.perf_counter() - t0 > 3.0:
                        break
                sec = (time.perf_counter() - t0) / reps
                out[f"scipy_fft_{name}"] = {"ms_per_step": sec * 1e3, "gflops": flops_step / sec / 1e9,
                                             "cores": os.cpu_count()}
        except Exception as e:  # noqa: BLE001 - context only
            out["scipy_fft"] = {"unavailable": str(e)[:200]}
    return out


def run_croft(args):
    import numpy as np
    import torch

    import synthetic_inputs as S
    from paper_2002_04896_gb300 import build as _build

    _build.ensure_built()
    from paper_2002_04896_gb300 import croft

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    x_h = S.config_input("pme256")
    shape = x_h.shape
    n_total = math.prod(shape)
    flops_step = 2 * nominal_flops(shape)
    stream = torch.cuda.Stream(device=dev)
    x = torch.from_numpy(x_h).to(dev)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(2 * l2, 1 << 30) // 4, dtype=torch.float32, device=dev)

    sched = {"auto": None, "three_pass": croft.CROFT_SCHEDULE_THREE_PASS,
             "plane_fused": croft.CROFT_SCHEDULE_PLANE_FUSED, "slab_l2": croft.CROFT_SCHEDULE_SLAB_L2}[args.schedule]
    plan = croft.Plan(*shape, schedule=sched)
    plan_desc = plan.describe()
    launches_per_step = 2 * croft.croft_plan_num_launches(plan.handle)
    sh = stream.cuda_stream

    gap_fills = [1]

    def step(record):
        """One forward + backward; device time between two events (none between the passes)."""
        with torch.cuda.stream(stream):
            for _ in range(gap_fills[0]):
                flush.fill_(1.0)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            croft.croft_exec_forward(plan.handle, x, y, sh)
            croft.croft_exec_backward(plan.handle, y, z, sh)
            e[1].record(stream)
        stream.synchronize()
        if record is not None:
            record.append(e[0].elapsed_time(e[1]))

    def step_per_pass(record):
        """The same step with an event after every pass (per-kernel durations)."""
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            croft.croft_exec_forward(plan.handle, x, y, sh)
        pf = croft.croft_plan_pass_times(plan.handle)
        with torch.cuda.stream(stream):
            croft.croft_exec_backward(plan.handle, y, z, sh)
        pb = croft.croft_plan_pass_times(plan.handle)
        stream.synchronize()
        record.append((pf, pb))

    for _ in range(args.warmup):
        step(None)
    # Untimed L2-flush writes between timed steps keep the GPU busy so that the
    # timed region spans >= ~2 s of wall time: long enough for the clock samples
    # to describe it, without idle gaps that would let the clocks drop.
    with torch.cuda.stream(stream):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(10):
            flush.fill_(1.0)
        b.record(stream)
    stream.synchronize()
    t_fill = a.elapsed_time(b) / 10 * 1e-3
    gap_fills[0] = max(1, int(math.ceil(args.clock_window_s / max(1, args.steps) / t_fill)))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    rec = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        step(rec)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    # per-kernel durations: the same steps again with per-pass events, right after the timed ones
    croft.croft_plan_set_timing(plan.handle, True)
    rec_pp = []
    for _ in range(args.steps):
        step_per_pass(rec_pp)
    croft.croft_plan_set_timing(plan.handle, False)
    clk = clocks.stop()
    ms_total = max_over_ranks(torch, sum(rec), dev)
    ms_step = ms_total / args.steps
    value = job_gflops(world, flops_step, ms_step)

    # per-pass kernel times (forward and backward run the same kernels)
    npass = len(rec_pp[0][0])
    pass_ms = [statistics.mean([r[0][i] for r in rec_pp] + [r[1][i] for r in rec_pp]) for i in range(npass)]
    dom = max(range(npass), key=lambda i: pass_ms[i])
    axis_names = {3: ["z", "y", "x"], 2: ["yz", "x"], 1: ["yz"]}.get(npass, [f"p{i}" for i in range(npass)])
    peak, peak_kind = measured_peaks()
    alg_bytes = 16.0 * n_total  # one read + one write of the grid per pass launch
    # The per-pass events give each pass's share of a transform; an event between two
    # passes also adds a gap and stops the next pass from launching early, so the sum of
    # the per-pass times exceeds the timed step.  The dominant pass's duration inside the
    # timed steps = its share x the timed time of one transform.
    achieved_events = alg_bytes / (pass_ms[dom] * 1e-3) / 1e9
    dom_ms_in_step = pass_ms[dom] / sum(pass_ms) * (ms_step / 2)
    achieved = alg_bytes / (dom_ms_in_step * 1e-3) / 1e9
    dom_key = f"pass_{axis_names[dom]}_{'x'.join(map(str, shape))}"
    traffic = ncu_traffic(dom_key)

    # end to end through the C ABI with host buffers: every step uploads its input grid from
    # pinned memory, runs forward + backward and downloads the result; the library's host
    # pipeline overlaps the copies of one step with the transforms of its neighbours.
    x_pin = torch.from_numpy(x_h).pin_memory()
    z_pin = torch.empty_like(x_pin).pin_memory()
    ops = croft.CROFT_OP_FORWARD | croft.CROFT_OP_BACKWARD
    croft.croft_exec_host_pipeline(plan.handle, [x_pin] * args.warmup, [z_pin] * args.warmup, ops, stream)
    stream.synchronize()
    with torch.cuda.stream(stream):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        croft.croft_exec_host_pipeline(plan.handle, [x_pin] * args.steps, [z_pin] * args.steps, ops, stream)
        b.record(stream)
    stream.synchronize()
    e2e_ms = a.elapsed_time(b) / args.steps
    # the same with each step's copies and transforms serialised on one stream, for reference
    e2e_serial = []
    for i in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            x.copy_(x_pin, non_blocking=True)
            croft.croft_exec_forward(plan.handle, x, y, sh)
            croft.croft_exec_backward(plan.handle, y, z, sh)
            z_pin.copy_(z, non_blocking=True)
            b.record(stream)
        stream.synchronize()
        if i >= args.warmup:
            e2e_serial.append(a.elapsed_time(b))
    e2e_serial_ms = statistics.mean(e2e_serial)
    # the host link's own rate for this traffic: one step's upload and download at once, on two
    # streams, copy engines only (the pipelined e2e step cannot beat it)
    s2 = torch.cuda.Stream(device=dev)
    link = []
    for i in range(5):
        with torch.cuda.stream(stream):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s2.wait_event(a)
            x.copy_(x_pin, non_blocking=True)
        with torch.cuda.stream(s2):
            z_pin.copy_(z, non_blocking=True)
            c = torch.cuda.Event()
            c.record(s2)
        with torch.cuda.stream(stream):
            stream.wait_event(c)
            b.record(stream)
        stream.synchronize()
        if i >= 1:
            link.append(a.elapsed_time(b))
    link_ms = statistics.median(link)
    link_gbs = 16.0 * n_total / (link_ms * 1e-3) / 1e9
    e2e_ms = max_over_ranks(torch, e2e_ms, dev)
    e2e_val = job_gflops(world, flops_step, e2e_ms)
    zr = z_pin.numpy().astype(np.complex128)
    xr = x_h.astype(np.complex128) * n_total
    e2e_check = float(np.linalg.norm(zr - xr) / np.linalg.norm(xr))

    rows = None
    if rank == 0 and not args.no_rows:
        only = None if args.rows == "all" else set(args.rows.split(","))
        rows = measure_rows(croft, torch, dev, stream, flush, peak, only)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # whole forward+backward steps of the oracle, repeated for >= 10 s (at most 30 s)
        t0 = time.perf_counter()
        fl, reps = 0.0, 0
        while True:
            fl += cpu_oracle_step(x_h, None)
            reps += 1
            dt = time.perf_counter() - t0
            if dt >= 10.0 or dt * (reps + 1) / reps > 30.0:
                break
        cpu = {"value": fl / dt / 1e9, "unit": "GFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 oracle (numpy matmul per-axis DFT), {reps} full forward+backward step(s) of the "
                         f"pme256 grid in {dt:.1f} s"}

    # library context (not targets, not oracles): cuFFT through torch.fft on the same grid and
    # protocol, and a multi-threaded CPU FFT (scipy's pocketfft) on the host cores
    context = None
    if rank == 0 and not args.no_rows:
        context = library_context(torch, x, flush, stream, x_h, flops_step, args.no_cpu_baseline)

    plan.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(shape), "direction": "forward+backward",
                       "l2": "flushed before every step (writes of a 1 GiB buffer, > 2x L2, outside the timed events)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "passes_per_direction": npass, "schedule": args.schedule, "plan": plan_desc},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": dom_key,
                         "kernel_source_sha": kernel_source_sha(),
                         "peak_source": peak_kind, "alg_bytes_per_launch": alg_bytes,
                         "pass_ms": pass_ms, "dominant_ms_in_timed_step": dom_ms_in_step,
                         "achieved_per_pass_events": achieved_events,
                         "frac_per_pass_events": achieved_events / peak,
                         "kernel_timing": "per-pass shares from CUDA events on the launch stream after "
                                          f"every pass, over {args.steps} forward+backward steps run right "
                                          "after the timed ones; absolute duration = share x the timed "
                                          "time of one transform (an event between two passes adds a gap "
                                          "and stops the next pass from launching early, so the timed "
                                          "steps carry events only at their ends; achieved_per_pass_events "
                                          "is the same figure from the per-pass events alone)"},
            "hbm_frac_whole_transform": (16.0 * n_total * 2 / (ms_step * 1e-3) / 1e9) / peak,
            "cpu_baseline": cpu,
            "library_context": context,
            "e2e": {"value": e2e_val, "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * n_total,
                    "d2h_bytes_per_step": 8 * n_total, "ms_per_step": e2e_ms,
                    "api": "croft_exec_host_pipeline (upload, forward, backward, download per step; "
                           "steps overlapped on three streams)",
                    "roundtrip_rel_l2": e2e_check,
                    "serialised_ms_per_step": e2e_serial_ms,
                    "serialised_value": job_gflops(world, flops_step, e2e_serial_ms),
                    "link_roofline": {"bound": "host link", "achieved_gbs": 16.0 * n_total / (e2e_ms * 1e-3) / 1e9,
                                      "peak_gbs": link_gbs, "frac": link_ms / e2e_ms,
                                      "peak_source": "this step's upload and download copied at once on two "
                                                     "streams, measured here"}},
            "gpu_launches": launches_per_step * args.steps,
            "gpu_launches_note": "croft kernels inside the device-timed steps (the e2e region launches the same per step)",
            "rows": rows,
            "clocks": clk,
            "wall_s_timed_region": t_wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="croft", choices=["croft", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", default="auto", choices=["auto", "three_pass", "plane_fused", "slab_l2"])
    ap.add_argument("--no-rows", action="store_true", help="skip the extra per-row measurements")
    ap.add_argument("--rows", default="all",
                    help="comma-separated subset of the extra rows (" + ", ".join(ROW_NAMES) + ") or 'all'")
    ap.add_argument("--clock-window-s", type=float, default=2.0,
                    help="minimum wall time of the timed region, padded with untimed L2-flush writes "
                         "between steps (0 under a profiler)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_croft(args)


if __name__ == "__main__":
    sys.exit(main())
