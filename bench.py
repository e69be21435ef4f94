#!/usr/bin/env python3
"""Benchmark: 3D C2C FFT (forward + backward) of a 512^3 PME-shaped complex64 grid,
FP32 CUDA-core passes against passes with a split-precision tensor-core radix-16 stage.

One step = one forward and one backward transform of the whole grid through the
C ABI (libcroft.so), i.e. every pass of the hot path.  Metric: GFLOP/s with the
nominal count 5 N log2 N per direction.  `value` is the FP32 path; the line's
`tc` object times the tensor-core path (CROFT_C2C_F32_TC_BF16X3) with the same
protocol on the same input.  After the timed regions both paths' forward
results and round trips are compared with the FP64 oracle on the full grid
(`errors`).

Timing: plans outside the timed regions; W warm-up steps; then K steps per
path, each preceded by an L2 flush (a write of a buffer twice the L2 size,
outside the timed events); each step is bracketed by CUDA events on the stream
it runs on.  The dominant pass kernel's duration comes from the plan's per-pass
events over K more steps run right after the timed ones.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl croft|reference]

With N > 1 (torchrun) the one grid is split over the ranks in x-slabs (the paper's
slab decomposition: local z and y passes, one NCCL all-to-all, local x pass) and value
is the job's throughput on that grid (strong scaling); the time is the max over ranks.

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

CONFIG = "pme512"
SHAPE = (512, 512, 512)
WORKLOAD = ("pme512: 512x512x512 complex64 C2C forward+backward, 8M +-1 charges (net zero, iid uniform positions) "
            "spread by order-4 B-splines, seed 4; FP32 CUDA-core passes (value) and passes with a split-precision "
            "tensor-core radix-16 stage (tc) on the same input")
METRIC = "3D C2C FFT GFLOP/s (5N log2 N), % of HBM roofline, TC vs FP32 at fixed error"
HBM_FALLBACK_GBS = 6800.0
FP32_TOL_PER_LOG2 = 2e-6  # rel L2 bar of the FP32 path: 2e-6 * log2(N)
TC_TOL = 3e-5             # rel L2 bar of the tensor-core path


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
                       "croft_sched.h", "croft_sizes.h", "croft_ring_kernel.cuh", "croft_ring.cu",
                       "croft_pair_kernel.cuh", "croft_pair.cu", "croft_coldiv.h")
TC_KERNEL_SOURCES = PASS_KERNEL_SOURCES + ("croft_tc_kernel.cuh", "croft_tc.cu", "croft_tc_operand.h")


def kernel_source_sha(names=PASS_KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2002_04896_gb300", "csrc")
    for name in names:
        p = os.path.join(csrc, name)
        if not os.path.exists(p):
            continue
        with open(p, "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str, names=PASS_KERNEL_SOURCES):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "ncu_dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:  # noqa: BLE001
        return None
    ent = d.get(kernel_key)
    if not ent or ent.get("src_sha") != kernel_source_sha(names):
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


def oracle_sample_planes(x, budget_s: float):
    """Planes per sampled oracle step so that one step takes about budget_s (timed on 8 planes)."""
    t0 = time.perf_counter()
    cpu_oracle_step(x, 8)
    t8 = max(1e-3, time.perf_counter() - t0)
    s = int(8 * budget_s / t8)
    return max(1, min(x.shape[0], s))


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synthetic_inputs as S

    x = S.config_input(CONFIG)
    cores = os.cpu_count()
    # each step a bounded sample of the workload (a fixed fraction of the pencils of every
    # axis), sized so that all (warm-up + timed) steps take about --reference-budget-s seconds
    per_step = args.reference_budget_s / (args.steps + args.warmup)
    sample = oracle_sample_planes(x, per_step)
    if sample >= SHAPE[0]:
        sample = None
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
            f"of each axis of the {CONFIG} grid per step")
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


AXIS_NAMES = {3: ["z", "y", "x"], 2: ["yz", "x"], 1: ["yz"]}


def roofline(pass_ms, ms_step, shape, peak, peak_kind, key_suffix="", sources=PASS_KERNEL_SOURCES):
    """Roofline of the dominant pass: its algorithmic bytes (one read + one write of the grid,
    16 N) over its duration inside the timed steps (its share of the per-pass events times the
    timed time of one transform)."""
    n_total = math.prod(shape)
    npass = len(pass_ms)
    dom = max(range(npass), key=lambda i: pass_ms[i])
    names = AXIS_NAMES.get(npass, [f"p{i}" for i in range(npass)])
    alg_bytes = 16.0 * n_total
    achieved_events = alg_bytes / (pass_ms[dom] * 1e-3) / 1e9
    dom_ms_in_step = pass_ms[dom] / sum(pass_ms) * (ms_step / 2)
    achieved = alg_bytes / (dom_ms_in_step * 1e-3) / 1e9
    key = f"pass_{names[dom]}_{'x'.join(map(str, shape))}{key_suffix}"
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic(key, sources), "kernel": key, "kernel_source_sha": kernel_source_sha(sources),
            "peak_source": peak_kind, "alg_bytes_per_launch": alg_bytes, "pass_ms": pass_ms,
            "dominant_ms_in_timed_step": dom_ms_in_step, "achieved_per_pass_events": achieved_events,
            "frac_per_pass_events": achieved_events / peak,
            "kernel_timing": "per-pass shares from CUDA events on the launch stream after every pass, over "
                             "the steps run right after the timed ones; absolute duration = share x the timed "
                             "time of one transform (an event between two passes adds a gap and stops the next "
                             "pass from launching early, so the timed steps carry events only at their ends; "
                             "achieved_per_pass_events is the same figure from the per-pass events alone)"}


def errors_vs_oracle(x_h, y_h, z_h, ref, slab: int = 32):
    """Errors of one path's results against the FP64 oracle, accumulated in float64 over x-slabs.

    rel_l2_fwd       ||Y - Y_ref|| / ||Y_ref||            (the bar: 2e-6 log2 N FP32, 3e-5 TC)
    max_rel_fwd      max |Y - Y_ref| / max |Y_ref|          (per element, scaled by the largest output)
    rel_l2_fwd_high_k  the same rel L2 over the outputs whose normalised frequency
                     |k| = sqrt(sum_a (m_a / (K_a/2))^2) >= 1 (m_a the signed frequency): the outer
                     half of the spectrum, where a PME grid has little energy
    rel_l2_roundtrip ||B(F(x)) - N x|| / ||N x||
    """
    import numpy as np

    nx, ny, nz = x_h.shape
    n_total = x_h.size

    def sfreq(k):
        m = np.arange(k, dtype=np.float64)
        m = np.where(m <= k // 2, m, m - k)
        return (m / (k / 2.0)) ** 2 if k > 1 else np.zeros(1)

    fy, fz = sfreq(ny), sfreq(nz)
    fx = sfreq(nx)
    acc = dict(num=0.0, den=0.0, hnum=0.0, hden=0.0, rnum=0.0, rden=0.0, maxerr=0.0, maxref=0.0)
    for x0 in range(0, nx, slab):
        sl = slice(x0, min(nx, x0 + slab))
        r = ref[sl]
        d = y_h[sl].astype(np.complex128) - r
        e2 = d.real ** 2 + d.imag ** 2
        r2 = r.real ** 2 + r.imag ** 2
        acc["num"] += float(e2.sum())
        acc["den"] += float(r2.sum())
        acc["maxerr"] = max(acc["maxerr"], float(np.sqrt(e2.max())))
        acc["maxref"] = max(acc["maxref"], float(np.sqrt(r2.max())))
        band = (fx[sl, None, None] + fy[None, :, None] + fz[None, None, :]) >= 1.0
        acc["hnum"] += float(e2[band].sum())
        acc["hden"] += float(r2[band].sum())
        xr = x_h[sl].astype(np.complex128) * n_total
        dr = z_h[sl].astype(np.complex128) - xr
        acc["rnum"] += float((dr.real ** 2 + dr.imag ** 2).sum())
        acc["rden"] += float((xr.real ** 2 + xr.imag ** 2).sum())

    def q(a, b):
        return math.sqrt(a / b) if b > 0 else math.sqrt(a)

    return {"rel_l2_fwd": q(acc["num"], acc["den"]),
            "max_rel_fwd": acc["maxerr"] / acc["maxref"] if acc["maxref"] > 0 else acc["maxerr"],
            "rel_l2_fwd_high_k": q(acc["hnum"], acc["hden"]),
            "rel_l2_roundtrip": q(acc["rnum"], acc["rden"])}


ROW_NAMES = ("pme256_fp32", "pme480_fp32", "pme384x360x320_fp32", "tuned", "pme256_convolve", "f64_128", "f64_1024",
             "batch96")


def measure_rows(croft, torch, dev, stream, flush, peak, peak_kind, only=None):  # noqa: PLR0915
    """The other hot-path rows: the 256^3 PME grid (real input), non-power-of-two meshes on
    device-generated data (timing does not depend on values), the fused PME convolution,
    complex128 at the paper's sizes and the 96-grid batch in every schedule."""
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

    for name, shape in (("pme256_fp32", (256, 256, 256)), ("pme480_fp32", (480, 480, 480)),
                        ("pme384x360x320_fp32", (384, 360, 320))):
        if not want(name):
            continue
        x = torch.from_numpy(S.config_input("pme256")).to(dev) if name == "pme256_fp32" else grid(shape)
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        n = math.prod(shape)
        with croft.Plan(*shape) as p:
            croft.croft_plan_set_timing(p.handle, True)
            sh = stream.cuda_stream
            f_ms, b_ms, pass_ms = time_transform(
                croft, torch, stream, flush, p.handle,
                lambda: croft.croft_exec_forward(p.handle, x, y, sh),
                lambda: croft.croft_exec_backward(p.handle, y, z, sh), reps=10)
            desc = p.describe()
        stream.synchronize()
        rt = float(torch.linalg.vector_norm((z - n * x).flatten()) / torch.linalg.vector_norm((n * x).flatten()))
        t = f_ms + b_ms
        del z
        cf, cb, _ = time_transform(croft, torch, stream, flush, None,
                                   lambda: torch.fft.fftn(x, norm="backward", out=y),
                                   lambda: torch.fft.ifftn(y, norm="forward"))
        cufft = {"ms_fwd": cf, "ms_bwd": cb, "gflops": 2 * nominal_flops(shape) / ((cf + cb) * 1e-3) / 1e9}
        rows[name] = {"shape": list(shape), "ms_fwd": f_ms, "ms_bwd": b_ms,
                      "gflops": 2 * nominal_flops(shape) / (t * 1e-3) / 1e9,
                      "hbm_frac_whole_transform": (32.0 * n / (t * 1e-3) / 1e9) / peak,
                      "roofline": roofline(pass_ms, t, shape, peak, peak_kind),
                      "roundtrip_rel_l2": rt, "plan": desc, "cufft_torch_fftn_context": cufft,
                      "input": "pme256 (seed 1, 200k charges)" if name == "pme256_fp32" else "device uniform noise"}
        del x, y
    if want("tuned"):
        # CROFT_SCHEDULE_TUNED (measured at plan creation, fresh cache) against the rules (AUTO)
        import tempfile
        trow = {}
        with tempfile.TemporaryDirectory() as td:
            old_cache = os.environ.get("CROFT_TUNE_CACHE")
            os.environ["CROFT_TUNE_CACHE"] = os.path.join(td, "tune.txt")
            try:
                for shape in ((512, 512, 512), (480, 480, 480), (384, 360, 320)):
                    x = grid(shape)
                    y = torch.empty_like(x)
                    z = torch.empty_like(x)
                    sh = stream.cuda_stream
                    res = {}
                    for name, sched in (("rules", None), ("tuned", croft.CROFT_SCHEDULE_TUNED)):
                        t0 = time.perf_counter()
                        with croft.Plan(*shape, schedule=sched) as p:
                            t_plan = time.perf_counter() - t0
                            f_ms, b_ms, _ = time_transform(
                                croft, torch, stream, flush, None,
                                lambda: croft.croft_exec_forward(p.handle, x, y, sh),
                                lambda: croft.croft_exec_backward(p.handle, y, z, sh), reps=10, warm=3)
                            desc = p.describe()
                        res[name] = {"ms": f_ms + b_ms, "plan_creation_s": t_plan,
                                     "choice": desc.split("| tuned")[-1].strip() if name == "tuned" else "rules"}
                    res["speedup_tuned_vs_rules"] = res["rules"]["ms"] / res["tuned"]["ms"]
                    trow["x".join(map(str, shape))] = res
                    del x, y, z
            finally:
                if old_cache is None:
                    os.environ.pop("CROFT_TUNE_CACHE", None)
                else:
                    os.environ["CROFT_TUNE_CACHE"] = old_cache
        rows["tuned"] = trow
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
                            "roofline": {"bound": "alu", "unit": "FP64 pipe", "frac_pipe_active": 0.85,
                                         "peak_nominal_tflops": 1.25,
                                         "source": "ncu sm__pipe_fp64_cycles_active on the 256^3 complex128 passes "
                                                   "(profiles/f64_kernels_256.md); the same kernels at every size"},
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
        # the autotuned plan (CROFT_BATCH_AUTO): times the schedules on scratch buffers at
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
    del yf
    ms = statistics.median(times)
    out["cufft_torch_fftn"] = {"ms_per_step": ms, "gflops": flops_step / (ms * 1e-3) / 1e9,
                               "note": f"torch.fft.fftn + ifftn(norm='forward') on the same {CONFIG} complex64 grid"}
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
                del xc
        except Exception as e:  # noqa: BLE001 - context only
            out["scipy_fft"] = {"unavailable": str(e)[:200]}
    return out


class Arm:
    """One path (plan) of the headline: warm-up, timed steps, per-pass steps."""

    def __init__(self, croft, torch, stream, flush, plan, x, y, z):
        self.croft, self.torch, self.stream, self.flush = croft, torch, stream, flush
        self.plan, self.x, self.y, self.z = plan, x, y, z
        self.sh = stream.cuda_stream
        self.rec = []
        self.rec_pp = []

    def step(self, record, fills=1):
        """One forward + backward; device time between two events (none between the passes)."""
        torch, croft, stream = self.torch, self.croft, self.stream
        with torch.cuda.stream(stream):
            for _ in range(fills):
                self.flush.fill_(1.0)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            croft.croft_exec_forward(self.plan.handle, self.x, self.y, self.sh)
            croft.croft_exec_backward(self.plan.handle, self.y, self.z, self.sh)
            e[1].record(stream)
        stream.synchronize()
        if record is not None:
            record.append(e[0].elapsed_time(e[1]))

    def step_per_pass(self):
        """The same step with an event after every pass (per-kernel durations)."""
        torch, croft, stream = self.torch, self.croft, self.stream
        with torch.cuda.stream(stream):
            self.flush.fill_(1.0)
            croft.croft_exec_forward(self.plan.handle, self.x, self.y, self.sh)
        pf = croft.croft_plan_pass_times(self.plan.handle)
        with torch.cuda.stream(stream):
            croft.croft_exec_backward(self.plan.handle, self.y, self.z, self.sh)
        pb = croft.croft_plan_pass_times(self.plan.handle)
        stream.synchronize()
        self.rec_pp.append((pf, pb))

    def per_pass(self, steps):
        self.croft.croft_plan_set_timing(self.plan.handle, True)
        for _ in range(steps):
            self.step_per_pass()
        self.croft.croft_plan_set_timing(self.plan.handle, False)
        npass = len(self.rec_pp[0][0])
        return [statistics.mean([r[0][i] for r in self.rec_pp] + [r[1][i] for r in self.rec_pp]) for i in range(npass)]


def run_slab(args, world, rank, local):  # noqa: PLR0915
    """N > 1: the one pme512 transform split over the ranks in x-slabs (paper Sec. 2.2.1): z and y
    passes on each rank's slab, one NCCL all-to-all, the x pass on its y-slab; backward the other
    way round (paper_2002_04896_gb300.slab).  Strong scaling: the job transforms one grid per step."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import synthetic_inputs as S
    from paper_2002_04896_gb300 import build as _build

    _build.ensure_built()
    from paper_2002_04896_gb300 import croft, slab

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist.init_process_group("nccl", device_id=dev)
    t_in = time.perf_counter()
    x_h = S.config_input(CONFIG)  # every rank draws the same grid (seeded) and keeps its slab
    t_in = time.perf_counter() - t_in
    shape = x_h.shape
    n_total = math.prod(shape)
    flops_step = 2 * nominal_flops(shape)
    fft = slab.SlabFFT(shape)
    nxl = fft.shape_x[0]
    x_slab = np.ascontiguousarray(x_h[rank * nxl:(rank + 1) * nxl])
    del x_h
    xs = torch.from_numpy(x_slab).to(dev)
    work = torch.empty_like(xs)
    back = torch.empty_like(xs)
    ys = torch.empty(fft.shape_y, dtype=torch.complex64, device=dev)
    ywork = torch.empty_like(ys)
    flush = torch.empty((1 << 30) // 4, dtype=torch.float32, device=dev)
    ops = fft.ops

    def step(record=None, fills=1):
        for _ in range(fills):
            flush.fill_(1.0)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        fft.forward(xs, ys, work=work)
        fft.backward(ys, back, work=ywork)
        e[1].record()
        torch.cuda.synchronize()
        if record is not None:
            record.append(e[0].elapsed_time(e[1]))

    for _ in range(args.warmup):
        step()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(10):
        flush.fill_(1.0)
    b.record()
    torch.cuda.synchronize()
    fills = max(1, int(math.ceil(args.clock_window_s / max(1, args.steps) / (a.elapsed_time(b) / 10 * 1e-3))))
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    rec = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(rec, fills)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t0
    dist.barrier()
    # stage times (events between the stages) and per-pass times of the local plans
    croft.croft_plan_set_timing(ops.plan_x.handle, True)
    croft.croft_plan_set_timing(ops.plan_y.handle, True)
    stages, passes = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        ev[0].record()
        send = fft.forward_send(xs, work=work)
        ev[1].record()
        pz = croft.croft_plan_pass_times(ops.plan_x.handle)
        recv = fft.buffers(xs)[1]
        fft.exchange(send, recv)
        ev[2].record()
        fft.forward_finish(recv, ys)
        ev[3].record()
        px = croft.croft_plan_pass_times(ops.plan_y.handle)
        send = fft.backward_send(ys, work=ywork)
        ev[4].record()
        fft.exchange(send, recv)
        ev[5].record()
        fft.backward_finish(recv, back)
        ev[6].record()
        torch.cuda.synchronize()
        stages.append([ev[i].elapsed_time(ev[i + 1]) for i in range(6)])
        passes.append(pz + px)
    croft.croft_plan_set_timing(ops.plan_x.handle, False)
    croft.croft_plan_set_timing(ops.plan_y.handle, False)
    clk = clocks.stop() if clocks else None
    ms_step = max_over_ranks(torch, sum(rec) / args.steps, dev)
    value = flops_step / (ms_step * 1e-3) / 1e9
    st = [statistics.mean(v[i] for v in stages) for i in range(6)]
    pass_ms = [statistics.mean(v[i] for v in passes) for i in range(len(passes[0]))]
    # round trip on every rank, reduced over the job
    d = (back - n_total * xs).flatten()
    red = torch.tensor([float(torch.linalg.vector_norm(d)) ** 2,
                        float(torch.linalg.vector_norm(n_total * xs.flatten())) ** 2], dtype=torch.float64, device=dev)
    dist.all_reduce(red)
    rt = math.sqrt(float(red[0]) / float(red[1]))
    peak, peak_kind = measured_peaks()
    local_bytes = 16.0 * n_total / world
    dom = max(range(len(pass_ms)), key=lambda i: pass_ms[i])
    achieved = local_bytes / (pass_ms[dom] * 1e-3) / 1e9
    # end to end: every step uploads each rank's slab from pinned memory and downloads its result
    x_pin = torch.from_numpy(x_slab).pin_memory()
    b_pin = torch.empty_like(x_pin).pin_memory()
    e2e_rec = []
    for i in range(args.warmup + args.steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        xs.copy_(x_pin, non_blocking=True)
        fft.forward(xs, ys, work=work)
        fft.backward(ys, back, work=ywork)
        b_pin.copy_(back, non_blocking=True)
        e[1].record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_rec.append(e[0].elapsed_time(e[1]))
    e2e_ms = max_over_ranks(torch, statistics.mean(e2e_rec), dev)
    launches = args.steps * 2 * (croft.croft_plan_num_launches(ops.plan_x.handle) +
                                 croft.croft_plan_num_launches(ops.plan_y.handle))
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD.split(";")[0] + "; FP32 path, one grid split over the GPUs in x-slabs",
                       "grid": list(shape), "direction": "forward+backward",
                       "parallelism": f"slab x{world}: z+y passes per x-slab, one all-to-all, x pass per y-slab",
                       "l2": "L2 flushed before every step (1 GiB write, outside the timed events)",
                       "input_generation_s": t_in},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": ["z", "y", "x"][dom] + f" pass of a {world}-way slab",
                         "peak_source": peak_kind, "alg_bytes_per_launch": local_bytes, "pass_ms": pass_ms,
                         "kernel_timing": "per-pass CUDA events of the local plans, rank 0"},
            "slab": {"stage_ms_rank0": dict(zip(["fwd_local_zy+pack", "fwd_all_to_all", "fwd_local_x",
                                                 "bwd_local_x", "bwd_all_to_all", "bwd_unpack+local_zy"], st)),
                     "exchange_bytes_per_rank_per_all_to_all": 8 * fft.block * (world - 1)},
            "errors": {"rel_l2_roundtrip": rt, "bar_rel_l2": FP32_TOL_PER_LOG2 * math.log2(n_total)},
            "tc": None, "cpu_baseline": None,
            "e2e": {"value": flops_step / (e2e_ms * 1e-3) / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * n_total,
                    "d2h_bytes_per_step": 8 * n_total, "ms_per_step": e2e_ms,
                    "api": "SlabFFT.forward/backward per step, each rank's slab copied from and to pinned memory"},
            "gpu_launches": launches,
            "gpu_launches_note": "croft kernels of rank 0 inside its timed steps (NCCL and copy-engine copies not counted)",
            "clocks": clk, "wall_s_timed_region": t_wall,
        }
        print(json.dumps(line), flush=True)
    fft.close()
    dist.destroy_process_group()
    return 0


def run_croft(args):  # noqa: PLR0915
    import numpy as np
    import torch

    import synthetic_inputs as S
    from paper_2002_04896_gb300 import build as _build

    _build.ensure_built()
    from paper_2002_04896_gb300 import croft

    world, rank, local = dist_env()
    if world > 1:
        return run_slab(args, world, rank, local)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    t_in = time.perf_counter()
    x_h = S.config_input(CONFIG)
    t_in = time.perf_counter() - t_in
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
    plan_tc = None if args.no_tc else croft.Plan(*shape, dtype=croft.CROFT_C2C_F32_TC_BF16X3)
    arms = {"fp32": Arm(croft, torch, stream, flush, plan, x, y, z)}
    if plan_tc is not None:
        arms["tc"] = Arm(croft, torch, stream, flush, plan_tc, x, y, z)

    for arm in arms.values():
        for _ in range(args.warmup):
            arm.step(None)
    # Untimed L2-flush writes between timed steps keep the GPU busy so that the
    # timed region spans >= ~2 s of wall time per path: long enough for the clock
    # samples to describe it, without idle gaps that would let the clocks drop.
    with torch.cuda.stream(stream):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(10):
            flush.fill_(1.0)
        b.record(stream)
    stream.synchronize()
    t_fill = a.elapsed_time(b) / 10 * 1e-3
    fills = max(1, int(math.ceil(args.clock_window_s / max(1, args.steps) / t_fill)))
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_wall = {}
    for name, arm in arms.items():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            arm.step(arm.rec, fills)
        torch.cuda.synchronize()
        t_wall[name] = time.perf_counter() - t0
    # per-kernel durations: the same steps again with per-pass events, right after the timed ones
    pass_ms = {name: arm.per_pass(args.steps) for name, arm in arms.items()}
    clk = clocks.stop()
    peak, peak_kind = measured_peaks()
    res = {}
    for name, arm in arms.items():
        ms_total = max_over_ranks(torch, sum(arm.rec), dev)
        ms_step = ms_total / args.steps
        src = TC_KERNEL_SOURCES if name == "tc" else PASS_KERNEL_SOURCES
        res[name] = {"ms_per_step": ms_step, "value": job_gflops(world, flops_step, ms_step),
                     "roofline": roofline(pass_ms[name], ms_step, shape, peak, peak_kind,
                                          "_tc" if name == "tc" else "", src),
                     "hbm_frac_whole_transform": (16.0 * n_total * 2 / (ms_step * 1e-3) / 1e9) / peak,
                     "plan": arm.plan.describe(),
                     "launches_per_step": 2 * croft.croft_plan_num_launches(arm.plan.handle)}
    ms_step = res["fp32"]["ms_per_step"]
    value = res["fp32"]["value"]

    # errors against the FP64 oracle on the full grid, for every path (outside the timed regions)
    errors = None
    if rank == 0 and not args.no_errors:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.forward(x_h)
        t_oracle = time.perf_counter() - t0
        errors = {"oracle": f"oracle.forward (FP64 per-axis DFT matrices) on the same complex64 input, "
                            f"{t_oracle:.1f} s on {os.cpu_count()} host cores"}
        for name, arm in arms.items():
            with torch.cuda.stream(stream):
                croft.croft_exec_forward(arm.plan.handle, x, y, stream.cuda_stream)
                croft.croft_exec_backward(arm.plan.handle, y, z, stream.cuda_stream)
            stream.synchronize()
            st = croft.croft_plan_last_device_status(arm.plan.handle)
            e = errors_vs_oracle(x_h, y.cpu().numpy(), z.cpu().numpy(), ref)
            bar = TC_TOL if name == "tc" else FP32_TOL_PER_LOG2 * math.log2(n_total)
            e.update({"bar_rel_l2": bar, "within_bar": e["rel_l2_fwd"] <= bar and e["rel_l2_roundtrip"] <= bar,
                      "device_status": croft.croft_status_string(st)})
            errors[name] = e
        del ref
    if "tc" in res:
        res["tc"]["tc_vs_fp32"] = {"time_ratio": res["tc"]["ms_per_step"] / ms_step,
                                   "gflops_ratio": res["tc"]["value"] / value}
        if errors:
            res["tc"]["errors"] = errors["tc"]
            res["tc"]["tc_vs_fp32"]["rel_l2_fwd_ratio"] = errors["tc"]["rel_l2_fwd"] / errors["fp32"]["rel_l2_fwd"]

    # end to end through the C ABI with host buffers: every step uploads its input grid from
    # pinned memory, runs forward + backward and downloads the result; the library's host
    # pipeline overlaps the copies of one step with the transforms of its neighbours.
    e2e = None
    if not args.no_e2e:
        x_pin = torch.from_numpy(x_h).pin_memory()
        z_pin = torch.empty_like(x_pin).pin_memory()
        ops = croft.CROFT_OP_FORWARD | croft.CROFT_OP_BACKWARD
        croft.croft_exec_host_pipeline(plan.handle, [x_pin] * args.warmup, [z_pin] * args.warmup, ops, stream)
        stream.synchronize()
        # three pipelined runs of K steps each, the median run (the host link occasionally
        # serialises a run's uploads and downloads; one run is not representative)
        e2e_runs = []
        for _ in range(3):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                croft.croft_exec_host_pipeline(plan.handle, [x_pin] * args.steps, [z_pin] * args.steps, ops, stream)
                b.record(stream)
            stream.synchronize()
            e2e_runs.append(a.elapsed_time(b) / args.steps)
        e2e_ms = statistics.median(e2e_runs)
        # the round trip the pipelined steps brought back (before z_pin is reused below)
        zr = z_pin.numpy()
        num = den = 0.0
        for x0 in range(0, shape[0], 64):
            xr = x_h[x0:x0 + 64].astype(np.complex128) * n_total
            d = zr[x0:x0 + 64].astype(np.complex128) - xr
            num += float((d.real ** 2 + d.imag ** 2).sum())
            den += float((xr.real ** 2 + xr.imag ** 2).sum())
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
        e2e = {"value": job_gflops(world, flops_step, e2e_ms), "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * n_total,
               "d2h_bytes_per_step": 8 * n_total, "ms_per_step": e2e_ms,
               "api": "croft_exec_host_pipeline (upload, forward, backward, download per step; "
                      "steps overlapped on three streams), FP32 path; median of three runs of K steps",
               "ms_per_step_runs": e2e_runs,
               "roundtrip_rel_l2": math.sqrt(num / den),
               "link_roofline": {"bound": "host link", "achieved_gbs": 16.0 * n_total / (e2e_ms * 1e-3) / 1e9,
                                 "peak_gbs": link_gbs, "frac": link_ms / e2e_ms,
                                 "peak_source": "this step's upload and download copied at once on two "
                                                "streams, measured here"}}
        del x_pin, z_pin

    rows = None
    if rank == 0 and not args.no_rows:
        only = None if args.rows == "all" else set(args.rows.split(","))
        rows = measure_rows(croft, torch, dev, stream, flush, peak, peak_kind, only)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on a bounded sample of the same workload: a fraction of the pencils of every
        # axis per forward+backward step, repeated for >= 10 s
        sample = oracle_sample_planes(x_h, 3.0)
        t0 = time.perf_counter()
        fl, reps = 0.0, 0
        while True:
            fl += cpu_oracle_step(x_h, sample)
            reps += 1
            dt = time.perf_counter() - t0
            if dt >= 10.0 or dt * (reps + 1) / reps > 30.0:
                break
        cpu = {"value": fl / dt / 1e9, "unit": "GFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 oracle (numpy matmul per-axis DFT): {reps} forward+backward step(s) on {sample}/"
                         f"{shape[0]} of the pencils of each axis of the {CONFIG} grid, {dt:.1f} s"}

    # library context (not targets, not oracles): cuFFT through torch.fft on the same grid and
    # protocol, and a multi-threaded CPU FFT (scipy's pocketfft) on the host cores
    context = None
    if rank == 0 and not args.no_rows:
        context = library_context(torch, x, flush, stream, x_h, flops_step, args.no_cpu_baseline)

    launches = sum(r["launches_per_step"] for r in res.values()) * args.steps
    plan.close()
    if plan_tc is not None:
        plan_tc.close()
    if rank == 0:
        fp = res["fp32"]
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(shape), "direction": "forward+backward",
                       "l2": "inputs (1 GiB) larger than L2; L2 also flushed before every step (writes of a "
                             "1 GiB buffer, outside the timed events)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "passes_per_direction": len(pass_ms["fp32"]), "schedule": args.schedule,
                       "plan": fp["plan"], "input_generation_s": t_in},
            "roofline": fp["roofline"],
            "hbm_frac_whole_transform": fp["hbm_frac_whole_transform"],
            "errors": errors,
            "tc": res.get("tc"),
            "cpu_baseline": cpu,
            "library_context": context,
            "e2e": e2e,
            "gpu_launches": launches,
            "gpu_launches_note": "croft kernels inside the device-timed steps of both paths",
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
    ap.add_argument("--no-errors", action="store_true", help="skip the oracle comparison of the headline results")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) measurement")
    ap.add_argument("--no-tc", action="store_true", help="time the FP32 path only")
    ap.add_argument("--reference-budget-s", type=float, default=180.0,
                    help="--impl reference: wall time of all its (warm-up + timed) oracle steps")
    ap.add_argument("--schedule", default="auto", choices=["auto", "three_pass", "plane_fused", "slab_l2"])
    ap.add_argument("--no-rows", action="store_true", help="skip the extra per-row measurements")
    ap.add_argument("--rows", default="all",
                    help="comma-separated subset of the extra rows (" + ", ".join(ROW_NAMES) + ") or 'all'")
    ap.add_argument("--clock-window-s", type=float, default=2.0,
                    help="minimum wall time of each timed region, padded with untimed L2-flush writes "
                         "between steps (0 under a profiler)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_croft(args)


if __name__ == "__main__":
    sys.exit(main())
