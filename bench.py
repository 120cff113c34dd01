#!/usr/bin/env python3
"""Benchmark of the permutation-avoiding FFT convolution on GB300.

One step = one whole convolution y = conj(A)((A^T x) o Hhat) of the main
workload (default: 2-D periodic convolution 3125^2, complex FP64, radix 5,
stage list [5,5,5,5,5] per axis, separable exponential filter spectrum
resident), inputs resident in HBM, L2 flushed (512 MiB write) before every
step outside the timed events.

Metric: GB/s of compulsory traffic B = 3 N S per convolution (read x, read
the resident spectrum, write y; N = 3125^2, S = 16 bytes), next to the same
GPU running the permuted form (same kernels plus explicit index-reversal
passes) and a cuFFT-based convolution, with the FP64 oracle timed on the
host and the result's relative L2 error against it.  Complex FP64 passes are
bound by GB300's FP64 pipe, so the line's roofline is the ALU one (flops
2 c_r N log2 N + 6 N over the FP64 peak), with the HBM fraction beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pac|reference]
                    [--workload conv2d-r5|conv2d-r3|conv3d|conv1d] [--dtype c128|c64|c128df]

With N > 1 (launched by torch.distributed.run) every rank runs an
independent replica on its own GPU; value = all ranks' bytes / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# One hardware work queue per stream for the serving queue's request streams
# (read when CUDA starts; the default of 8 lets a small request's kernels
# queue behind a large request's on a shared hardware queue: measured p99 of
# small FP32 requests 26 -> 8.3 ms).  A value the caller set is kept.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "perm-free conv GB/s & %HBM roofline vs permuted path; served p50/p99 latency"
UNIT = "GB/s"
FLUSH_BYTES = 512 << 20


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["pac", "reference"], default="pac")
    ap.add_argument("--radix", type=int, default=4, help="radix of the conv3d workload")
    ap.add_argument("--dtype", choices=["c64", "c128", "c128df"], default="c128",
                    help="c128df (complex FP64 arrays in double-float arithmetic) runs with --quick only")
    ap.add_argument("--n", type=int, default=128, help="edge of the 3-D cube")
    ap.add_argument("--workload", choices=["conv3d", "conv2d-r3", "conv2d-r5", "conv1d"], default="conv2d-r5",
                    help="the main leg's problem (default: the 2-D 3125^2 radix-5 workload)")
    ap.add_argument("--quick", action="store_true", help="main leg only (for profiler runs)")
    ap.add_argument("--profile-path", choices=["none", "permuted", "single", "mixed", "pfa", "batched"], default="none",
                    help="profiler runs: time one other path instead of the main line and print its times "
                         "(permuted: the comparator on the main workload; single: the one-launch cooperative "
                         "form of 3-D 128^3 FP32 radix 4; mixed: 2-D 1000^2 FP32 with groups spanning prime "
                         "bases; pfa: the prime factor form of 1-D 2^10 3^5 5^3 FP32; batched: --batch instances of "
                         "the batched workload in one pac_convolve_many call)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline and the oracle checks")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--legs", default="configs,batched,served",  # "none": the main leg only
                    help="extra legs after the main one: configs (every workload shape, dtype and radix, "
                         "with its permuted form and cuFFT), batched (4096 mixed convolutions in one call), "
                         "served (Poisson request stream through the queue)")
    ap.add_argument("--max-inflight", type=int, default=16, help="served leg: requests running at once")
    ap.add_argument("--serve-repeats", type=int, default=5, help="served leg: times the request stream is served")
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default pass schedules)")
    ap.add_argument("--flush-mb", type=int, default=FLUSH_BYTES >> 20,
                    help="L2 flush buffer written before each step (0: none, for profiler runs only)")
    args = ap.parse_args(argv)
    if args.dtype == "c128df" and not args.quick:
        ap.error("--dtype c128df runs with --quick (the full line compares entry points that take FP64 plans)")
    return args


# ------------------------------------------------------------------ ranks


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(local_ms: float, local_units: float, world: int, device=None):
    """Max time and summed work over ranks (replicas): returns (max_ms, total_units)."""
    if world <= 1:
        return local_ms, local_units
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []  # (t, sm_mhz, max_mhz, reasons)
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            reasons = []
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                 parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.append(name)
            self.samples.append((time.time(), sm, mx, reasons))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        inside = [s for s in self.samples if t0 <= s[0] <= t1]
        note = None
        if not inside:  # the timed window fell between two samples: take the nearest
            inside = [min(self.samples, key=lambda s: min(abs(s[0] - t0), abs(s[0] - t1)))]
            note = "nearest sample to the timed window"
        reasons = sorted({r for s in inside for r in s[3]})
        out = {"sm_mhz": statistics.median(s[1] for s in inside), "sm_max_mhz": max(s[2] for s in inside),
               "reasons": reasons, "samples": len(inside)}
        if note:
            out["note"] = note
        return out


# ------------------------------------------------------------------ timing


def time_steps(torch, fn, steps, warmup, flush, stream):
    """Run warmup + steps calls of fn on `stream`, flushing L2 before each;
    returns per-step device times (ms) from CUDA events on that stream."""
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush()
            fn()
        stream.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            flush()
            starts[i].record(stream)
            fn()
            ends[i].record(stream)
        stream.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


# sources that define the pass and plane kernels and their launch shapes
KERNEL_SOURCES = ("fft_device.cuh", "config.h", "pass_args.h", "roots.h", "kern_launch.cuh", "kern_c64_p2.cu",
                  "kern_c128_p2.cu", "kern_plane.cu")


def source_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2506_12718_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")  # JSON text
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = data.get(workload, {}).get(kernel)
    if not ent or ent.get("source_hash") != source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def measured_peak_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ------------------------------------------------------- roofline arithmetic

# ALU peaks from the GB300's unit counts and maximum SM clock: 152 SMs at
# 2070 MHz; FP64: 2 fused multiply-adds per clock per SM (4 flops), i.e.
# 1.26 TFLOP/s, GB300's published FP64 rate of 1.25 TFLOP/s; FP32: 128 FMA
# lanes per SM (256 flops per clock), 80.5 TFLOP/s.  The FMA probe of the
# library (pac_measure_fma_peak) is reported beside them.
SMS, SM_MAX_MHZ = 152, 2070.0
ALU_PEAK_GFLOPS = {"c128": SMS * SM_MAX_MHZ * 4 / 1e3, "c64": SMS * SM_MAX_MHZ * 256 / 1e3}

# Flops per point and log2 of the length of one transform, c_r in
# c_r N log2 N: the paper's counts for radix 2, 4, 8 (5, 4.25, 4.08; Section
# 5); for powers of 3 and 5 the estimate (flops(DFT_p) + 6 (p - 1)) / p per
# point and stage over log2 p (16-flop DFT_3, 44-flop DFT_5: 5.9 both).  One
# count per prime base, whatever radix label a plan carries: the smallest of
# base 2's (4.08), since radix 2, 4 and 8 plans of the same size run the
# same rounds here.
C_BASE = {2: 4.08, 3: 5.9, 5: 5.9}


def c_r_of(dims) -> float:
    """c_r of a problem: the per-base counts weighted by each base's share of log2 N."""
    tot, acc = 0.0, 0.0
    for n in dims:
        for p in (2, 3, 5):
            while n % p == 0:
                n //= p
                acc += C_BASE[p] * math.log2(p)
                tot += math.log2(p)
    return acc / tot if tot else C_BASE[2]


def alg_flops(dims) -> float:
    """Algorithmic flops of one convolution with the spectrum resident: a forward
    and an inverse transform (c_r N log2 N each) and the product (6 N)."""
    N = math.prod(dims)
    return 2 * c_r_of(dims) * N * math.log2(N) + 6 * N if N > 1 else 6.0


def launch_table(pac, plan, c):
    """Per launch of pac_convolve, in launch order: (kernel instantiation as ncu
    lists it, algorithmic bytes, algorithmic flops).  A pass over group g
    (size M) moves 2 N S and computes c_r N log2 M; the fused pass (forward,
    product, inverse of the last group) and the plane pass (the last two
    groups) move 3 N S and compute twice that plus the product's 6 N."""
    N, S = c.n_total, c.elem_bytes
    cr = c_r_of(c.dims)
    cap = plan.query(pac.Q_GROUP_CAP)
    groups = pac.pac_plan_groups(c.dims, c.radix, 0 if c.dtype == "c64" else 1, False, cap)
    G = len(groups)
    if G != plan.query(pac.Q_GROUPS):  # a schedule the host hook does not reproduce
        return None
    V = "float2" if c.dtype == "c64" else "double2"
    plane = plan.query(pac.Q_PLANE) > 0

    def one(g):
        return (f"pass_kernel<{V},{groups[g][1]},{'lines' if g == G - 1 else 'rows'}>", 2 * N * S,
                cr * N * math.log2(groups[g][1]))

    if plane and G >= 2:
        m1, m2 = groups[G - 2][1], groups[G - 1][1]
        mid = [(f"plane_kernel<{V},{m1},{m2}>", 3 * N * S, 2 * cr * N * math.log2(m1 * m2) + 6 * N)]
        outer = list(range(G - 2))
    else:
        mg = groups[G - 1][1]
        mid = [(f"pass_kernel<{V},{mg},lines>", 3 * N * S,
                2 * cr * N * math.log2(mg) + 6 * N)]
        outer = list(range(G - 1))
    return [one(g) for g in outer] + mid + [one(g) for g in reversed(outer)]


def tolerance(c) -> float:
    """Relative L2 tolerance: 1e-12 for complex FP64 arrays (computed in FP64
    or in double-float arithmetic), 1e-5 log2 N for complex FP32."""
    return 1e-12 if c.dtype in ("c128", "c128df") else 1e-5 * math.log2(max(2, c.n_total))


def oracle_run(c, x, h, fs, points=None):
    """One oracle evaluation of problem c (as it stands, on the threads set):
    O2 over the whole array for a separable filter when points is None, else
    O1 at the given output indices.  Returns (values, seconds, description)."""
    import oracle
    t0 = time.perf_counter()
    if points is None:
        ref = oracle.conv_separable(fs, x) if fs is not None else oracle.conv_direct(h, x)
        what = ("separable-direct convolution over the whole array (oracle route O2, FP64)" if fs is not None
                else "direct definition over the whole array (oracle route O1, FP64)")
    else:
        ref = oracle.conv_direct_points(h, x, points)
        what = f"direct definition at {len(points)} seeded output points (oracle route O1, FP64)"
    return ref, time.perf_counter() - t0, what


def oracle_check(c, x, h, fs, y, whole_macs=7e10, point_macs=1e10, cache=None):
    """Relative L2 error of the GPU result y against the FP64 oracle, with the
    oracle's time on all host cores and on one core (the CPU baseline of
    problem c).  Route: O2 over the whole array when the filter is separable
    and that takes at most whole_macs multiply-adds (O1 over the whole array
    for a non-separable filter within the same bound), else O1 at
    P = point_macs / N seeded points (64 <= P <= 4096).  One core: the same
    route when it would take at most about 6 s, else O1 at a smaller seeded
    sample, timed on one core and on all cores.  GB/s = 3 N S per whole
    convolution over the time, scaled by the computed fraction of outputs."""
    import oracle
    # the same inputs (and oracle) for FP64 and double-float plans of one workload
    key = (c.dims, "c128" if c.dtype == "c128df" else c.dtype, c.x_kind, c.h_kind, c.seed, c.h_seed, c.h_param)
    if cache is not None and key in cache:  # same inputs (e.g. one shape at several radices)
        ref, pts, base = cache[key]
        yv = np.asarray(y, dtype=np.complex128).reshape(-1)
        err = oracle.rel_l2(yv if pts is None else yv[pts], ref.reshape(-1))
        return {**base, "rel_l2_vs_oracle": err, "within_tolerance": bool(err <= base["tolerance"])}
    N, S = c.n_total, c.elem_bytes
    B = 3 * N * S
    cores = oracle.num_threads()
    macs_whole = N * (sum(c.dims) if fs is not None else N)
    yv = np.asarray(y, dtype=np.complex128).reshape(-1)
    if macs_whole <= whole_macs:
        pts = None
        ref, dt, what = oracle_run(c, x, h, fs)
        err = oracle.rel_l2(yv, ref.reshape(-1))
        frac, macs = 1.0, macs_whole
    else:
        npts = int(min(4096, max(64, point_macs // N)))
        pts = pin_sample(N, npts, 9000 + N % 9973)
        ref, dt, what = oracle_run(c, x, h, fs, pts)
        err = oracle.rel_l2(yv[pts], ref)
        frac, macs = npts / N, N * npts
    out = {"rel_l2_vs_oracle": err, "tolerance": tolerance(c), "within_tolerance": bool(err <= tolerance(c)),
           "oracle_route": what,
           "cpu_oracle": {"all_cores": {"cores": cores, "s": dt, "GBps": B * frac / dt / 1e9, "route": what}}}
    oracle.set_threads(1)
    try:
        if dt * cores <= 6.0:
            _, dt1, what1 = oracle_run(c, x, h, fs, pts)
            out["cpu_oracle"]["one_core"] = {"cores": 1, "s": dt1, "GBps": B * frac / dt1 / 1e9, "route": what1}
        else:
            n1 = int(max(1, min(4096, 4e8 // N)))
            p1 = pin_sample(N, n1, 7000 + N % 9973)
            _, dt1, what1 = oracle_run(c, x, h, fs, p1)
            oracle.set_threads(cores)
            _, dta, _ = oracle_run(c, x, h, fs, p1)
            out["cpu_oracle"]["one_core"] = {"cores": 1, "s": dt1, "GBps": B * n1 / N / dt1 / 1e9, "route": what1,
                                             "same_sample_all_cores": {"cores": cores, "s": dta,
                                                                       "GBps": B * n1 / N / dta / 1e9}}
    finally:
        oracle.set_threads(cores)
    if cache is not None:
        cache[key] = (ref, pts, {k: v for k, v in out.items() if k not in ("rel_l2_vs_oracle", "within_tolerance")})
    return out


def pin_sample(n_total, count, seed):
    import pac_inputs as pin
    return pin.sample_points(n_total, count, seed)


# --------------------------------------------------------------- the legs


def roofline_block(a, torch, pac, plan, c, x, y, stream, flush, ms_per_step, peak, peak_kind):
    """The line's roofline.  Whole step (reproducible from the line's value):
    complex FP64 is bound by the FP64 pipe, so bound = alu with frac =
    flops / t / FP64 peak; complex FP32 is bound by HBM, frac = 3 N S / t /
    the measured copy peak.  Both fractions are given.  The dominant kernel
    (most device time per step, by CUDA events around each launch on the
    launching stream) is described per launch: algorithmic flops and bytes,
    its ALU fraction and its pass-model HBM fraction (bytes the pass itself
    must move, not the compulsory 3 N S of the convolution), and the ncu DRAM
    traffic of one launch when the committed capture matches the sources."""
    N, S = c.n_total, c.elem_bytes
    B = 3 * N * S
    t = ms_per_step * 1e-3
    flops = alg_flops(c.dims)
    alu_peak = ALU_PEAK_GFLOPS[c.dtype]
    probe = pac.pac_measure_fma_peak(c.dtype)
    frac_alu = flops / t / 1e9 / alu_peak
    frac_hbm = B / t / 1e9 / peak
    reps = max(5, min(a.steps, 50))
    seqs = []
    with torch.cuda.stream(stream):
        for k in range(reps):
            flush()
            seqs.append(pac.pac_convolve_timed(plan.handle, 0, x, y, stream.cuda_stream))
    per = {}
    for seq in seqs:
        for name, tt in seq:
            per.setdefault(name, []).append(tt)
    table = launch_table(pac, plan, c)
    byk = {}
    if table is not None and all(len(seq) == len(table) for seq in seqs):
        for i, (kname, bts, fl) in enumerate(table):
            ent = byk.setdefault(kname, {"ms": [], "bytes": bts, "flops": fl})
            ent["ms"].extend(seq[i][1] for seq in seqs)
    kernel = None
    if byk:
        dom = max(byk, key=lambda k: sum(byk[k]["ms"]))
        e = byk[dom]
        avg = sum(e["ms"]) / len(e["ms"])
        kernel = {"name": dom, "avg_launch_ms": avg, "launches_per_step": len(e["ms"]) / reps,
                  "time_share": sum(e["ms"]) / sum(sum(v["ms"]) for v in byk.values()),
                  "alg_flops_per_launch": e["flops"], "achieved_tflops": e["flops"] / (avg * 1e-3) / 1e12,
                  "frac_alu": e["flops"] / (avg * 1e-3) / 1e9 / alu_peak,
                  "pass_model_bytes_per_launch": e["bytes"],
                  "pass_model_frac_hbm": e["bytes"] / (avg * 1e-3) / 1e9 / peak,
                  "pass_model_rule": "2 N S per rows pass, 3 N S per fused or plane pass (the pass' own traffic, "
                                     "not the convolution's compulsory bytes)"}
    traffic = ncu_traffic(kernel["name"], traffic_key(a)) if kernel else None
    if kernel:
        kernel["traffic"] = traffic
    alu = c.dtype == "c128"
    out = {"bound": "alu" if alu else "hbm",
           "achieved": flops / t / 1e12 if alu else B / t / 1e9,
           "peak": alu_peak / 1e3 if alu else peak,
           "unit": "TFLOP/s" if alu else "GB/s",
           "frac": frac_alu if alu else frac_hbm,
           "traffic": traffic, "traffic_kernel": kernel["name"] if kernel else None,
           "frac_alu": frac_alu, "frac_hbm": frac_hbm,
           "flops_per_step": flops, "bytes_per_step": B,
           "flop_count": f"2 c_r N log2 N + 6 N with c_r = {c_r_of(c.dims):.3f} (per prime base: 2 -> 4.08, "
                         "3 -> 5.9, 5 -> 5.9)",
           "alu_peak_kind": ("FP64: 152 SMs x 2 FMA/clk x 2 flops x 2070 MHz (GB300's 1.25 TFLOP/s FP64)" if alu else
                             "FP32: 152 SMs x 128 FMA lanes x 2 flops x 2070 MHz"),
           "alu_probe_tflops": probe / 1e3,
           "hbm_peak_gbps": peak, "hbm_peak_kind": f"{peak_kind} copy bandwidth",
           "kernel": kernel}
    return out, {k: sum(v) / reps for k, v in per.items()}


def traffic_key(a) -> str:
    """Key of the main workload in the committed ncu traffic summary."""
    base = {"conv2d-r5": "conv2d_3125", "conv2d-r3": "conv2d_2187", "conv1d": "conv1d"}.get(
        a.workload, f"conv3d_{a.n}")
    return f"{base}_{a.dtype}"


def workload_conv(a, pin):
    """The main leg's problem: --workload conv3d (default: n^3, --radix, --dtype), conv2d-r3 (2187^2),
    conv2d-r5 (3125^2) or conv1d (n = 2^10, radix 2, FP64)."""
    if a.workload == "conv2d-r3":
        return pin.c3(3, a.dtype)
    if a.workload == "conv2d-r5":
        return pin.c3(5, a.dtype)
    if a.workload == "conv1d":
        return pin.c1()
    return pin.c2(a.radix, a.dtype, a.n)


def workload_name(a, c=None):
    prec = {"c64": "complex FP32", "c128": "complex FP64",
            "c128df": "complex FP64 arrays in double-float arithmetic"}[a.dtype]
    if a.workload == "conv2d-r3":
        return f"2-D periodic convolution 2187^2, {prec}, radix 3, periodised exponential filter spectrum resident"
    if a.workload == "conv2d-r5":
        return f"2-D periodic convolution 3125^2, {prec}, radix 5, periodised exponential filter spectrum resident"
    if a.workload == "conv1d":
        return "1-D circular convolution n=2^10, complex FP64, radix 2, uniform filter spectrum resident"
    return (f"3-D periodic convolution {a.n}^3, {prec}, radix {a.radix}, "
            f"periodised Gaussian sigma=4 filter spectrum resident")


def oracle_convolution(c, x, h, fs):
    """One whole convolution by the oracle, as it stands: the separable
    per-axis definition (O2) for a separable filter, else the direct
    definition (O1).  Returns the route's description."""
    import oracle
    if fs is not None:
        oracle.conv_separable(fs, x)
        return "separable-direct convolution (oracle route O2, FP64, OpenMP)"
    oracle.conv_direct(h, x)
    return "direct definition (oracle route O1, FP64, OpenMP)"


def oracle_macs(c, fs):
    """Complex multiply-adds of one whole oracle convolution of problem c."""
    return c.n_total * (sum(c.dims) if fs is not None else c.n_total)


def cpu_baseline_leg(a, y_gpu):
    """The FP64 oracle as it stands on the host cores, on the main workload's
    own inputs: the GPU result's relative L2 error against it, and its time
    on all cores and on one core (oracle_check)."""
    import oracle
    import pac_inputs as pin
    c = workload_conv(a, pin)
    x, (h, fs) = pin.make_x(c), pin.make_h(c)
    oracle.build()
    chk = oracle_check(c, x, h, fs, y_gpu)
    allc, one = chk["cpu_oracle"]["all_cores"], chk["cpu_oracle"]["one_core"]
    base = {"value": allc["GBps"], "unit": UNIT, "cores": allc["cores"], "kind": "oracle",
            "sample": f"{'x'.join(map(str, c.dims))}: {allc['route']}, {allc['s']:.2f} s on {allc['cores']} "
                      "cores; GB/s = 3*N*S of the computed outputs / time",
            "one_core": one}
    return {"rel_l2_vs_oracle": chk["rel_l2_vs_oracle"], "tolerance": chk["tolerance"],
            "oracle_route": chk["oracle_route"], "cpu_baseline": base}


def reference_arm(a):
    """--impl reference: the oracle timed as it stands on the host cores, each
    step one whole convolution of the workload by the route the main line's
    cpu_baseline times (O2 for separable filters, O1 otherwise); where that
    would exceed about 3e9 multiply-adds per step, the direct definition (O1)
    at 64 seeded output points, scaled to a whole convolution's bytes."""
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    import pac_inputs as pin
    oracle.build()
    c = workload_conv(a, pin)
    x, (h, fs) = pin.make_x(c), pin.make_h(c)
    B = 3 * c.n_total * c.elem_bytes
    whole = oracle_macs(c, fs) <= 3e9
    npts = 64
    ts = []
    route = ""
    for k in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        if whole:
            route = oracle_convolution(c, x, h, fs)
        else:
            oracle.conv_direct_points(h, x, pin.sample_points(c.n_total, npts, seed=1000 + k))
        if k >= a.warmup:
            ts.append(time.perf_counter() - t0)
    tot = sum(ts)
    frac = 1.0 if whole else npts / c.n_total
    value = a.steps * B * frac / tot / 1e9
    if whole:
        sample = f"one whole {'x'.join(map(str, c.dims))} {route} per step; GB/s = 3*N*S / time"
    else:
        sample = (f"direct definition (oracle route O1, FP64, compensated sums) at {npts} seeded output points "
                  f"per step; GB/s scaled by the computed fraction of outputs")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": tot / a.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "dims": list(c.dims), "radix": c.radix,
                       "inputs": "the workload's seeded inputs rounded once to its precision, promoted to FP64 "
                                 "for the oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def configs_leg(a, torch, pac, pin, dev, stream, flush, peak):
    """Every single-convolution workload: 1-D 2^10 FP64 radix 2; 3-D 128^3
    radix 2/4/8 FP32 and FP64; 2-D 2187^2 radix 3 and 3125^2 radix 5, FP32
    and FP64; mixed radix (2^a 3^b 5^c) 2-D 1000^2 and 6000^2 and 3-D 120^3,
    FP32; the anisotropic 2^24 x 2 and 2^22 x 2 x 2, FP32.  Each: GB/s of
    3 N S and its HBM fraction, the ALU fraction of the algorithmic flops, the
    permuted form and cuFFT on the same GPU, launches per convolution and the
    pass schedule (autotuned unless --no-tune), the relative L2 error against
    the FP64 oracle and the oracle's time on all host cores and on one core.
    Inputs are each workload's seeded recipe (pac_inputs), made on the host
    (x: re, im N(0,1) or U[-1,1]; the workload's filter)."""
    out = []
    probe = {dt: pac.pac_measure_fma_peak(dt) for dt in ("c64", "c128")}
    cases = [(pin.c1(), "1-D n=2^10, radix 2, complex FP64")]
    for dt in ("c64", "c128"):
        for r in (2, 4, 8):
            cases.append((pin.c2(r, dt), f"3-D 128^3, radix {r}, complex {'FP32' if dt == 'c64' else 'FP64'}"))
    for dt in ("c64", "c128"):
        for r in (3, 5):
            c = pin.c3(r, dt)
            cases.append((c, f"2-D {c.dims[0]}^2, radix {r}, complex {'FP32' if dt == 'c64' else 'FP64'}"))
    # complex FP64 arrays computed in double-float arithmetic (PAC_C128_DF), the same inputs as the FP64 rows
    for r in (2, 4, 8):
        cases.append((pin.c2(r, "c128df"), f"3-D 128^3, radix {r}, complex FP64 arrays, double-float arithmetic"))
    for r in (3, 5):
        c = pin.c3(r, "c128df")
        cases.append((c, f"2-D {c.dims[0]}^2, radix {r}, complex FP64 arrays, double-float arithmetic"))
    # mixed radix (Section 7.1): 1000 = 2^3 5^3, 6000 = 2^4 3 5^3, 120 = 2^3 3 5
    cases.append((pin.mixed((1000, 1000)), "2-D 1000^2, mixed radix 2^3 5^3, complex FP32"))
    cases.append((pin.mixed((6000, 6000)), "2-D 6000^2, mixed radix 2^4 3 5^3, complex FP32"))
    cases.append((pin.mixed((120, 120, 120)), "3-D 120^3, mixed radix 2^3 3 5, complex FP32"))
    # the paper's anisotropic shapes (a long axis with axes of 2)
    cases.append((pin.aniso((2 ** 24, 2)), "2-D 2^24 x 2, radix 2, complex FP32 (anisotropic)"))
    cases.append((pin.aniso((2 ** 22, 2, 2)), "3-D 2^22 x 2 x 2, radix 2, complex FP32 (anisotropic)"))
    sh = stream.cuda_stream
    oracle_cache = {}
    for c, name in cases:
        N, S = c.n_total, c.elem_bytes
        B = 3 * N * S
        x_np, (h_np, fs) = pin.make_x(c), pin.make_h(c)
        x = torch.from_numpy(x_np).to(dev)
        h = torch.from_numpy(h_np).to(dev)
        y = torch.empty_like(x)
        tuned_us = None
        if not a.no_tune:
            tuned_us = pac.pac_tune(c.dims, c.radix, c.dtype, 5)
        plan = pac.Plan(c.dims, c.radix, c.dtype)
        plan.filter_spectrum(h)
        steps = 30 if N * S < (64 << 20) else 10
        ms = time_steps(torch, lambda: pac.pac_convolve(plan.handle, x, y, sh), steps, 3, flush, stream)
        if c.dtype == "c128df":
            out.append(double_float_entry(a, torch, pac, c, name, plan, x, h, y, ms, steps, flush, stream, peak,
                                          x_np, h_np, fs, oracle_cache, tuned_us))
            continue
        msp = time_steps(torch, lambda: pac.pac_convolve_permuted(plan.handle, x, y, sh), steps, 3, flush, stream)
        Hn = torch.fft.fftn(h)
        yc = torch.empty_like(x)

        def cufft_step():
            torch.fft.ifftn(torch.fft.fftn(x) * Hn, out=yc)

        msc = time_steps(torch, cufft_step, steps, 3, flush, stream)
        # the paper's transform-level comparison: unordered DIF output (uFFT2) against the ordered
        # DFT with its index-reversal pass (FFT2), and the permutation's share of the latter
        msu = time_steps(torch, lambda: pac.pac_forward_unordered(plan.handle, x, y, sh), steps, 3, flush, stream)
        mso = time_steps(torch, lambda: pac.pac_fft(plan.handle, x, y, False, sh), steps, 3, flush, stream)
        per = {}
        with torch.cuda.stream(stream):
            for _ in range(5):
                flush()
                for kname, tt in pac.pac_convolve_timed(plan.handle, 2, x, y, sh):
                    per[kname] = per.get(kname, 0.0) + tt
        pac.pac_convolve(plan.handle, x, y, sh)
        stream.synchronize()
        diff = float(torch.linalg.vector_norm(y - yc) / torch.linalg.vector_norm(yc))
        t, tp, tc = (statistics.median(v) for v in (ms, msp, msc))
        flops = alg_flops(c.dims)
        ent = {"workload": name, "dims": list(c.dims), "radix": c.radix, "dtype": c.dtype,
               "ms": t, "GBps": B / (t * 1e-3) / 1e9, "pct_hbm_roofline": B / (t * 1e-3) / 1e9 / peak,
               "permuted_GBps": B / (tp * 1e-3) / 1e9, "speedup_vs_permuted": tp / t,
               "cufft_GBps": B / (tc * 1e-3) / 1e9, "speedup_vs_cufft": tc / t,
               "launches": plan.query(pac.Q_LAUNCHES_CONVOLVE), "groups": plan.query(pac.Q_GROUPS),
               "plane_ctas": plan.query(pac.Q_PLANE), "group_cap": plan.query(pac.Q_GROUP_CAP),
               "tuned_us": tuned_us, "rel_l2_vs_cufft": diff,
               "transform": {"unordered_us": statistics.median(msu) * 1e3,
                             "ordered_us": statistics.median(mso) * 1e3,
                             "permutation_share_of_ordered": per.get("permute", 0.0) / sum(per.values())},
               "alu": {"flops_per_conv": flops, "c_r": c_r_of(c.dims), "achieved_gflops": flops / (t * 1e-3) / 1e9,
                       "peak_gflops": ALU_PEAK_GFLOPS[c.dtype], "probe_gflops": probe[c.dtype],
                       "frac": flops / (t * 1e-3) / 1e9 / ALU_PEAK_GFLOPS[c.dtype]}}
        y_host = y.cpu().numpy()
        plan.close()
        del x, y, h, yc, Hn
        torch.cuda.empty_cache()
        if not a.no_cpu:
            ent.update(oracle_check(c, x_np, h_np, fs, y_host, cache=oracle_cache))
        out.append(ent)
    out.append(prime_factor_entry(a, torch, pac, pin, dev, stream, flush, peak))
    return out


def double_float_entry(a, torch, pac, c, name, plan, x, h, y, ms, steps, flush, stream, peak, x_np, h_np, fs,
                       oracle_cache, tuned_us):
    """A configs row of a double-float plan (PAC_C128_DF): complex FP64 arrays,
    butterflies in pairs of FP32 values.  Against the FP64 plan and cuFFT
    (FP64) on the same GPU and inputs; the algorithmic flops per second as a
    fraction of the FP64 pipe's peak (above 1: faster than FP64 arithmetic can
    be); the relative L2 error against the FP64 oracle (same inputs as the
    FP64 row, whose oracle result is reused)."""
    sh = stream.cuda_stream
    N, S = c.n_total, c.elem_bytes
    B = 3 * N * S
    p64 = pac.Plan(c.dims, c.radix, "c128")
    p64.filter_spectrum(h)
    y64 = torch.empty_like(x)
    ms64 = time_steps(torch, lambda: pac.pac_convolve(p64.handle, x, y64, sh), steps, 3, flush, stream)
    Hn = torch.fft.fftn(h)
    yc = torch.empty_like(x)
    msc = time_steps(torch, lambda: torch.fft.ifftn(torch.fft.fftn(x) * Hn, out=yc), steps, 3, flush, stream)
    pac.pac_convolve(plan.handle, x, y, sh)
    stream.synchronize()
    t, t64, tc = (statistics.median(v) for v in (ms, ms64, msc))
    flops = alg_flops(c.dims)
    ent = {"workload": name, "dims": list(c.dims), "radix": c.radix, "dtype": c.dtype,
           "ms": t, "GBps": B / (t * 1e-3) / 1e9, "pct_hbm_roofline": B / (t * 1e-3) / 1e9 / peak,
           "fp64_plan_ms": t64, "speedup_vs_fp64_plan": t64 / t,
           "cufft_GBps": B / (tc * 1e-3) / 1e9, "speedup_vs_cufft": tc / t,
           "launches": plan.query(pac.Q_LAUNCHES_CONVOLVE), "groups": plan.query(pac.Q_GROUPS),
           "group_cap": plan.query(pac.Q_GROUP_CAP), "tuned_us": tuned_us,
           "rel_l2_vs_fp64_plan": float(torch.linalg.vector_norm(y - y64) / torch.linalg.vector_norm(y64)),
           "rel_l2_vs_cufft": float(torch.linalg.vector_norm(y - yc) / torch.linalg.vector_norm(yc)),
           "alu": {"flops_per_conv": flops, "c_r": c_r_of(c.dims), "achieved_gflops": flops / (t * 1e-3) / 1e9,
                   "frac_of_fp64_peak": flops / (t * 1e-3) / 1e9 / ALU_PEAK_GFLOPS["c128"],
                   "note": "algorithmic flops of the convolution over the FP64 pipe's peak; the kernels run "
                           "about 15 FP32 instructions per FP64 operation on the FP32 pipes"}}
    y_host = y.cpu().numpy()
    p64.close()
    plan.close()
    del x, y, y64, h, yc, Hn
    torch.cuda.empty_cache()
    if not a.no_cpu:
        ent.update(oracle_check(c, x_np, h_np, fs, y_host, cache=oracle_cache))
    return ent


def prime_factor_entry(a, torch, pac, pin, dev, stream, flush, peak):
    """The prime factor form (Section 7.2) of a 1-D length n = 2^10 3^5 5^3
    (FP32): three permutations around the 3-D convolution of shape
    (1024, 243, 125), against the permutation-free mixed-radix 1-D plan of
    the same n and cuFFT; the two per-call permutations' share of the prime
    factor form's time; both results against the FP64 oracle at seeded
    points.  x: re, im U[-1,1]; h: re, im U[-1,1] (seeded)."""
    n = 2 ** 10 * 3 ** 5 * 5 ** 3
    B = 3 * n * 8
    c = pin.Conv((n,), 0, "c64", "uniform", "uniform", seed=7, h_seed=107)
    x_np, (h_np, _) = pin.make_x(c), pin.make_h(c)
    x = torch.from_numpy(x_np).to(dev)
    h = torch.from_numpy(h_np).to(dev)
    y = torch.empty_like(x)
    sh = stream.cuda_stream
    pfa = pac.Pfa(n, "c64")
    plan = pac.Plan((n,), 0, "c64")
    try:
        pfa.filter_spectrum(h)
        plan.filter_spectrum(h)
        inner = pac.pac_pfa_plan(pfa.handle)
        xt = torch.empty_like(x)
        ms_pfa = time_steps(torch, lambda: pac.pac_pfa_convolve(pfa.handle, x, y, sh), 10, 3, flush, stream)
        ms_inner = time_steps(torch, lambda: pac.pac_convolve(inner, x, xt, sh), 10, 3, flush, stream)
        ms_ct = time_steps(torch, lambda: pac.pac_convolve(plan.handle, x, y, sh), 10, 3, flush, stream)
        Hn = torch.fft.fft(h)
        ms_cufft = time_steps(torch, lambda: torch.fft.ifft(torch.fft.fft(x) * Hn, out=xt), 10, 3, flush, stream)
        t_pfa, t_inner, t_ct, t_cu = (statistics.median(v) for v in (ms_pfa, ms_inner, ms_ct, ms_cufft))
        chk = {}
        if not a.no_cpu:
            pac.pac_pfa_convolve(pfa.handle, x, y, sh)
            stream.synchronize()
            y_pfa = y.cpu().numpy()
            pac.pac_convolve(plan.handle, x, y, sh)
            stream.synchronize()
            chk = oracle_check(c, x_np, h_np, None, y.cpu().numpy())
            pts = pin_sample(n, 256, 4242)
            import oracle
            ref = oracle.conv_direct_points(h_np, x_np, pts)
            chk["prime_factor_rel_l2_vs_oracle"] = oracle.rel_l2(y_pfa.reshape(-1)[pts], ref)
            chk["prime_factor_oracle_route"] = "direct definition at 256 seeded output points (oracle route O1)"
        return {**chk, "workload": "1-D n=2^10 3^5 5^3 (31.1 M), complex FP32: prime factor form (Section 7.2) "
                                   "against the mixed-radix plan",
                "dims": [n], "radix": 0, "dtype": "c64", "ms": t_ct, "GBps": B / (t_ct * 1e-3) / 1e9,
                "pct_hbm_roofline": B / (t_ct * 1e-3) / 1e9 / peak,
                "launches": plan.query(pac.Q_LAUNCHES_CONVOLVE), "groups": plan.query(pac.Q_GROUPS),
                "cufft_GBps": B / (t_cu * 1e-3) / 1e9, "speedup_vs_cufft": t_cu / t_ct,
                "prime_factor": {"shape": list(pfa.shape), "ms": t_pfa, "GBps": B / (t_pfa * 1e-3) / 1e9,
                                 "launches": pfa.query(pac.Q_LAUNCHES_CONVOLVE),
                                 "permutation_share": max(0.0, 1.0 - t_inner / t_pfa),
                                 "mixed_radix_speedup": t_pfa / t_ct}}
    finally:
        pfa.close()
        plan.close()
        del x, y, h
        torch.cuda.empty_cache()


def batched_leg(a, torch, pac, pin, dev, stream, flush):
    """4096 independent complex FP32 convolutions, sizes from 20 classes
    (1-D 2^8..2^16 and 3^5..3^10, 2-D (2^6..2^10)^2), 64 filter ids, in one
    pac_convolve_many call (one persistent launch replayed as a CUDA graph),
    next to the merged-launch form (one launch per level and shape).
    Inputs are drawn on the device from seeded generators (x: re, im
    N(0,1); filters: re, im U[-1,1] per filter id and shape)."""
    insts = pin.c4_instances(a.batch)
    gx = torch.Generator(device=dev)
    gx.manual_seed(4)
    plans, handles, xs, ys = {}, [], [], []
    total = 0
    t_setup = time.perf_counter()
    if not a.no_tune:  # one schedule per size class (20 classes)
        for dims, radix in pin.C4_CLASSES:
            pac.pac_tune(dims, radix, "c64", 3)
    for c in insts:
        key = (c.dims, c.radix, c.h_seed)
        if key not in plans:
            gh = torch.Generator(device=dev)
            gh.manual_seed(c.h_seed * 7919 + c.n_total)
            h = (torch.rand(*c.dims, 2, generator=gh, device=dev) * 2 - 1).contiguous()
            p = pac.Plan(c.dims, c.radix, "c64")
            p.filter_spectrum(torch.view_as_complex(h))
            plans[key] = p
        handles.append(plans[key].handle)
        x = torch.view_as_complex(torch.randn(*c.dims, 2, generator=gx, device=dev).contiguous())
        xs.append(x)
        ys.append(torch.empty_like(x))
        total += 3 * c.n_total * 8
    setup_s = time.perf_counter() - t_setup
    launches = pac.pac_convolve_many_launches(handles)
    sh = stream.cuda_stream
    steps = max(5, min(a.steps, 20))
    ms = time_steps(torch, lambda: pac.pac_convolve_many(handles, xs, ys, sh), steps, max(3, a.warmup // 3),
                    flush, stream)
    t = sum(ms) / steps
    # the merged-launch form of the same batch (one launch per level and shape, a captured graph)
    os.environ["PAC_BATCH"] = "graph"
    try:
        launches_g = pac.pac_convolve_many_launches(handles)
        msg = time_steps(torch, lambda: pac.pac_convolve_many(handles, xs, ys, sh), steps, max(3, a.warmup // 3),
                         flush, stream)
    finally:
        os.environ.pop("PAC_BATCH", None)
    tg = sum(msg) / steps
    # the same instances one call each (no merging, no graph), for comparison
    ms1 = time_steps(torch, lambda: [pac.pac_convolve(hd, x, y, sh) for hd, x, y in zip(handles, xs, ys)],
                     3, 1, flush, stream)
    t1 = sum(ms1) / 3
    out = {"workload": f"{len(insts)} complex FP32 convolutions, 20 size classes, 64 filter ids",
           "value": total / (t * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": t, "bytes_per_step": total,
           "launches_per_step": launches, "plans": len(plans),
           "form": "one persistent launch (graph of one kernel)" if launches == 1 else "merged launches per level",
           "merged_launches": {"value": total / (tg * 1e-3) / 1e9, "ms_per_step": tg, "launches_per_step": launches_g},
           "one_call_each": {"value": total / (t1 * 1e-3) / 1e9, "ms_per_step": t1},
           "setup_s": setup_s, "inputs": "device-generated, seeded (torch Philox)",
           "schedules": "autotuned per size class" if not a.no_tune else "default"}
    for p in plans.values():
        p.close()
    del xs, ys
    torch.cuda.empty_cache()
    return out


def served_leg(a, torch, pac, pin, dev):
    """Poisson arrivals (2000 req/s, seeded) of mixed 1-D/2-D/3-D, radix 2/3,
    70 % FP32 / 30 % FP64 convolutions through the request queue (continuous
    batching, admission by HBM budget); filters from a resident pool of 32
    (Gaussian / exponential); latency = submit to completion."""
    reqs = pin.c5_requests(a.serve_seconds)
    pool = pin.c5_filter_pool()
    max_inflight, budget = a.max_inflight, 64 << 30
    t_setup = time.perf_counter()
    plans, xbuf, ybuf, rr = {}, {}, {}, {}
    K = max_inflight + 2

    def factors(kind, param, dims):
        fs = pin.gaussian_factors(dims, param) if kind == "gauss" else pin.exponential_factors(dims, param)
        return [torch.from_numpy(f).to(dev) for f in fs]

    for r in reqs:
        c = r.conv
        key = (c.dims, c.radix, c.dtype, r.filter_id)
        if key not in plans:
            fs = factors(*pool[r.filter_id], c.dims)
            h = fs[0]
            for f in fs[1:]:
                h = torch.outer(h.reshape(-1), f).reshape(*h.shape, f.shape[0])
            h = h.to(torch.complex64 if c.dtype == "c64" else torch.complex128).contiguous()
            p = pac.Plan(c.dims, c.radix, c.dtype)
            p.filter_spectrum(h)
            plans[key] = p
        sk = (c.dims, c.dtype)
        if sk not in xbuf:
            g = torch.Generator(device=dev)
            g.manual_seed(50_000 + len(xbuf))
            real = torch.float32 if c.dtype == "c64" else torch.float64
            xbuf[sk] = torch.view_as_complex(torch.randn(*c.dims, 2, generator=g, device=dev, dtype=real))
            ybuf[sk] = [torch.empty_like(xbuf[sk]) for _ in range(K)]
            rr[sk] = 0
    # warm-up: every plan once, outside the timed stream (first-use costs of
    # its kernels and streams are not part of a served request's latency)
    for (dims, radix, dtype, fid), p in plans.items():
        pac.pac_convolve(p.handle, xbuf[(dims, dtype)], ybuf[(dims, dtype)][0])
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup

    def pct_of(v, p):
        v = sorted(v)
        return v[min(len(v) - 1, max(0, math.ceil(p / 100 * len(v)) - 1))]

    def one_run():
        q = pac.pac_queue_create(budget, max_inflight)
        tickets, nbytes = [], 0
        t0 = time.perf_counter()
        for r in reqs:
            c = r.conv
            while time.perf_counter() - t0 < r.t_arrive:
                pass
            sk = (c.dims, c.dtype)
            y = ybuf[sk][rr[sk] % K]
            rr[sk] += 1
            tickets.append(pac.pac_submit(q, plans[(c.dims, c.radix, c.dtype, r.filter_id)].handle, xbuf[sk], y))
            nbytes += 3 * c.n_total * c.elem_bytes
        pac.pac_queue_drain(q, 600000)
        t_end = time.perf_counter()
        lats, by_class = [], {}
        for tk, r in zip(tickets, reqs):
            st, lat = pac.pac_poll(q, tk)
            lats.append(lat)
            small = 2 * r.conv.n_total * r.conv.elem_bytes <= (8 << 20)  # the queue's small-request class
            by_class.setdefault(f"{'small' if small else 'large'} {'FP32' if r.conv.dtype == 'c64' else 'FP64'}",
                                []).append(lat)
        pac.pac_queue_destroy(q)
        span = t_end - t0
        return {"p50_us": pct_of(lats, 50), "p99_us": pct_of(lats, 99), "mean_us": sum(lats) / len(lats),
                "GBps": nbytes / span / 1e9, "span_s": span, "offered_GBps": nbytes / a.serve_seconds / 1e9,
                "by_class": {k: {"n": len(v), "p50_us": pct_of(v, 50), "p99_us": pct_of(v, 99)}
                             for k, v in sorted(by_class.items())}}

    runs = [one_run() for _ in range(max(1, a.serve_repeats))]
    for p in plans.values():
        p.close()

    def spread(vals):
        med = statistics.median(vals)
        return {"median": med, "min": min(vals), "max": max(vals),
                "max_rel_dev": max(abs(v - med) for v in vals) / med if med else 0.0}

    classes = sorted({k for r in runs for k in r["by_class"]})
    out = {"workload": f"Poisson {len(reqs) / a.serve_seconds:.0f} req/s for {a.serve_seconds:g} s: 1-D/2-D/3-D, "
                       "radix 2/3, 70% FP32 / 30% FP64, 32 resident filters",
           "requests": len(reqs), "repeats": len(runs),
           "p50_us": statistics.median(r["p50_us"] for r in runs),
           "p99_us": statistics.median(r["p99_us"] for r in runs),
           "value": statistics.median(r["GBps"] for r in runs), "unit": "GB/s",
           "offered_GBps": runs[0]["offered_GBps"],
           "spread": {"p50_us": spread([r["p50_us"] for r in runs]), "p99_us": spread([r["p99_us"] for r in runs])},
           "by_class": {k: {"p50_us": spread([r["by_class"][k]["p50_us"] for r in runs if k in r["by_class"]]),
                            "p99_us": spread([r["by_class"][k]["p99_us"] for r in runs if k in r["by_class"]]),
                            "n": runs[0]["by_class"].get(k, {}).get("n", 0)} for k in classes},
           "runs": [{k: v for k, v in r.items() if k != "by_class"} for r in runs],
           "max_inflight": max_inflight, "hbm_budget_bytes": budget, "plans": len(plans),
           "by_class_note": "small = at most 8 MiB of device bytes (2 N S): high-priority streams, reserved slots; "
                            "at most two large FP64 requests run at once",
           "note": f"the same seeded request stream served {len(runs)} times; medians over the runs, "
                   "max_rel_dev = largest deviation of a run from the median, relative",
           "setup_s": setup_s}
    torch.cuda.empty_cache()
    return out


def profile_path_leg(a, torch, pac, pin, dev):
    """--profile-path: warm-up and timed calls of one other path (for ncu
    launch lists and captures of its kernels); prints one JSON line of times."""
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    if a.profile_path == "batched":
        insts = pin.c4_instances(a.batch)
        plans, handles, xs, ys = {}, [], [], []
        for c in insts:
            key = (c.dims, c.radix, c.h_seed)
            if key not in plans:
                p = pac.Plan(c.dims, c.radix, "c64")
                p.filter_spectrum(torch.from_numpy(pin.make_h(c)[0]).to(dev))
                plans[key] = p
            handles.append(plans[key].handle)
            xs.append(torch.from_numpy(pin.make_x(c)).to(dev))
            ys.append(torch.empty_like(xs[-1]))
        ms = time_steps(torch, lambda: pac.pac_convolve_many(handles, xs, ys, sh), a.steps, a.warmup, lambda: None,
                        stream)
        print(json.dumps({"profile_path": "batched", "instances": len(insts),
                          "launches_per_call": pac.pac_convolve_many_launches(handles), "ms": ms}), flush=True)
        for p in plans.values():
            p.close()
        return 0
    env = {}
    if a.profile_path == "permuted":
        c = workload_conv(a, pin)
    elif a.profile_path == "single":
        c = pin.c2(4, "c64", 128)
        env = {"PAC_SINGLE_LAUNCH": "1", "PAC_PLANE": "0"}
    elif a.profile_path == "mixed":
        c = pin.mixed((1000, 1000))
        env = {"PAC_MIXED": "1"}
    else:
        n = 2 ** 10 * 3 ** 5 * 5 ** 3
        c = pin.Conv((n,), 0, "c64", "uniform", "uniform", seed=7, h_seed=107)
    x = torch.from_numpy(pin.make_x(c)).to(dev)
    h = torch.from_numpy(pin.make_h(c)[0]).to(dev)
    y = torch.empty_like(x)
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        obj = pac.Pfa(c.n_total, c.dtype) if a.profile_path == "pfa" else pac.Plan(c.dims, c.radix, c.dtype)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    obj.filter_spectrum(h)
    if a.profile_path == "permuted":
        fn = lambda: pac.pac_convolve_permuted(obj.handle, x, y, sh)  # noqa: E731
    elif a.profile_path == "pfa":
        fn = lambda: pac.pac_pfa_convolve(obj.handle, x, y, sh)  # noqa: E731
    else:
        fn = lambda: pac.pac_convolve(obj.handle, x, y, sh)  # noqa: E731
    ms = time_steps(torch, fn, a.steps, a.warmup, lambda: None, stream)
    print(json.dumps({"profile_path": a.profile_path, "dims": list(c.dims), "dtype": c.dtype,
                      "launches_per_call": obj.query(pac.Q_LAUNCHES_CONVOLVE), "ms": ms}), flush=True)
    obj.close()
    return 0


def main(argv=None):
    a = parse_args(argv)
    world, rank, local = dist_env()
    if a.impl == "reference":
        line = reference_arm(a)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0

    import numpy as np
    import torch

    import pac_inputs as pin
    import paper_2506_12718_gb300 as pac
    from paper_2506_12718_gb300 import _build

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        _build.build()
    barrier(world)
    pac.load()

    if a.profile_path != "none":
        return profile_path_leg(a, torch, pac, pin, dev)

    c = workload_conv(a, pin)
    x_np, (h_np, _) = pin.make_x(c), pin.make_h(c)
    N, S = c.n_total, c.elem_bytes
    B = 3 * N * S
    x = torch.from_numpy(x_np).to(dev)
    h = torch.from_numpy(h_np).to(dev)
    y = torch.empty_like(x)
    flush_buf = torch.empty(max(1, (a.flush_mb << 20) // 4), dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream

    def flush():
        if a.flush_mb > 0:
            flush_buf.fill_(1)

    tuned_us = None
    if not a.quick and not a.no_tune:  # pass schedule picked by the autotuner (setup, not timed)
        tuned_us = pac.pac_tune(c.dims, c.radix, c.dtype, 5)
    plan = pac.Plan(c.dims, c.radix, c.dtype)
    plan.filter_spectrum(h)
    launches = plan.query(pac.Q_LAUNCHES_CONVOLVE)

    sampler = ClockSampler(torch.cuda.current_device()).start() if rank == 0 else None
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ms = time_steps(torch, lambda: pac.pac_convolve(plan.handle, x, y, sh), a.steps, a.warmup, flush, stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier(world)
    tot_ms, tot_bytes = aggregate(sum(ms), a.steps * B, world, dev)
    value = tot_bytes / (tot_ms * 1e-3) / 1e9
    ms_per_step = tot_ms / a.steps

    peak, peak_kind = measured_peak_hbm()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"c64": "f32", "c128": "f64", "c128df": "f32x2 (double-float)"}[c.dtype], "data": "synthetic",
            "config": {"workload": workload_name(a), "dims": list(c.dims), "radix": c.radix,
                       "stages_per_axis": plan.stages(0), "bytes_per_step": B,
                       "schedule": {"passes": launches, "groups": plan.query(pac.Q_GROUPS),
                                    "plane_ctas": plan.query(pac.Q_PLANE), "group_cap": plan.query(pac.Q_GROUP_CAP),
                                    "autotuned": tuned_us is not None},
                       "l2": (f"flushed before every step ({a.flush_mb} MiB write, outside the timed events)"
                              if a.flush_mb > 0 else "not flushed (profiling run)"),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "pct_hbm_roofline": value / world / peak, "gpu_launches": a.steps * launches,
            "launches_per_step": launches}

    if not a.quick:
        line["roofline"], line["kernel_ms_per_step"] = roofline_block(a, torch, pac, plan, c, x, y, stream, flush,
                                                                      ms_per_step, peak, peak_kind)

        # the permuted form on the same GPU, same bytes B
        msp = time_steps(torch, lambda: pac.pac_convolve_permuted(plan.handle, x, y, sh), a.steps, a.warmup, flush,
                         stream)
        tp, _ = aggregate(sum(msp), 0, world, dev)
        line["permuted"] = {"value": world * a.steps * B / (tp * 1e-3) / 1e9, "unit": UNIT,
                            "ms_per_step": tp / a.steps, "launches_per_step": plan.query(pac.Q_LAUNCHES_PERMUTED)}
        line["speedup_vs_permuted"] = (tp / a.steps) / ms_per_step

        # cuFFT-based convolution (torch.fft on the same buffers), spectrum precomputed
        Hn = torch.fft.fftn(h)
        yc = torch.empty_like(x)

        def cufft_step():
            torch.fft.ifftn(torch.fft.fftn(x) * Hn, out=yc)

        msc = time_steps(torch, cufft_step, a.steps, a.warmup, flush, stream)
        tc, _ = aggregate(sum(msc), 0, world, dev)
        line["cufft"] = {"value": world * a.steps * B / (tc * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": tc / a.steps,
                         "note": "torch.fft (cuFFT) fftn -> product -> ifftn, reported baseline"}

        # end to end through the public C-ABI call with HOST buffers (pinned)
        xh = torch.from_numpy(x_np.copy()).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        mse = time_steps(torch, lambda: pac.pac_convolve_host(plan.handle, xh, yh, sh), max(10, a.steps // 4),
                         a.warmup, flush, stream)
        te, _ = aggregate(sum(mse), 0, world, dev)
        ke = max(10, a.steps // 4)
        line["e2e"] = {"value": world * ke * B / (te * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": N * S,
                       "d2h_bytes_per_step": N * S, "ms_per_step": te / ke,
                       "call": "pac_convolve_host (pinned host x -> device -> convolve -> host y)"}
        # the same workload and inputs as complex FP64 arrays computed in double-float arithmetic
        # (PAC_C128_DF: pairs of FP32 values on the FP32 pipes), device and host buffers
        ydf = None
        if c.dtype == "c128":
            pdf = pac.Plan(c.dims, c.radix, "c128df")
            pdf.filter_spectrum(h)
            ydf = torch.empty_like(x)
            msd = time_steps(torch, lambda: pac.pac_convolve(pdf.handle, x, ydf, sh), a.steps, a.warmup, flush,
                             stream)
            td, _ = aggregate(sum(msd), 0, world, dev)
            msde = time_steps(torch, lambda: pac.pac_convolve_host(pdf.handle, xh, yh, sh), ke, a.warmup, flush,
                              stream)
            tde, _ = aggregate(sum(msde), 0, world, dev)
            pac.pac_convolve(pdf.handle, x, ydf, sh)
            stream.synchronize()
            line["double_float"] = {
                "value": world * a.steps * B / (td * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": td / a.steps,
                "speedup_vs_fp64": ms_per_step / (td / a.steps), "launches_per_step": pdf.query(pac.Q_LAUNCHES_CONVOLVE),
                "alu_frac_of_fp64_peak": alg_flops(c.dims) / (td / a.steps * 1e-3) / 1e9 / ALU_PEAK_GFLOPS["c128"],
                "e2e": {"value": world * ke * B / (tde * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": tde / ke,
                        "h2d_bytes_per_step": N * S, "d2h_bytes_per_step": N * S},
                "note": "dtype c128df: complex FP64 arrays in and out, butterflies, twiddles and product in "
                        "double-float arithmetic; rel_l2 against the FP64 oracle in the configs leg"}
            pdf.close()
        y_main = None
        if rank == 0:
            pac.pac_convolve(plan.handle, x, y, sh)  # y was reused by the comparison legs
            stream.synchronize()
            y_main = y.cpu().numpy()
            ref = yc.cpu().numpy()
            line["check_vs_cufft_rel_l2"] = float(np.linalg.norm(y_main - ref) / np.linalg.norm(ref))
            if ydf is not None:
                ydf_h = ydf.cpu().numpy()
                line["double_float"]["rel_l2_vs_fp64_path"] = float(np.linalg.norm(ydf_h - y_main) /
                                                                    np.linalg.norm(y_main))
                line["double_float"]["rel_l2_vs_cufft"] = float(np.linalg.norm(ydf_h - ref) / np.linalg.norm(ref))
        del ydf

    if sampler:
        sampler.stop()
        line["clocks"] = sampler.summary(t_wall0, t_wall1)
    # the extra legs describe one GPU; a multi-GPU (replicas) run reports the main leg only
    extra = not a.quick and world == 1
    if extra and "configs" in a.legs:
        line["configs"] = configs_leg(a, torch, pac, pin, dev, stream, flush, peak)
    if extra and "batched" in a.legs:
        line["batched"] = batched_leg(a, torch, pac, pin, dev, stream, flush)
    if extra and "served" in a.legs:
        line["served"] = served_leg(a, torch, pac, pin, dev)
    if rank == 0 and world == 1 and not a.no_cpu and not a.quick:
        chk = cpu_baseline_leg(a, y_main)
        line["rel_l2_vs_oracle"] = chk["rel_l2_vs_oracle"]
        line["tolerance"] = chk["tolerance"]
        line["oracle_route"] = chk["oracle_route"]
        line["cpu_baseline"] = chk["cpu_baseline"]
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
