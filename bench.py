#!/usr/bin/env python3
"""Benchmark of the branch-free sine-cosine pair path on GB300.

Prints ONE JSON line.  A step is one pass of the forward hot path over the
headline workload: 2^28 binary32 angles uniform in [-1000, 1000) (seed 1),
binary32 sines and cosines out, plain reduction, one `sincos_pairs` launch.
Inputs (1 GiB) and outputs (2 GiB) exceed the 129 MB L2, so no flush is
needed between steps.  `value` is pairs/s over all ranks (weak scaling:
each rank owns its own 2^28 angles; no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the slow C restatement of the method)
on the host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "sin-cos pairs/s and HBM GB/s vs peak at 1 GB300; max abs/ulp err vs FP64 oracle"
UNIT = "pairs/s"
WORKLOAD = "bandwidth_2p28"
WORKLOAD_DESC = ("2^28 float32 angles uniform in [-1000, 1000) (seed 1), float32 sin and cos "
                 "outputs (1 GiB in, 2 GiB out), plain reduction, normalized coefficients")
BYTES_PER_PAIR = 12            # 4 B angle read + 4 B sine + 4 B cosine written
# FP32 operations per Huygens term by its definition (an FMA, sqrt_rn and
# rcp_rn count as one each): 3 differences, 3 for r^2, sqrt, reciprocal, k*r,
# 26 for the pair with the compensated reduction, 4 for the complex product
# and 2 accumulating FMAs.
HUYGENS_OPS_PER_TERM = 41
# FMA-pipe operations per term of the bit-exact kernel at the least: the 39
# operations of the definition other than the square root and the reciprocal,
# plus the 9 FMA-pipe operations of the correctly rounded root and reciprocal
# (7 and 2 Newton steps after rsqrt.approx and rcp.approx, which run on the
# XU pipe).  At one operation per FP32 lane per clock this bounds the kernel.
HUYGENS_FMA_OPS_BIT_EXACT = 48
FP32_LANES_PER_SM = 128
HBM_FALLBACK_GBS = 6800.0      # only when the measured-peaks file is absent
# The paper's own figures (Sec. Results), quoted for context: other hardware,
# one core, not a target.
PAPER_CONTEXT = {
    "hardware": "PowerPC 7400 (G4), 500 MHz, AltiVec 4-wide, one core",
    "latency_ns_per_4_pairs": 140,
    "interleaved_pairs_per_s": 8.0e7,
    "accuracy_normalized": {"rms_euclid": 1.2e-7, "max_euclid": 4.8e-7, "max_amplitude": 1.8e-7},
    "accuracy_dagger": {"rms_euclid": 9.8e-8, "max_euclid": 3.8e-7},
}
E2E_ROUTES = {
    "zero-copy": "sincos_pairs_host on page-locked, mapped host buffers: one kernel reads x "
                 "and writes s, c across NVLink-C2C",
    "pipeline": "sincos_pairs_host through the chunked copy pipeline: host -> device copy, "
                "kernel, device -> host copy on three rotating streams",
    "zero-copy-pageable": "sincos_pairs_host on ordinary pageable host memory: one kernel "
                          "reads x and writes s, c through the host's page tables across "
                          "NVLink-C2C",
}
FWD_SOURCES = ["core.cuh", "core_x2.cuh", "bulk.cuh", "forward.cuh", "forward_f32.cu"]
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "ncu_forward_f32_bandwidth_2p28.md")


def parse_args():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="time the library's default plans instead of tuning each op first")
    p.add_argument("--split", action="store_true",
                   help="strong scaling: one 2^28-angle array cut into contiguous blocks of "
                        "n/N angles, one per rank (default: weak scaling, 2^28 per rank)")
    return p.parse_args()


# -----------------------------------------------------------------------------
# Distributed plumbing (one process per GPU; no data-path collective)
# -----------------------------------------------------------------------------

class Dist:
    def __init__(self, want: int):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if want > 1 and self.world != want:
            raise SystemExit(f"--gpus {want} needs torchrun with {want} ranks (WORLD_SIZE="
                             f"{self.world})")

    def init(self, backend: str):
        import torch.distributed as dist
        if self.world > 1:
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if torch.cuda.is_available() and self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# -----------------------------------------------------------------------------
# Clocks during the timed region
# -----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "clocks.mem")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str):
        self.samples = []
        self.proc = None
        self.error = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception as e:  # nvidia-smi missing
            self.error = str(e)

    def _read(self):
        for line in self.proc.stdout:
            parts = [t.strip() for t in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        win = [p for (t, p) in self.samples if t0 <= t <= t1]
        if not win:     # the timed region was shorter than one sampling period
            win = [p for (t, p) in self.samples if t0 - 0.25 <= t <= t1 + 0.25]
        if not win:
            return {"error": self.error or "no nvidia-smi samples in the timed region"}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return float("nan")
        sm = [num(p[0]) for p in win]
        mx = [num(p[1]) for p in win]
        pw = [num(p[2]) for p in win]
        reasons = sorted({name for p in win for name, v in zip(self.REASONS, p[4:8])
                          if v.strip().lower() == "active"})
        mem = [num(p[8]) for p in win]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": reasons,
                "samples": len(win), "power_w_max": max(pw), "mem_mhz": statistics.median(mem)}


def live_copy_gbs(torch) -> float:
    """This GPU's copy bandwidth now: torch's copy of 2^30 bf16 elements
    (read + write bytes), best of ten, CUDA events; the same measurement as
    the copy peak the roofline is quoted against, taken on this machine for
    context."""
    a = torch.empty(1 << 30, dtype=torch.bfloat16, device="cuda")
    b = torch.empty_like(a)
    best = float("inf")
    for i in range(12):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.copy_(a)
        e1.record()
        e1.synchronize()
        if i >= 2:
            best = min(best, e0.elapsed_time(e1))
    nbytes = 2 * a.numel() * a.element_size()
    del a, b
    return nbytes / (best * 1e-3) / 1e9


def gpu_query_id(torch) -> str:
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[0] if vis else "0"


# -----------------------------------------------------------------------------
# Helpers
# -----------------------------------------------------------------------------

def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def measured_sm_max_mhz() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def code_only(src: str) -> str:
    """C++ source with its comments and blank-line runs removed, so that a
    change of comments alone does not count as a change of the kernel."""
    out, i, n = [], 0, len(src)
    while i < n:
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif src[i] == '"':                       # string literal: kept as is
            j = i + 1
            while j < n and src[j] != '"':
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(src[i])
            i += 1
    lines = [ln.rstrip() for ln in "".join(out).splitlines()]
    return "\n".join(ln for ln in lines if ln)


def kernel_source_sha() -> str:
    """Hash of the timed kernel's source files, comments left out."""
    h = hashlib.sha1()
    for name in FWD_SOURCES:
        with open(os.path.join(ROOT, "paper_cs_0406049_gb300", "csrc", name)) as f:
            h.update(code_only(f.read()).encode())
    return h.hexdigest()[:12]


def profiled_traffic():
    """DRAM bytes per launch of the timed kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    try:
        with open(TRAFFIC_PROFILE) as f:
            text = f.read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    sha = re.search(r"kernel_sources_sha1:\s*([0-9a-f]+)", text)
    if not m or not sha or sha.group(1) != kernel_source_sha():
        return None
    return float(m.group(1))


def cudart_memory_attributes(dev: int):
    """(peak memory clock in kHz, bus width in bits) from cudaDeviceGetAttribute
    through the CUDA runtime already loaded by PyTorch; (0, 0) if unavailable."""
    import ctypes
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
        except OSError:
            continue
        vals = []
        for attr in (36, 37):      # cudaDevAttrMemoryClockRate, cudaDevAttrGlobalMemoryBusWidth
            v = ctypes.c_int(0)
            if rt.cudaDeviceGetAttribute(ctypes.byref(v), ctypes.c_int(attr), ctypes.c_int(dev)):
                vals = []
                break
            vals.append(v.value)
        if len(vals) == 2:
            return vals[0], vals[1]
    return 0, 0


def vendor_peak(torch, achieved_gbs: float) -> dict:
    """The nominal HBM bandwidth from the device's attributes (peak memory
    clock x bus width x 2 transfers per clock), reported beside the measured
    copy peak; empty if this PyTorch does not expose the attributes."""
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    khz = getattr(props, "memory_clock_rate", 0) or 0
    bits = getattr(props, "memory_bus_width", 0) or 0
    if not khz or not bits:
        khz, bits = cudart_memory_attributes(dev)
    if not khz or not bits:
        return {}
    gbs = khz * 1e3 * bits / 8 * 2 / 1e9
    return {"peak_vendor": gbs, "frac_vendor": achieved_gbs / gbs,
            "peak_vendor_kind": f"memory clock {khz / 1e3:.0f} MHz x {bits}-bit bus x 2"}


def shard_bounds(n: int, rank: int, world: int) -> tuple:
    """Rank `rank`'s contiguous block [lo, hi) of an n-element array cut into
    `world` blocks whose sizes differ by at most one; the blocks tile [0, n).
    Every element is independent, so no rank needs another's data."""
    return n * rank // world, n * (rank + 1) // world


def aggregate_value(world: int, n_per_rank: int, steps: int, max_ms: float) -> float:
    """Whole-job pairs/s: every rank computed n_per_rank pairs per step; the
    slowest rank's time for all steps bounds the job."""
    return world * n_per_rank * steps / (max_ms * 1e-3)


def fp64_errors(x: np.ndarray, s: np.ndarray, c: np.ndarray) -> dict:
    """Max abs error of binary32 results against FP64 sin/cos of the same
    angles, also in units of ulp(1.0) = 2^-23, and the largest per-result ulp
    error among results with |ref| >= 2^-4."""
    xd = x.astype(np.float64)
    rs, rc = np.sin(xd), np.cos(xd)
    ok = np.isfinite(rs) & np.isfinite(s) & np.isfinite(c)
    d = np.concatenate([np.abs(s[ok] - rs[ok]), np.abs(c[ok] - rc[ok])])
    ref = np.concatenate([rs[ok], rc[ok]])
    big = np.abs(ref) >= 2.0 ** -4
    ulp = np.spacing(np.abs(ref[big]).astype(np.float32)).astype(np.float64)
    return {"max_abs": float(d.max()), "max_abs_ulp1": float(d.max() / 2.0 ** -23),
            "max_ulp_rel_ge_2m4": float((d[big] / ulp).max()), "sample": int(ok.sum())}


def backward_fp64_errors(x, gs, gc, gx) -> dict:
    """gx against the FP64 analytic gradient gs cos x - gc sin x of the same
    binary32 inputs: max abs error, and the max relative to |gs| + |gc|."""
    xd = x.astype(np.float64)
    gsd, gcd = gs.astype(np.float64), gc.astype(np.float64)
    ref = gsd * np.cos(xd) - gcd * np.sin(xd)
    ok = np.isfinite(ref)
    d = np.abs(gx.astype(np.float64)[ok] - ref[ok])
    scale = np.abs(gsd[ok]) + np.abs(gcd[ok])
    return {"max_abs": float(d.max()), "max_rel_to_abs_gs_plus_abs_gc": float((d / scale).max()),
            "sample": int(ok.sum()), "reference": "FP64 gs*cos(x) - gc*sin(x)"}


def huygens_fp64_errors(w, u, pts) -> dict:
    """The Huygens sums of the points `pts` against an FP64 direct sum of
    a_j exp(i k r) / r over the same binary32 coordinates and amplitudes:
    max abs error, and the max relative to the point's sum of |a_j| / r."""
    p = [v[pts].astype(np.float64) for v in w.p]
    q = [v.astype(np.float64) for v in w.q]
    a = w.a.astype(np.complex128)
    k = float(np.float32(w.k))
    r = np.sqrt((p[0][:, None] - q[0][None, :]) ** 2 + (p[1][:, None] - q[1][None, :]) ** 2 +
                (p[2][:, None] - q[2][None, :]) ** 2)
    ref = (a[None, :] * np.exp(1j * k * r) / r).sum(axis=1)
    scale = (np.abs(a)[None, :] / r).sum(axis=1)
    got = u[pts, 0].astype(np.float64) + 1j * u[pts, 1].astype(np.float64)
    d = np.abs(got - ref)
    return {"max_abs": float(d.max()), "max_rel_to_sum_abs_terms": float((d / scale).max()),
            "sample": int(pts.size), "reference": "FP64 direct sum over all sources"}


def batch_sample(offsets, lens, seed: int = 0) -> np.ndarray:
    """Indices of the first and last 64 and 64 random angles of every array."""
    rng = np.random.default_rng(seed)
    idx = []
    for off, n in zip(offsets, lens):
        k = min(int(n), 64)
        idx += [off + np.arange(k), off + n - k + np.arange(k), off + rng.integers(0, n, 64)]
    return np.unique(np.concatenate(idx))


def time_flushed(torch, fn, steps: int, warmup: int, flush) -> list:
    """Per-call device ms of fn with the L2 flushed before every call (a
    write of `flush`, larger than L2, outside the timed events)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    per = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        per.append(a.elapsed_time(b))
    return per


def time_each(torch, fn, steps: int, warmup: int, dist: Dist) -> list:
    """Device ms of each of K calls of fn, timed one at a time with CUDA events
    (a synchronize after each), the ranks' maxima per step.  For calls whose
    duration varies from call to call by host-side effects (the driver's
    staging of pageable copies), whose median is then the representative
    figure."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    dist.barrier()
    per = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        per.append(dist.max(a.elapsed_time(b)))
    return per


def gpu_local_cpus(torch, dev: int) -> set:
    """CPUs the kernel lists as local to the GPU's PCI function
    (local_cpulist in sysfs), among those this process may run on; empty if
    unknown."""
    p = torch.cuda.get_device_properties(dev)
    try:
        path = (f"/sys/bus/pci/devices/{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:"
                f"{p.pci_device_id:02x}.0/local_cpulist")
        with open(path) as f:
            text = f.read().strip()
    except (AttributeError, OSError):
        return set()
    return parse_cpulist(text) & os.sched_getaffinity(0)


def parse_cpulist(text: str) -> set:
    """A Linux CPU list ("0-3,8,10-11") as a set of CPU numbers."""
    cpus = set()
    for part in text.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def pinned_near_gpu(torch, dev: int, make):
    """Run make() (which allocates page-locked host memory) on the CPUs local
    to the GPU, so that the pages are placed on the GPU's NUMA node; returns
    (make()'s result, a note of where it ran)."""
    local = gpu_local_cpus(torch, dev)
    saved = os.sched_getaffinity(0)
    if not local or local == saved:
        return make(), ("on the process's CPUs (already the GPU's local CPUs)" if local
                        else "on the process's CPUs (GPU-local CPU list unknown)")
    os.sched_setaffinity(0, local)
    try:
        return make(), f"on the {len(local)} CPUs local to the GPU"
    finally:
        os.sched_setaffinity(0, saved)


def e1_stats(x: np.ndarray, s: np.ndarray, c: np.ndarray) -> dict:
    """The paper's accuracy statistics (Sec. Results): RMS and max of the
    Euclidean error sqrt(ds^2 + dc^2) against FP64 sin/cos, and the max
    amplitude error |sqrt(s^2 + c^2) - 1|, all evaluated in FP64.  The max
    is given twice: against the binary32 angle, and against the reduced
    angle the method sees, 2 pi fl(x K) with K = fl(1 / (2 * 3.1415926536))
    (the difference is the rounding of x K)."""
    xd = x.astype(np.float64)
    sd, cd = s.astype(np.float64), c.astype(np.float64)
    e = np.hypot(sd - np.sin(xd), cd - np.cos(xd))
    k32 = np.float32(1.0 / (2.0 * 3.1415926536))
    a = 2.0 * np.pi * (np.asarray(x, np.float32) * k32).astype(np.float64)
    e_red = np.hypot(sd - np.sin(a), cd - np.cos(a))
    return {"rms_euclid": float(np.sqrt(np.mean(e * e))), "max_euclid": float(e.max()),
            "max_euclid_reduced_angle": float(e_red.max()),
            "max_amplitude": float(np.abs(np.hypot(sd, cd) - 1.0).max()), "sample": int(x.size)}


def time_loop(torch, fn, steps: int, warmup: int, dist: Dist, sampler=None):
    """W untimed steps, then K steps back to back between barriers +
    synchronizes, with one CUDA event before the first and one after the last
    on the current stream (nothing else is enqueued between steps, so
    consecutive launches can overlap one's drain with the next one's start,
    as in any stream of calls).  Returns (device ms for all K steps, mean ms
    per step, clocks)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    t_begin.record(stream)
    for _ in range(steps):
        fn()
    t_end.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    dist.barrier()
    torch.cuda.synchronize()
    total = t_begin.elapsed_time(t_end)
    clocks = sampler.summary(w0, w1) if sampler else None
    return total, total / steps, clocks


# -----------------------------------------------------------------------------
# Reference arm: the CPU oracle on host cores
# -----------------------------------------------------------------------------

def run_reference(args, dist: Dist):
    if dist.rank != 0:
        return
    import oracle
    from paper_cs_0406049_gb300 import workloads
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    x_full = workloads.bandwidth()
    # size each step's sample so that warmup + steps take about two minutes
    probe = x_full[: 1 << 22]
    s = np.empty_like(probe)
    c = np.empty_like(probe)
    t = time.perf_counter()
    used = oracle.sincos_mt(probe, s, c, threads=cores)
    rate = probe.size / (time.perf_counter() - t)
    per_step = int(rate * 120.0 / max(1, args.steps + args.warmup))
    per_step = int(min(max(per_step, 1 << 16), 1 << 26))
    xs = x_full[:per_step]
    s = np.empty_like(xs)
    c = np.empty_like(xs)
    for _ in range(args.warmup):
        oracle.sincos_mt(xs, s, c, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        used = oracle.sincos_mt(xs, s, c, threads=cores)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    sample = f"first {per_step} angles of the {WORKLOAD} workload per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC,
                   "reference": "CPU oracle (plain C binary32, fmaf) on host cores",
                   "sample_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# -----------------------------------------------------------------------------
# Our arm
# -----------------------------------------------------------------------------

def cpu_baseline(x: np.ndarray) -> dict:
    """The oracle as it stands on the host cores, on a bounded sample."""
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    xs = x[: 1 << 26]
    s = np.empty_like(xs)
    c = np.empty_like(xs)
    # about 20 s of CPU work: 1.5 s of wall time on 16 cores, or 20 passes
    reps, used, t0 = 0, 0, time.perf_counter()
    while reps < 2 or (time.perf_counter() - t0 < 20.0 / cores and reps < 200) or reps < 20:
        used = oracle.sincos_mt(xs, s, c, threads=cores)
        reps += 1
    dt = time.perf_counter() - t0
    # the same oracle on one thread, for the per-core rate
    x1 = xs[: 1 << 24]
    reps1, t1 = 0, time.perf_counter()
    while reps1 < 1 or (time.perf_counter() - t1 < 2.0 and reps1 < 10):
        oracle.sincos_mt(x1, s[: x1.size], c[: x1.size], threads=1)
        reps1 += 1
    dt1 = time.perf_counter() - t1
    return {"value": xs.size * reps / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"first 2^26 angles of the {WORKLOAD} workload, {reps} passes, "
                      f"{dt:.1f} s wall on {used} threads",
            "single_thread": {"value": x1.size * reps1 / dt1, "unit": UNIT,
                              "sample": f"first 2^24 angles, {reps1} passes, {dt1:.1f} s"}}


def cuda_libm_context(torch, x_np, x, s, c, dist, steps: int) -> dict:
    """CUDA's sincosf and __sincosf on the same 2^28 angles and buffers, for
    context: GB/s and FP64 errors on a sample.  sincosf is timed under each
    nvcc flag set of the context build (defaults, -use_fast_math, and the
    -prec-div/-prec-sqrt/-ftz switches alone); __sincosf under the defaults."""
    import ctypes
    from paper_cs_0406049_gb300 import build as libbuild
    out = {}
    n = x.numel()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, n, 1 << 20)
    it = torch.from_numpy(idx).cuda()
    for variant, path in libbuild.build_context_all().items():
        lib = ctypes.CDLL(path)
        lib.context_libm_sincos.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
        cases = (("sincosf", 0), ("__sincosf", 1)) if variant == "default" else (("sincosf", 0),)
        for name, fast in cases:
            st = torch.cuda.current_stream().cuda_stream
            run = lambda: lib.context_libm_sincos(x.data_ptr(), s.data_ptr(), c.data_ptr(), n,
                                                  fast, st)
            total, ms, _ = time_loop(torch, run, steps, 3, dist)
            err = fp64_errors(x_np[idx], s[it].cpu().numpy().astype(np.float64),
                              c[it].cpu().numpy().astype(np.float64))
            key = name if variant == "default" else f"{name} [{variant}]"
            out[key] = {"pairs_per_s": n / (ms * 1e-3), "gbs": 12 * n / (ms * 1e-3) / 1e9,
                        "nvcc_flags": " ".join(libbuild.CONTEXT_VARIANTS[variant]) or "defaults",
                        "errors": err}
    return out


def extras(torch, api, workloads, dist, steps_hint: int, autotune: bool) -> dict:
    """Secondary workloads, each with its own GB/s and errors (not the headline)."""
    out = {}
    k = max(20, min(steps_hint, 200))
    peak, _ = measured_peak()
    vendor = vendor_peak(torch, 1.0).get("peak_vendor")   # nominal HBM GB/s, or None

    def of_vendor(gbs):
        return gbs / vendor if vendor else None

    # plain: 2^20 angles U[-pi, pi) (12.6 MB, L2-resident), L2 flushed before
    # every call (the flush also keeps the host ahead of the GPU, so the event
    # pair times the kernel, not the launch path); launch-bound, reported with
    # the paper's accuracy statistics
    x = workloads.plain()
    xt = torch.from_numpy(x).cuda()
    s = torch.empty_like(xt)
    c = torch.empty_like(xt)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")   # 256 MB > L2
    if autotune:
        api.sincos_autotune_pairs(xt, s, c)
    per = time_flushed(torch, lambda: api.sincos_pairs(xt, s, c), max(30, k // 4), 3, flush)
    ms = statistics.median(per)
    # floors taken the same way: a one-element torch kernel, and torch's x * 2
    # into s (4 MB read, 4 MB written).  The event timestamps of these short
    # calls come in steps of about 2 us on GB300, so the medians do too.
    tiny = torch.zeros(1, device="cuda")
    floor_empty = statistics.median(time_flushed(torch, lambda: tiny.add_(1.0), max(30, k // 4), 3,
                                                 flush))
    floor_mul = statistics.median(time_flushed(torch, lambda: torch.mul(xt, 2.0, out=s),
                                               max(30, k // 4), 3, flush))
    del tiny
    api.sincos_pairs(xt, s, c)
    torch.cuda.synchronize()
    s_np, c_np = s.cpu().numpy(), c.cpu().numpy()
    out["plain_2p20"] = {
        "pairs_per_s": x.size / (ms * 1e-3), "us_per_call": 1e3 * ms,
        "l2_flushed": True, "bound": "launch and ramp (12.6 MB: about 2 us of HBM time)",
        "floor_us": {"empty_one_element_kernel": 1e3 * floor_empty,
                     "torch_mul_4MB_in_4MB_out": 1e3 * floor_mul},
        "errors": fp64_errors(x, s_np.astype(np.float64), c_np.astype(np.float64)),
        "accuracy": e1_stats(x, s_np, c_np),
        "accuracy_paper": {"rms_euclid": 1.2e-7, "max_euclid": 4.8e-7, "max_amplitude": 1.8e-7,
                           "source": "Sec. Results, normalized set (domain not stated)"},
        "plan": api.sincos_plan_get("pairs", "f32", x.size)}
    del xt, s, c, flush

    # precision: 2^26 angles, |x| log-uniform in [1e-3, 1e5], four variants
    x = workloads.precision()
    xt = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(0)
    idx = torch.from_numpy(rng.integers(0, x.size, 1 << 20)).cuda()
    prec = {}
    for name, dt, red, coef in (("f32_plain", torch.float32, "plain", "normalized"),
                                ("f32_compensated", torch.float32, "compensated", "normalized"),
                                ("f32_plain_dagger", torch.float32, "plain", "dagger"),
                                ("bf16_compensated", torch.bfloat16, "compensated", "normalized"),
                                ("f16_compensated", torch.float16, "compensated", "normalized")):
        s = torch.empty(x.size, dtype=dt, device="cuda")
        c = torch.empty_like(s)
        if autotune:
            api.sincos_autotune_pairs(xt, s, c, red, coef)
        total, ms, _ = time_loop(torch, lambda: api.sincos_pairs_ex(xt, s, c, red, coef), k, 3,
                                  dist)
        bytes_ = x.size * (4 + 2 * s.element_size())
        err = fp64_errors(x[idx.cpu().numpy()], s[idx].float().cpu().numpy().astype(np.float64),
                          c[idx].float().cpu().numpy().astype(np.float64))
        prec[name] = {"pairs_per_s": x.size / (ms * 1e-3), "gbs": bytes_ / (ms * 1e-3) / 1e9,
                      "frac_of_peak": bytes_ / (ms * 1e-3) / 1e9 / peak,
                      "frac_of_vendor_peak": of_vendor(bytes_ / (ms * 1e-3) / 1e9),
                      "ms": ms, "errors": err,
                      "plan": api.sincos_plan_get("pairs", dt, x.size)}
        del s, c
    out["precision_2p26"] = prec

    # exp(i x) as interleaved complex64 on the same angles: 12 B per angle
    z = torch.empty(x.size, dtype=torch.complex64, device="cuda")
    if autotune:
        api.sincos_autotune_expi(xt, z)
    total, ms, _ = time_loop(torch, lambda: api.sincos_expi(xt, z), k, 3, dist)
    zs = torch.view_as_real(z[idx]).cpu().numpy().astype(np.float64)
    out["expi_complex64_2p26"] = {"gbs": 12 * x.size / (ms * 1e-3) / 1e9, "ms": ms,
                                  "frac_of_peak": 12 * x.size / (ms * 1e-3) / 1e9 / peak,
                                  "frac_of_vendor_peak": of_vendor(12 * x.size / (ms * 1e-3) / 1e9),
                                  "reduction": "plain",
                                  "errors": fp64_errors(x[idx.cpu().numpy()], zs[:, 1], zs[:, 0]),
                                  "plan": api.sincos_plan_get("expi", "f32", x.size)}
    del z, xt

    # Huygens field sum (ALU-bound): 512 x 512 points, 4096 sources
    w = workloads.diffraction()
    P = tuple(torch.from_numpy(v).cuda() for v in w.p)
    Q = tuple(torch.from_numpy(v).cuda() for v in w.q)
    A = torch.from_numpy(w.a).cuda()
    m, nsrc = w.p[0].size, w.q[0].size
    u = torch.empty(m, dtype=torch.complex64, device="cuda")
    if autotune:
        api.sincos_autotune_huygens(P, Q, A, w.k, u)
    sampler = ClockSampler(gpu_query_id(torch)) if dist.rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    t0 = time.time()
    total, ms, _ = time_loop(torch, lambda: api.sincos_huygens(P, Q, A, w.k, u),
                              max(20, k // 4), 3, dist)
    clocks = sampler.summary(t0, time.time()) if sampler else None
    if sampler:
        sampler.stop()
    terms = m * nsrc
    u_np = torch.view_as_real(u).cpu().numpy()
    hy_err = huygens_fp64_errors(w, u_np, np.random.default_rng(0).choice(m, 256, replace=False))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    max_mhz = measured_sm_max_mhz()
    achieved = terms * HUYGENS_OPS_PER_TERM / (ms * 1e-3) / 1e12
    peak_alu = sms * FP32_LANES_PER_SM * max_mhz * 1e6 / 1e12
    out["diffraction_512x512_4096"] = {
        "terms_per_s": terms / (ms * 1e-3), "ms": ms, "terms": terms,
        "plan": api.sincos_plan_get("huygens", "f32", m),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_alu,
                     "unit": "TFLOP32-ops/s", "frac": achieved / peak_alu,
                     "peak_kind": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {max_mhz} MHz",
                     "ops_per_term": HUYGENS_OPS_PER_TERM,
                     "fma_pipe_ops_per_term_bit_exact": HUYGENS_FMA_OPS_BIT_EXACT,
                     "ceiling_bit_exact_terms_per_s": peak_alu * 1e12 / HUYGENS_FMA_OPS_BIT_EXACT,
                     "frac_of_bit_exact_ceiling": terms / (ms * 1e-3) /
                                                  (peak_alu * 1e12 / HUYGENS_FMA_OPS_BIT_EXACT)},
        "errors": hy_err,
        "clocks": clocks}
    del P, Q, A, u

    # backward: 2^26 angles U[-50, 50), gs, gc ~ N(0, 1): 20 B per element
    w = workloads.differentiation_inputs()
    xt = torch.from_numpy(w.x).cuda()
    gs = torch.from_numpy(w.gs).cuda()
    gc = torch.from_numpy(w.gc).cuda()
    s = torch.empty_like(xt)
    c = torch.empty_like(xt)
    api.sincos_pairs(xt, s, c)
    gx = torch.empty_like(xt)
    if autotune:
        api.sincos_autotune_backward(gs, gc, s, c, gx)
    total, ms, _ = time_loop(torch, lambda: api.sincos_backward(gs, gc, s, c, gx), k, 3, dist)
    bwd = {"gbs": 20 * xt.numel() / (ms * 1e-3) / 1e9, "ms": ms,
           "plan": api.sincos_plan_get("backward", "f32", xt.numel())}
    bwd["frac_of_peak"] = bwd["gbs"] / peak
    bwd["frac_of_vendor_peak"] = of_vendor(bwd["gbs"])
    di = np.random.default_rng(0).integers(0, w.x.size, 1 << 20)
    dit = torch.from_numpy(di).cuda()
    bwd["errors"] = {
        "forward": fp64_errors(w.x[di], s[dit].cpu().numpy().astype(np.float64),
                               c[dit].cpu().numpy().astype(np.float64)),
        "backward": backward_fp64_errors(w.x[di], w.gs[di], w.gc[di], gx[dit].cpu().numpy())}
    xg = xt.clone().requires_grad_(True)

    def fwd_bwd():
        ss, cc = api.sincos_autograd(xg)
        torch.autograd.backward([ss, cc], [gs, gc])
        xg.grad = None
    total, ms, _ = time_loop(torch, fwd_bwd, max(10, k // 4), 3, dist)
    bwd["autograd_fwd_bwd_ms"] = ms
    out["differentiation_2p26"] = bwd
    del xt, gs, gc, s, c, gx, xg

    # batching: 4096 arrays packed back to back, one persistent launch vs
    # its CUDA graph vs 4096 single-array launches (direct and graph-captured)
    b = workloads.batching()
    xt = torch.from_numpy(b.angles).cuda()
    s = torch.empty_like(xt)
    c = torch.empty_like(xt)
    segs, lens = api.segments(xt, s, c, b.offsets, b.lens)
    bytes_ = BYTES_PER_PAIR * b.total
    bat = {"total_pairs": b.total, "count": b.count}
    if autotune:
        api.sincos_autotune_batched(segs, lens)
    bat["plan"] = api.sincos_plan_get("batched", "f32", b.count)
    total, ms, _ = time_loop(torch, lambda: api.sincos_batched(segs, lens), k, 3, dist)
    bat["persistent_gbs"] = bytes_ / (ms * 1e-3) / 1e9
    g = api.BatchedGraph(segs, lens)
    total, ms, _ = time_loop(torch, g.launch, k, 3, dist)
    bat["graph_gbs"] = bytes_ / (ms * 1e-3) / 1e9
    bat["graph_frac_of_peak"] = bat["graph_gbs"] / peak
    bat["graph_frac_of_vendor_peak"] = of_vendor(bat["graph_gbs"])
    g.close()
    offs = b.offsets.tolist()
    ln = b.lens.tolist()
    views = [(xt[o:o + n], s[o:o + n], c[o:o + n]) for o, n in zip(offs, ln)]

    def separate():
        for v in views:
            api.sincos_pairs(*v)
    total, ms, _ = time_loop(torch, separate, 5, 1, dist)
    bat["separate_launches_gbs"] = bytes_ / (ms * 1e-3) / 1e9
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        separate()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=cap):
            separate()
    torch.cuda.synchronize()
    total, ms, _ = time_loop(torch, graph.replay, 10, 2, dist)
    bat["separate_launches_graph_gbs"] = bytes_ / (ms * 1e-3) / 1e9
    del graph
    bi = batch_sample(b.offsets, b.lens)
    bit = torch.from_numpy(bi).cuda()
    bat["errors"] = fp64_errors(b.angles[bi], s[bit].cpu().numpy().astype(np.float64),
                                c[bit].cpu().numpy().astype(np.float64))
    bat["errors"]["sample_kind"] = "first and last 64 and 64 random angles of every array"
    out["batching_4096"] = bat
    return out


def run_ours(args, dist: Dist):
    import torch
    from paper_cs_0406049_gb300 import api, workloads
    from paper_cs_0406049_gb300 import build as libbuild

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU fallback)")
    torch.cuda.set_device(dist.local)
    dist.init("nccl")
    libbuild.build()
    api.lib()
    dev_name = torch.cuda.get_device_name()

    x_np = workloads.bandwidth()
    n_total = x_np.size
    lo, hi = shard_bounds(n_total, dist.rank, dist.world) if args.split else (0, n_total)
    x_np = np.ascontiguousarray(x_np[lo:hi])
    n = x_np.size                       # this rank's angles
    x = torch.from_numpy(x_np).cuda()
    s = torch.empty_like(x)
    c = torch.empty_like(x)
    if not args.no_autotune:
        api.sincos_autotune_pairs(x, s, c)
    plan = api.sincos_plan_get("pairs", "f32", n)

    sampler = ClockSampler(gpu_query_id(torch)) if dist.rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    launches0 = api.sincos_launch_count()
    total_ms, kernel_ms, clocks = time_loop(torch, lambda: api.sincos_pairs(x, s, c), args.steps,
                                            args.warmup, dist, sampler)
    launches = api.sincos_launch_count() - launches0 - args.warmup
    # re-measure once if the clocks show a thermal or hardware slowdown
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    remeasured = False
    if clocks and bad & set(clocks.get("reasons", [])):
        remeasured = True
        launches0 = api.sincos_launch_count()
        total_ms, kernel_ms, clocks = time_loop(torch, lambda: api.sincos_pairs(x, s, c),
                                                args.steps, args.warmup, dist, sampler)
        launches = api.sincos_launch_count() - launches0 - args.warmup
    if sampler:
        sampler.stop()
    # bounded waits in the kernels that gave up (read after the timed region:
    # the read synchronizes the device)
    wait_timeouts = int(api.sincos_device_wait_timeouts())
    max_ms = dist.max(total_ms)
    # whole-job pairs/s: the slowest rank's time bounds the job
    value = (n_total * args.steps / (max_ms * 1e-3) if args.split
             else aggregate_value(dist.world, n, args.steps, max_ms))
    peak, peak_kind = measured_peak()
    achieved = BYTES_PER_PAIR * n / (kernel_ms * 1e-3) / 1e9
    traffic = profiled_traffic()
    # the same copy measurement as the peak, on this machine now (boxes differ)
    live_copy = live_copy_gbs(torch)

    rng = np.random.default_rng(0)
    idx = rng.integers(0, n, 1 << 20)
    it = torch.from_numpy(idx).cuda()
    err = fp64_errors(x_np[idx], s[it].cpu().numpy().astype(np.float64),
                      c[it].cpu().numpy().astype(np.float64))

    e2e = None
    if not args.no_e2e:
        (xh, sh, ch), placed = pinned_near_gpu(
            torch, torch.cuda.current_device(),
            lambda: (torch.from_numpy(x_np).pin_memory(),
                     torch.empty(n, dtype=torch.float32).pin_memory(),
                     torch.empty(n, dtype=torch.float32).pin_memory()))
        ws = torch.empty(api.sincos_host_workspace_bytes("f32", 1 << 24), dtype=torch.uint8,
                         device="cuda")
        e_steps = max(3, min(args.steps, 10))
        tot, _, _ = time_loop(torch, lambda: api.sincos_pairs_host(xh, sh, ch, ws), e_steps,
                                  2, dist)
        tot = dist.max(tot)
        route = api.sincos_host_last_path()
        assert torch.equal(sh[:1024], s[:1024].cpu()), "host path differs from device path"
        e2e = {"value": (n_total if args.split else dist.world * n) * e_steps / (tot * 1e-3),
               "unit": UNIT,
               "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 8 * n,
               "ms_per_step": tot / e_steps,
               "path": route,
               "path_note": E2E_ROUTES.get(route, route),
               "host_buffers_pinned": placed}
        del xh, sh, ch
        if not args.no_extras:
            # the same call on ordinary (pageable) host memory: what a caller
            # without page-locked buffers gets (zero-copy where the device
            # reaches pageable memory), and the copy pipeline on it for context
            # (outputs written once by the CPU first: a page the GPU touches
            # first is populated by that call, about 0.65 s for 2 GiB).  Each
            # call is timed alone and the median reported: the driver's
            # staging of pageable copies makes some pipeline calls 4-18 times
            # slower than the rest (74-322 ms against 18 ms).
            xp = torch.from_numpy(x_np)
            sp, cp = torch.empty(n, dtype=torch.float32), torch.empty(n, dtype=torch.float32)
            sp.fill_(0.0)
            cp.fill_(0.0)
            for key, policy, p_steps in (("pageable", "auto", 5), ("pageable_pipeline", "pipeline", 7)):
                api.sincos_host_route_set(policy)
                try:
                    per = time_each(torch, lambda: api.sincos_pairs_host(xp, sp, cp, ws),
                                    p_steps, 2, dist)
                    route_p = api.sincos_host_last_path()
                finally:
                    api.sincos_host_route_set("auto")
                tp = statistics.median(per)
                e2e[key] = {"value": (n_total if args.split else dist.world * n) / (tp * 1e-3),
                            "unit": UNIT, "ms_per_step": tp, "ms_min": min(per),
                            "ms_max": max(per), "steps": p_steps,
                            "timing": "median of calls timed one at a time",
                            "path": route_p}
            assert torch.equal(sp[:1024], s[:1024].cpu()), "pageable path differs from device path"
            del xp, sp, cp
        del ws

    ext = None
    if not args.no_extras:
        libm = cuda_libm_context(torch, x_np, x, s, c, dist, max(20, min(args.steps, 100)))
        del s, c
        ext = extras(torch, api, workloads, dist, args.steps, not args.no_autotune)
        ext["context_cuda_libm_2p28"] = libm

    cpu = None
    if dist.rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(x_np)

    if ext is not None:
        # the batched and backward forms against the headline kernel's GB/s
        ext["batching_4096"]["graph_vs_forward_gbs"] = ext["batching_4096"]["graph_gbs"] / achieved
        ext["differentiation_2p26"]["backward_vs_forward_gbs"] = \
            ext["differentiation_2p26"]["gbs"] / achieved

    wait_timeouts += int(api.sincos_device_wait_timeouts())
    if dist.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "strong" if args.split else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC, "n": n,
                       "out_dtype": "f32", "reduction": "plain", "coef": "normalized",
                       "plan": plan, "l2": "inputs larger than L2 (3.2 GB per step vs 129 MB)",
                       "parallelism": (f"one {n_total}-angle array in {dist.world} contiguous "
                                       f"blocks, one per GPU, no collective on the data"
                                       if args.split else
                                       f"independent {n}-angle arrays per GPU x{dist.world}"),
                       "device": dev_name, "remeasured_for_clocks": remeasured},
            "gbs": achieved * dist.world,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "kernel": (f"k_forward_bulk<float, plain, normalized, {plan['block']}, "
                                    f"{4096 if plan['ctas_per_sm'] >= 2 else 8192}>"
                                    if plan["vec_bytes"] == 0 else
                                    f"k_forward<float, plain, normalized, {plan['unroll']}, "
                                    f"{plan['vec_bytes']}>"),
                         "bytes_per_launch": BYTES_PER_PAIR * n, "kernel_ms": kernel_ms,
                         "peak_live_copy": live_copy, "frac_of_live_copy": achieved / live_copy,
                         **vendor_peak(torch, achieved)},
            "errors_vs_fp64": err,
            "paper_context": PAPER_CONTEXT,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "wait_timeouts": wait_timeouts,
            "clocks": clocks,
            "impl": "ours",
        }
        if ext is not None:
            line["extras"] = ext
        print(json.dumps(line), flush=True)
    dist.close()
    if wait_timeouts:
        sys.stderr.write(f"bench: {wait_timeouts} bounded waits gave up inside the kernels; "
                         "some launches stopped early and the numbers above are not valid\n")
        raise SystemExit(3)


def main():
    args = parse_args()
    dist = Dist(args.gpus)
    if args.impl == "reference":
        run_reference(args, dist)
        return
    run_ours(args, dist)


if __name__ == "__main__":
    main()
