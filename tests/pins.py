"""Pins for the CPU oracle: checks against what the paper and mathematics fix.

Each ``pin_*`` function raises ``AssertionError`` when the oracle it is given
breaks the fact it encodes.  ``test_oracle_pins.py`` runs them on the real
oracle; ``test_oracle_mutations.py`` runs them on copies of the oracle with a
planted mistake and requires at least one to fail.  Nothing here retypes the
oracle's formulas: the references are FP64 library sin/cos, printed numbers,
analytic bounds, library roundings (numpy float16, torch bfloat16) and exact
invariants of the method.
"""
from __future__ import annotations

import math
import os
import re

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def paper_coefficients() -> dict:
    return {r[0]: r[1] for r in _golden_rows("paper_coefficients.txt")}


def paper_error_bounds() -> dict:
    return {r[0]: (float(r[1]), float(r[2])) for r in _golden_rows("paper_error_stats.txt")}


def _stats(x, s, c):
    import oracle
    return oracle.error_stats(x, s, c)


def evenly_spaced(n: int) -> np.ndarray:
    return np.linspace(-math.pi, math.pi, n, endpoint=False).astype(np.float32)


K32 = np.float32(1.0 / (2.0 * 3.1415926536))   # the paper's scale, for building test angles


def angles_with_scaled_value(targets, keep_missing: bool = False) -> np.ndarray:
    """For each exact binary32 target t, a binary32 x with fl(x*K) == t.

    Searches 300 ulps either side of t/K.  Targets with no solution are
    dropped, or returned as NaN when ``keep_missing`` is set."""
    t = np.asarray(targets, np.float32).ravel()
    x0 = (t.astype(np.float64) / np.float64(K32)).astype(np.float32)
    offs = np.arange(-300, 301, dtype=np.int32)
    cand = (x0.view(np.int32)[:, None] + offs[None, :]).view(np.float32)
    hit = (cand * K32) == t[:, None]
    found = hit.any(axis=1)
    # the hit closest to the middle of the window
    dist = np.where(hit, np.abs(offs)[None, :], 1 << 20)
    pick = cand[np.arange(t.size), dist.argmin(axis=1)]
    if keep_missing:
        return np.where(found, pick, np.float32(np.nan)).astype(np.float32)
    return pick[found].astype(np.float32)


# ----------------------------------------------------------------------------
# Source-level pin: the printed coefficients.
# ----------------------------------------------------------------------------

def pin_coefficients_source(src_text: str):
    """The oracle's literal coefficients are the paper's printed decimals."""
    want = paper_coefficients()
    for name, dec in want.items():
        m = re.search(r"\b%s\s*=\s*\(float\)\s*([-+0-9.eE]+)\s*;" % name, src_text)
        assert m, f"{name} not found in oracle source"
        assert float(m.group(1)) == float(dec), (name, m.group(1), dec)
    m = re.search(r"#define\s+ORC_K\s+\(\(float\)\(1\.0 / \(2\.0 \* ([0-9.]+)\)\)\)", src_text)
    assert m and m.group(1) == "3.1415926536", "scale factor is not the paper's 1/(2*3.1415926536)"


# ----------------------------------------------------------------------------
# Printed error statistics (E1, E2).
# ----------------------------------------------------------------------------

def pin_e1_normalized(lib, n: int = 1 << 24):
    b = paper_error_bounds()
    x = evenly_spaced(n)
    s, c = lib.sincos(x)
    st = _stats(x, s, c)
    assert st["rms_euclid"] <= b["normalized.rms_euclid"][1], st
    assert st["max_euclid"] <= b["normalized.max_euclid"][1], st
    assert st["max_amp"] <= b["normalized.max_amp"][1], st
    return st


def pin_e2_dagger(lib, n: int = 1 << 24):
    b = paper_error_bounds()
    x = evenly_spaced(n)
    s, c = lib.sincos(x, coef="dagger")
    st = _stats(x, s, c)
    assert st["rms_euclid"] <= b["dagger.rms_euclid"][1], st
    assert st["max_euclid"] <= b["dagger.max_euclid"][1], st
    return st


# ----------------------------------------------------------------------------
# Brute force against FP64 on every binary32 in small ranges.
# ----------------------------------------------------------------------------

def all_floats(lo: float, hi: float) -> np.ndarray:
    a = np.float32(lo).view(np.int32)
    b = np.float32(hi).view(np.int32)
    return np.arange(a, b, dtype=np.int32).view(np.float32)


def core_error(x, s, c) -> np.ndarray:
    """Euclidean error against FP64 (sin, cos)(2 pi fl(x*K)): the error of the
    method at the reduced angle it actually sees, excluding the reduction's."""
    x1 = (np.asarray(x, np.float32) * K32).astype(np.float64)
    return np.hypot(s - np.sin(2 * np.pi * x1), c - np.cos(2 * np.pi * x1))


def reduction_bound(x) -> np.ndarray:
    """Angle error of the plain reduction: fl(x*K) is within ulp(x1)/2 of x*K,
    and K within |K|*2^-24 of 1/(2 pi), so at most 2 pi (ulp(x1)/2 + |x1| 2^-24)."""
    x1 = np.abs(np.asarray(x, np.float32) * K32)
    return 2 * math.pi * (np.spacing(x1).astype(np.float64) / 2 + x1.astype(np.float64) * 2.0 ** -24)


CORE_BOUND = 5.0e-7     # the paper prints 4.8e-7 as the maximum error (first method)


def pin_bruteforce(lib, ranges=((0.5, 1.0), (1.0, 2.0), (2.0, 4.0), (4.0, 8.0))):
    """Every binary32 in each range, against FP64.

    Plain reduction: core error <= 5e-7 and total error <= 5e-7 plus the
    reduction bound.  Compensated reduction: total error <= 7e-7."""
    for lo, hi in ranges:
        x = all_floats(lo, hi)
        s, c = lib.sincos(x)
        assert core_error(x, s, c).max() <= CORE_BOUND, (lo, hi)
        rs, rc = np.sin(x.astype(np.float64)), np.cos(x.astype(np.float64))
        total = np.hypot(s - rs, c - rc)
        assert np.all(total <= CORE_BOUND + reduction_bound(x)), (lo, hi)
        s, c = lib.sincos(x, reduction="compensated")
        assert np.hypot(s - rs, c - rc).max() <= 7e-7, (lo, hi)


def _bruteforce_bits(lib_cls, path, lo_bits, hi_bits):
    """Worker of pin_bruteforce_small_angles: every positive binary32 whose bit
    pattern is in [lo_bits, hi_bits), against FP64.  Returns the largest core
    error, the largest excess of the plain total error over its bound, and the
    largest compensated error."""
    lib = lib_cls(path)
    x = np.arange(lo_bits, hi_bits, dtype=np.int32).view(np.float32)
    s, c = lib.sincos(x)
    core = float(core_error(x, s, c).max())
    rs, rc = np.sin(x.astype(np.float64)), np.cos(x.astype(np.float64))
    excess = float((np.hypot(s - rs, c - rc) - reduction_bound(x)).max())
    s, c = lib.sincos(x, reduction="compensated")
    comp = float(np.hypot(s - rs, c - rc).max())
    return core, excess, comp


def pin_bruteforce_small_angles(lib, processes: int | None = None):
    """Every binary32 in [0, 1/2), zero and subnormals included, one binade per
    task over a spawned process pool: the same bounds as pin_bruteforce.  With
    pin_bruteforce ([1/2, 8)) and pin_symmetry this covers every float in
    [-pi, pi)."""
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor

    top = int(np.float32(0.5).view(np.int32))
    step = 1 << 23                                  # one binade of bit patterns
    tasks = [(b, min(b + step, top)) for b in range(0, top, step)]
    workers = processes or min(8, len(os.sched_getaffinity(0)))
    with ProcessPoolExecutor(workers, mp_context=multiprocessing.get_context("spawn")) as ex:
        futs = [ex.submit(_bruteforce_bits, type(lib), lib.path, lo, hi) for lo, hi in tasks]
        results = [f.result() for f in futs]
    for (lo, hi), (core, excess, comp) in zip(tasks, results):
        where = (float(np.int32(lo).view(np.float32)), float(np.int32(hi).view(np.float32)))
        assert core <= CORE_BOUND, (where, core)
        assert excess <= CORE_BOUND, (where, excess)
        assert comp <= 7e-7, (where, comp)


# ----------------------------------------------------------------------------
# Exact invariants.
# ----------------------------------------------------------------------------

def symmetry_angles(n: int = 1 << 20, seed: int = 11) -> np.ndarray:
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(-40, 38, n)
    x = mag.astype(np.float32)
    x[: n // 4] = rng.uniform(0, 2000, n // 4).astype(np.float32)
    return x


def pin_symmetry(lib):
    """s(-x) == -s(x) and c(-x) == c(x) for every x (rint is sign-symmetric)."""
    x = symmetry_angles()
    for red in ("plain", "compensated"):
        for coef in ("normalized", "dagger"):
            s, c = lib.sincos(x, reduction=red, coef=coef)
            sn, cn = lib.sincos(-x, reduction=red, coef=coef)
            assert np.array_equal(sn, -s), (red, coef)
            assert np.array_equal(cn, c), (red, coef)


def periodic_pairs(n: int = 8192, seed: int = 12):
    """Angle pairs (x, y) with fl(y*K) == fl(x*K) + k exactly for integer k != 0."""
    rng = np.random.default_rng(seed)
    t = (rng.integers(-2047, 2048, n) / 4096.0).astype(np.float32)
    k = rng.integers(1, 2000, n)
    ty = (t.astype(np.float64) + k).astype(np.float32)     # exact: <= 23 significant bits
    x = angles_with_scaled_value(t, keep_missing=True)
    y = angles_with_scaled_value(ty, keep_missing=True)
    ok = ~np.isnan(x) & ~np.isnan(y)
    return x[ok], y[ok]


def pin_periodicity(lib):
    """Angles whose scaled values differ by an integer give bit-identical pairs."""
    x, y = periodic_pairs()
    assert x.size > 1000
    s, c = lib.sincos(x)
    sy, cy = lib.sincos(y)
    assert np.array_equal(s, sy) and np.array_equal(c, cy)


def pin_exact_at_whole_turns(lib):
    """fl(x*K) an integer -> reduced angle 0 -> (s, c) == (0, 1) exactly."""
    x = angles_with_scaled_value(np.arange(-4000, 4001, 3, dtype=np.float32))
    x = np.concatenate([x, np.float32([0.0, -0.0])])
    assert x.size > 1500
    s, c = lib.sincos(x)
    assert np.all(s == 0.0) and np.all(c == 1.0)


def pin_quarter_turns(lib, bound: float = 3.5e-7):
    """fl(x*K) in Z/4 -> within 3.5e-7 of the exact (sin, cos)(2 pi fl(x*K))."""
    t = (np.arange(-2000, 2001, dtype=np.float64) / 4.0).astype(np.float32)
    x = angles_with_scaled_value(t)
    x1 = (x * K32).astype(np.float64)
    q = x1 - np.round(x1)            # exact quarter turns: 0, +-1/4, +-1/2
    quadrant = np.rint(q * 4).astype(int) % 4
    exact_s = np.array([0.0, 1.0, 0.0, -1.0])[quadrant]
    exact_c = np.array([1.0, 0.0, -1.0, 0.0])[quadrant]
    s, c = lib.sincos(x)
    assert np.max(np.abs(s - exact_s)) <= bound
    assert np.max(np.abs(c - exact_c)) <= bound


def pin_ties_to_even(lib):
    """fl(x*K) = k + 1/2 reduces to +1/2 for even k and -1/2 for odd k.

    AltiVec vec_round rounds to nearest with ties to even, so the sine of a
    half-turn tie alternates its tiny sign with the parity of k."""
    t = np.float32([0.5, 1.5, 2.5, 3.5, 4.5, 5.5])
    x = angles_with_scaled_value(t)
    assert x.size == t.size
    s, c = lib.sincos(x)
    assert np.all(np.abs(s) <= 3.5e-7) and np.all(np.abs(c + 1.0) <= 3.5e-7)
    assert s[0] != 0.0
    assert np.all(s[0::2] == s[0]) and np.all(s[1::2] == -s[0])


def pin_special_values(lib):
    """NaN and +-Inf give NaN; |fl(x*K)| >= 2^23 reduces to 0 -> (0, 1) exactly."""
    x = np.float32([np.nan, np.inf, -np.inf])
    for red in ("plain", "compensated"):
        s, c = lib.sincos(x, reduction=red)
        assert np.all(np.isnan(s)) and np.all(np.isnan(c)), red
    huge = np.float32([2.0 ** 26, -2.0 ** 26, 1e20, -3e38, 2.0 ** 30 + 128])
    s, c = lib.sincos(huge)
    assert np.all(s == 0.0) and np.all(c == 1.0)
    s, c = lib.sincos(huge, reduction="compensated")
    assert np.all(np.isfinite(s)) and np.all(np.isfinite(c))
    assert np.all(np.abs(np.hypot(s.astype(np.float64), c) - 1.0) <= 2e-7)
    tiny = np.float32([1e-30, -1e-30, 1e-40, -1e-40, 1e-45, 2.0 ** -126])
    s, c = lib.sincos(tiny)
    assert np.all(c == 1.0)
    # a handful of roundings on the subnormal grid (2^-149) on top of 1e-6 relative
    err = np.abs(s.astype(np.float64) - np.sin(tiny.astype(np.float64)))
    assert np.all(err <= 1e-6 * np.abs(tiny) + 2.0 ** -144), err


def pin_plain_reduction_bound(lib, n: int = 1 << 20):
    """Plain reduction on [-1000, 1000): each pair within the core bound plus
    the analytic reduction bound of FP64, and within the core bound of FP64
    at the reduced angle."""
    rng = np.random.default_rng(13)
    x = rng.uniform(-1000, 1000, n).astype(np.float32)
    s, c = lib.sincos(x)
    rs, rc = np.sin(x.astype(np.float64)), np.cos(x.astype(np.float64))
    assert np.all(np.hypot(s - rs, c - rc) <= CORE_BOUND + reduction_bound(x))
    assert core_error(x, s, c).max() <= CORE_BOUND


def pin_compensated(lib, bound: float = 7e-7):
    """Compensated reduction: within 7e-7 of FP64 up to |x| = 1e5."""
    rng = np.random.default_rng(14)
    x = np.concatenate([
        rng.uniform(-1e5, 1e5, 1 << 20),
        (10.0 ** rng.uniform(-3, 5, 1 << 20)) * np.where(rng.random(1 << 20) < 0.5, -1, 1),
        [1e5, -1e5, 99999.99, 65536.0, 8192.0 * math.pi],
    ]).astype(np.float32)
    s, c = lib.sincos(x, reduction="compensated")
    st = _stats(x, s, c)
    assert st["max_abs"] <= bound, st


def pin_drift_correction(lib):
    """Drift correction: the corrected pair has |1 - |(s, c)|| <= 2e-7.

    Without it the two doublings leave the quarter-angle pair's amplitude error
    multiplied by four (Section "Methodology": a^(2n) ~ 1 + 2n eps), about
    5e-7 here; the correction cancels it to first order."""
    x = evenly_spaced(1 << 22)
    s, c = lib.sincos(x)
    amp = np.abs(1.0 - np.hypot(s.astype(np.float64), c.astype(np.float64)))
    assert amp.max() <= 2e-7, amp.max()


# ----------------------------------------------------------------------------
# 16-bit output rounding against library conversions.
# ----------------------------------------------------------------------------

def rounding_sweep(seed: int = 15) -> np.ndarray:
    rng = np.random.default_rng(seed)
    bits = [rng.integers(0, 2 ** 32, 1 << 20, dtype=np.uint64).astype(np.uint32)]
    # every pattern near fp16 / bf16 rounding boundaries and the fp16 subnormal range
    base = np.arange(0, 1 << 16, dtype=np.uint32)
    for e in (0x33000000, 0x33800000, 0x38000000, 0x38800000, 0x3f000000, 0x3f800000,
              0x477f0000, 0x477fe000, 0x00000000, 0x7f7f0000):
        bits.append(e + base)
        bits.append((e + base) | 0x80000000)
    # exact ties: low 16 bits 0x8000 (bf16) and low 13 bits 0x1000 (fp16)
    hi = rng.integers(0, 2 ** 16, 1 << 14, dtype=np.uint64).astype(np.uint32) << 16
    bits.append(hi | 0x8000)
    mid = rng.integers(0x38800000 >> 13, 0x477fe000 >> 13, 1 << 14,
                       dtype=np.uint64).astype(np.uint32) << 13
    bits.append(mid | 0x1000)
    v = np.concatenate(bits).view(np.float32)
    return v[~np.isnan(v)]


def pin_bf16_rounding(lib):
    """Hand-written bf16 RNE == torch's float32 -> bfloat16 conversion."""
    import torch
    v = rounding_sweep()
    got = lib.round16(v, "bf16")
    want = torch.from_numpy(v.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got, want)
    nan = lib.round16(np.float32([np.nan]), "bf16")
    assert (nan[0] & 0x7f80) == 0x7f80 and (nan[0] & 0x7f) != 0


def pin_f16_rounding(lib):
    """Hand-written fp16 RNE == numpy's float32 -> float16 conversion."""
    v = rounding_sweep()
    got = lib.round16(v, "f16")
    with np.errstate(over="ignore"):
        want = v.astype(np.float16).view(np.uint16)
    assert np.array_equal(got, want)
    nan = lib.round16(np.float32([np.nan]), "f16")
    assert (nan[0] & 0x7c00) == 0x7c00 and (nan[0] & 0x3ff) != 0


def pin_16bit_outputs(lib):
    """bf16/fp16 outputs are the binary32 outputs rounded by the library routines."""
    import torch
    x = np.concatenate([evenly_spaced(1 << 16), symmetry_angles(1 << 16)])
    for red in ("plain", "compensated"):
        s, c = lib.sincos(x, reduction=red)
        sb, cb = lib.sincos(x, reduction=red, out="bf16")
        sh, ch = lib.sincos(x, reduction=red, out="f16")
        to_bf = lambda a: torch.from_numpy(a.copy()).to(torch.bfloat16).view(torch.int16) \
            .numpy().view(np.uint16)
        assert np.array_equal(sb, to_bf(s)) and np.array_equal(cb, to_bf(c))
        assert np.array_equal(sh, s.astype(np.float16).view(np.uint16))
        assert np.array_equal(ch, c.astype(np.float16).view(np.uint16))


# ----------------------------------------------------------------------------
# Backward.
# ----------------------------------------------------------------------------

def pin_backward(lib, n: int = 4096):
    """gx against FP64: the analytic gs*cos(x) - gc*sin(x), central finite
    differences of L = gs*sin + gc*cos (h = 1e-3), and the one-rounding bound
    of the fused form on the same (s, c)."""
    rng = np.random.default_rng(16)
    x = rng.uniform(-50, 50, n).astype(np.float32)
    gs = rng.standard_normal(n).astype(np.float32)
    gc = rng.standard_normal(n).astype(np.float32)
    s, c = lib.sincos(x)
    gx = lib.backward(gs, gc, s, c).astype(np.float64)
    xd, gsd, gcd = x.astype(np.float64), gs.astype(np.float64), gc.astype(np.float64)
    scale = np.abs(gsd) + np.abs(gcd)
    analytic = gsd * np.cos(xd) - gcd * np.sin(xd)
    assert np.all(np.abs(gx - analytic) <= 1e-4 * scale)
    h = 1e-3
    L = lambda t: gsd * np.sin(t) + gcd * np.cos(t)
    fd = (L(xd + h) - L(xd - h)) / (2 * h)
    assert np.all(np.abs(gx - fd) <= 1e-4 * scale)
    # the fused form on the same binary32 (s, c): one rounding of gs*c plus gc*s's rounding
    exact = gsd * c.astype(np.float64) - gcd * s.astype(np.float64)
    tol = 2.0 ** -24 * (np.abs(exact) + np.abs(gcd * s.astype(np.float64))) + 1e-45
    assert np.all(np.abs(gx - exact) <= tol)
    # null upstream gradients stand for zeros
    g_only_s = lib.backward(gs, None, s, c).astype(np.float64)
    assert np.all(np.abs(g_only_s - gsd * c) <= 2.0 ** -24 * np.abs(gsd * c) + 1e-45)
    g_only_c = lib.backward(None, gc, s, c).astype(np.float64)
    assert np.all(np.abs(g_only_c + gcd * s) <= 2.0 ** -24 * np.abs(gcd * s) + 1e-45)
    assert np.all(lib.backward(None, None, s, c) == 0.0)


# ----------------------------------------------------------------------------
# Huygens field sum.
# ----------------------------------------------------------------------------

def huygens_case(m=48, n=300, seed=21, distance=400.0):
    rng = np.random.default_rng(seed)
    p = (rng.uniform(-60, 60, m).astype(np.float32), rng.uniform(-60, 60, m).astype(np.float32),
         np.full(m, distance, np.float32))
    q = (rng.uniform(-14, 14, n).astype(np.float32), rng.uniform(-14, 14, n).astype(np.float32),
         rng.uniform(-1, 1, n).astype(np.float32))
    a = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    return p, q, a, float(np.float32(2 * np.pi))


def pin_huygens_fp64(lib):
    """Against the FP64 sum of a_j exp(i k r)/r with libm: every point within
    the per-term bound sum_j |a_j|/r_ij (k r_ij 2^-22 + 1.5e-6) (binary32
    rounding of r and of k r, plus the method's error) plus the sequential
    binary32 summation bound n 2^-24 sum_j |a_j|/r_ij."""
    import oracle
    for red in ("compensated", "plain"):
        p, q, a, k = huygens_case()
        u = lib.huygens(p, q, a, k, red).astype(np.complex128)
        ref = oracle.huygens_fp64(p, q, a, k)
        P = np.stack([v.astype(np.float64) for v in p], 1)
        Q = np.stack([v.astype(np.float64) for v in q], 1)
        r = np.sqrt(((P[:, None, :] - Q[None, :, :]) ** 2).sum(2))
        t = np.abs(a.astype(np.complex128))[None, :] / r
        method = 1.5e-6 if red == "compensated" else 1.5e-6 + 2 * np.pi * (k * r / (2 * np.pi)) * 2.0 ** -23
        bound = (t * (k * r * 2.0 ** -22 + method)).sum(1) + q[0].size * 2.0 ** -24 * t.sum(1)
        assert np.all(np.abs(u - ref) <= bound), (red, np.max(np.abs(u - ref) / bound))


def pin_huygens_airy(lib):
    """Far field of a uniformly lit circular aperture (Fraunhofer, Fresnel
    number 0.01): |u|^2 / |u(0)|^2 follows (2 J1(v)/v)^2 with v = k a sin(t),
    the Airy pattern, to within 0.01 over the first three lobes."""
    from scipy.special import j1
    radius, spacing, z = 10.0, 0.25, 1.0e4
    g = np.arange(-radius, radius + spacing / 2, spacing)
    gx, gy = np.meshgrid(g, g)
    keep = gx * gx + gy * gy <= radius * radius
    q = (gx[keep].astype(np.float32), gy[keep].astype(np.float32),
         np.zeros(int(keep.sum()), np.float32))
    a = np.ones(q[0].size, np.complex64)
    ang = np.linspace(0.0, 0.15, 61)
    p = ((z * np.tan(ang)).astype(np.float32), np.zeros(ang.size, np.float32),
         np.full(ang.size, z, np.float32))
    k = float(np.float32(2 * np.pi))
    u = lib.huygens(p, q, a, k, "compensated").astype(np.complex128)
    inten = np.abs(u) ** 2 / np.abs(u[0]) ** 2
    v = k * radius * np.sin(ang)
    with np.errstate(invalid="ignore", divide="ignore"):
        airy = np.where(v == 0, 1.0, (2 * j1(v) / v) ** 2)
    assert np.max(np.abs(inten - airy)) < 0.01, np.max(np.abs(inten - airy))


def pin_huygens_edges(lib):
    """No sources: a zero field.  One source: a single term, a exp(i k r)/r,
    within the per-term bound of pin_huygens_fp64 (no summation error)."""
    p, q, a, k = huygens_case(m=7, n=1)
    z = lib.huygens(p, (q[0][:0], q[1][:0], q[2][:0]), a[:0], k)
    assert np.all(z == 0)
    u = lib.huygens(p, q, a, k, "compensated").astype(np.complex128)
    P = np.stack([v.astype(np.float64) for v in p], 1)
    Q = np.array([q[0][0], q[1][0], q[2][0]], np.float64)
    r = np.sqrt(((P - Q) ** 2).sum(1))
    ref = complex(a[0]) * np.exp(1j * float(k) * r) / r
    bound = abs(complex(a[0])) / r * (k * r * 2.0 ** -22 + 1.5e-6)
    assert np.all(np.abs(u - ref) <= bound)


# ----------------------------------------------------------------------------
# Threaded driver (the CPU-baseline timing and the all-inputs GPU comparison).
# ----------------------------------------------------------------------------

MT_SIZES = (0, 1, 2, 3, 17, 1000003, (1 << 20) + 5)
MT_THREADS = (1, 2, 3, 7, 16, 33, 600)     # 600 is above the driver's clamp of 512


def _mt_angles(n: int) -> np.ndarray:
    """Angles where the two reductions and the two coefficient sets all give
    different results: uniform on [-pi, pi), log-uniform magnitudes up to 1e5
    with random signs, and the special values."""
    rng = np.random.default_rng(31)
    third = n // 3
    mag = 10.0 ** rng.uniform(-3, 5, n - 2 * third)
    x = np.concatenate([rng.uniform(-math.pi, math.pi, third),
                        rng.uniform(-1e3, 1e3, third),
                        mag * np.where(rng.random(mag.size) < 0.5, -1.0, 1.0)])
    sp = np.float32([np.nan, np.inf, -np.inf, 0.0, -0.0, 2.0 ** 26, 1e-40, 0.5])
    k = min(sp.size, n)
    x = x.astype(np.float32)
    x[:k] = sp[:k]
    return x


def pin_threaded_driver(lib, sizes=MT_SIZES, threads=MT_THREADS):
    """The threaded driver gives, for every size and thread count (ragged
    splits, threads without work, the clamp), exactly the bits of the
    single-threaded forward for each reduction and coefficient set, writes
    nothing outside [0, n), and stays within the method's error of FP64 at the
    reduced angle."""
    guard = 8
    sentinel = np.uint32(0x7FC0DEAD)          # a NaN no result of the method carries
    variants = [(r, cf) for r in ("plain", "compensated") for cf in ("normalized", "dagger")]
    for n in sizes:
        x = _mt_angles(n)
        for red, cf in variants:
            want_s, want_c = lib.sincos(x, reduction=red, coef=cf)
            if n and red == "plain" and cf == "normalized":
                fin = np.isfinite(x) & (np.abs(x) <= 4.0)
                if fin.any():
                    assert core_error(x[fin], want_s[fin], want_c[fin]).max() <= CORE_BOUND
            for t in threads:
                sb = np.full(n + 2 * guard, sentinel, np.uint32).view(np.float32)
                cb = np.full(n + 2 * guard, sentinel, np.uint32).view(np.float32)
                s, c = sb[guard:guard + n], cb[guard:guard + n]
                used = lib.sincos_mt(x, s, c, reduction=red, coef=cf, threads=t)
                assert 0 <= used <= min(t, 512), (n, t, used)
                what = f"n={n} threads={t} {red}/{cf}"
                for buf in (sb, cb):
                    assert np.all(buf[:guard].view(np.uint32) == sentinel), what + ": wrote before"
                    assert np.all(buf[guard + n:].view(np.uint32) == sentinel), what + ": wrote after"
                assert np.array_equal(s.view(np.uint32), want_s.view(np.uint32)), what + ": s"
                assert np.array_equal(c.view(np.uint32), want_c.view(np.uint32)), what + ": c"


ALL_PINS = [
    pin_e1_normalized, pin_e2_dagger, pin_drift_correction, pin_bruteforce,
    pin_bruteforce_small_angles, pin_symmetry,
    pin_periodicity, pin_exact_at_whole_turns, pin_quarter_turns, pin_ties_to_even,
    pin_special_values, pin_plain_reduction_bound, pin_compensated, pin_bf16_rounding,
    pin_f16_rounding, pin_16bit_outputs, pin_backward, pin_huygens_fp64, pin_huygens_airy,
    pin_huygens_edges, pin_threaded_driver,
]
