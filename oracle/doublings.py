"""The method with n angle doublings instead of two: a CPU study model.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: nothing on the product
path imports it.  It maps the trade-off the paper points at in its
Methodology section: evaluate shorter or longer power series of the pair at
2 pi q1 / 2^n, then double the angle n times with Eq. (1), correcting the
amplitude drift with the pair before the last doubling (Fig. 1's form of the
correction).  The paper's design is n = 2 with sine and cosine series of
degree 7 and 6 (series index d = 3 below).

Binary32 arithmetic is emulated in float64 numpy so that any (n, d) can be
studied without generating C:

* a product of two binary32 values is exact in float64 and is rounded once;
* a fused multiply-add forms that exact product, adds the addend with an
  error-free two-sum, rounds the float64 sum to odd and then to binary32,
  which is the correctly rounded result (rounding to odd in a format with
  at least two more bits makes the second rounding innocuous; Boldo and
  Melquiond, "Emulation of FMA and correctly rounded sums: proved
  algorithms using rounding to odd", IEEE TC 2008).

With the paper's printed coefficients, n = 2 and d = 3 this reproduces the
C oracle bit for bit (``tests/test_doubling_study.py``), which pins the
emulation.  The coefficients for other (n, d) are least-squares fits of
sin(2 pi q / 2^n) and cos(2 pi q / 2^n) - 1 on q in [-1/2, 1/2], the paper's
first method (small normalisation error), rounded to binary32.

Errors are measured on the reduced angle: against the FP64 sine and cosine of
2 pi q1 for binary32 q1 in [-1/2, 1/2], so the reduction's own rounding (the
same for every n and d) is left out.

Run ``python -m oracle.doublings`` to rewrite ``tests/golden/doubling_study.txt``.
"""
from __future__ import annotations

import os
import sys

import numpy as np

K_SCALE = np.float32(1.0 / (2.0 * 3.1415926536))   # Sec. Methodology: scale by 1/2pi

# Printed normalized set (Sec. Methodology, first method): sin = q (ss1 + ss2 q^2 + ...),
# cos = 1 + cc1 q^2 + ...
PAPER_SS = (1.5707963235, -0.645963615, 0.0796819754, -0.0046075748)
PAPER_CC = (-1.2336977925, 0.2536086171, -0.0204391631)


# -- binary32 arithmetic in float64 --------------------------------------------

def f32(a) -> np.ndarray:
    """Round float64 values to binary32 (nearest even) and widen back."""
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def mul32(a, b) -> np.ndarray:
    """Correctly rounded binary32 product (the float64 product is exact)."""
    return f32(np.asarray(a, np.float64) * b)


def fma32(a, b, c) -> np.ndarray:
    """Correctly rounded binary32 a*b + c (exact product, two-sum, round to odd)."""
    a = np.asarray(a, np.float64)
    p = a * b
    c = np.broadcast_to(np.asarray(c, np.float64), p.shape)
    s = p + c
    bb = s - p
    err = (p - (s - bb)) + (c - bb)
    bits = s.view(np.uint64)
    needs_odd = (err != 0) & ((bits & np.uint64(1)) == 0)
    toward = np.where(err > 0, np.inf, -np.inf)
    s = np.where(needs_odd, np.nextafter(s, toward), s)
    return f32(s)


def reduce_plain(x) -> np.ndarray:
    """q1 = fl(x K) - rint(fl(x K)) (Sec. Methodology); the subtraction is exact."""
    x1 = mul32(f32(x), float(K_SCALE))
    return x1 - np.rint(x1)


# -- the method for any n and d -----------------------------------------------------

def fit_series(n: int, d: int, points: int = 40001):
    """Least-squares series at the angle 2 pi q / 2^n, q in [-1/2, 1/2].

    Sine: q (ss[0] + ss[1] q^2 + ... + ss[d] q^{2d}), degree 2d + 1.
    Cosine: 1 + cc[0] q^2 + ... + cc[d-1] q^{2d}, degree 2d.
    Both rounded to binary32."""
    q = np.linspace(-0.5, 0.5, points)
    phi = 2.0 * np.pi * q / 2.0 ** n
    a_sin = np.stack([q ** (2 * k + 1) for k in range(d + 1)], axis=1)
    a_cos = np.stack([q ** (2 * k) for k in range(1, d + 1)], axis=1)
    ss = np.linalg.lstsq(a_sin, np.sin(phi), rcond=None)[0]
    cc = np.linalg.lstsq(a_cos, np.cos(phi) - 1.0, rcond=None)[0]
    return f32(ss), f32(cc)


def series_pair(q1, ss, cc):
    """The pair at the scaled-down angle, by Horner's rule in q2 = q1^2."""
    q1 = np.asarray(q1, np.float64)
    q2 = mul32(q1, q1)
    hs = np.full_like(q1, ss[-1])
    for k in range(len(ss) - 2, -1, -1):
        hs = fma32(q2, hs, ss[k])
    s = mul32(q1, hs)
    if len(cc) == 0:
        return s, np.ones_like(q1)
    hc = np.full_like(q1, cc[-1])
    for k in range(len(cc) - 2, -1, -1):
        hc = fma32(q2, hc, cc[k])
    c = fma32(q2, hc, 1.0)
    return s, c


def double(s, c):
    """One application of Eq. (1): (c^2 - s^2, 2 s c) in the oracle's order."""
    return mul32(2.0, mul32(s, c)), fma32(-s, s, mul32(c, c))


def drift_factor(s, c):
    """Fig. 1's amplitude correction from the pair before the last doubling:
    2 - s^2 - c^2 (1 - alpha/2 to first order, alpha the doubled pair's drift)."""
    return fma32(-s, s, fma32(-c, c, 2.0))


def pair_n(q1, n: int, ss, cc, correct: bool = True):
    """Series at 2 pi q1 / 2^n, then n doublings; the drift correction (when
    n >= 1 and ``correct``) uses the pair before the last doubling."""
    s, c = series_pair(q1, ss, cc)
    fix = None
    for i in range(n):
        if correct and i == n - 1:
            fix = drift_factor(s, c)
        s, c = double(s, c)
    if fix is not None:
        s, c = mul32(s, fix), mul32(c, fix)
    return s, c


def op_count(n: int, d: int) -> int:
    """Binary32 operations per pair: reduction 3 (multiply, rint, subtract),
    q^2 1, sine d fmas + 1 multiply, cosine d fmas, 4 per doubling, and 4 for
    the correction (2 fmas, 2 multiplies) when n >= 1.  23 at the paper's
    n = 2, d = 3."""
    return 3 + 1 + (d + 1) + d + 4 * n + (4 if n >= 1 else 0)


# -- the study ------------------------------------------------------------------------

def sample_q1(random: int = 1 << 21, grid: int = 1 << 20, seed: int = 0) -> np.ndarray:
    """Binary32 reduced angles: uniform draws plus an even grid on [-1/2, 1/2]."""
    rng = np.random.default_rng(seed)
    return f32(np.concatenate([rng.uniform(-0.5, 0.5, random), np.linspace(-0.5, 0.5, grid)]))


def error_stats(q1, s, c):
    """(max, RMS) Euclidean error against FP64 at 2 pi q1, and max |1 - amplitude|."""
    ref_s, ref_c = np.sin(2.0 * np.pi * q1), np.cos(2.0 * np.pi * q1)
    e = np.hypot(s - ref_s, c - ref_c)
    amp = np.abs(1.0 - np.hypot(s, c))
    return float(e.max()), float(np.sqrt(np.mean(e * e))), float(amp.max())


def study_row(n: int, d: int, q1=None) -> dict:
    q1 = sample_q1() if q1 is None else q1
    ss, cc = fit_series(n, d)
    s, c = pair_n(q1, n, ss, cc)
    mx, rms, amp = error_stats(q1, s, c)
    return {"n": n, "d": d, "ops": op_count(n, d), "max": mx, "rms": rms, "amp": amp}


GOLDEN_ROWS = [(n, d) for n in range(0, 5) for d in range(2, 9)]


def write_golden(path: str) -> None:
    q1 = sample_q1()
    lines = ["# n-doubling trade-off of the method (Sec. Methodology, Eq. (1), Fig. 1's",
             "# correction): least-squares series of index d (sine degree 2d+1, cosine 2d)",
             "# at 2 pi q / 2^n, n doublings.  Errors at the reduced angle over",
             "# sample_q1() (2^21 uniform + 2^20 grid binary32 q1 in [-1/2, 1/2]).",
             "# Written by `python -m oracle.doublings`.",
             "# n d ops max_err rms_err max_amp"]
    for n, d in GOLDEN_ROWS:
        r = study_row(n, d, q1)
        lines.append(f"{n} {d} {r['ops']} {r['max']:.4e} {r['rms']:.4e} {r['amp']:.4e}")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def read_golden(path: str) -> dict:
    rows = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, d, ops, mx, rms, amp = line.split()
            rows[(int(n), int(d))] = {"ops": int(ops), "max": float(mx), "rms": float(rms),
                                      "amp": float(amp)}
    return rows


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "..", "tests", "golden",
                                                                "doubling_study.txt")
    write_golden(out)
    print(open(out).read())
