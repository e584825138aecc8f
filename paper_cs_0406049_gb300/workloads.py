"""Seeded synthetic inputs for the sine-cosine pair path.

This module holds no arithmetic of the method: it only draws angles, segment
lengths and upstream gradients from ``numpy.random.default_rng(seed)`` (PCG64).
Both the CUDA path (tests, benchmark) and the CPU oracle are fed from here.

Every workload is drawn in float64 and rounded once to float32.  Draws are made
in chunks of ``CHUNK`` values; for a single stream of uniforms this gives the
same values as one large draw, and it bounds host memory at the 2^28 size.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CHUNK = 1 << 22


def _uniform(rng: np.random.Generator, n: int, lo: float, hi: float) -> np.ndarray:
    out = np.empty(n, np.float32)
    for i in range(0, n, CHUNK):
        m = min(CHUNK, n - i)
        out[i:i + m] = rng.uniform(lo, hi, m)
    return out


def angles_uniform(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n float32 angles, uniform in [lo, hi) drawn in float64, in random order."""
    return _uniform(np.random.default_rng(seed), n, lo, hi)


def angles_log_magnitude(n: int, lo_exp: float, hi_exp: float, seed: int) -> np.ndarray:
    """n float32 angles with |x| = 10**U[lo_exp, hi_exp] and a random sign.

    All n magnitude exponents are drawn first, then n sign uniforms."""
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(lo_exp, hi_exp, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return (mag * sign).astype(np.float32)


def batch_lengths(count: int, max_log2: int, rng: np.random.Generator) -> np.ndarray:
    """Segment lengths clamp(round(2**(max_log2*U)), 1, 2**max_log2), int64."""
    u = rng.random(count)
    lens = np.rint(np.exp2(max_log2 * u))
    return np.clip(lens, 1, 2 ** max_log2).astype(np.int64)


@dataclass
class Batch:
    """A batch of arrays packed back to back in one float32 buffer.

    Segment i is ``angles[offsets[i] : offsets[i] + lens[i]]``; most segments
    therefore start at an address that is not 16-byte aligned."""
    angles: np.ndarray
    lens: np.ndarray
    offsets: np.ndarray = field(init=False)

    def __post_init__(self):
        self.offsets = np.concatenate([[0], np.cumsum(self.lens)[:-1]]).astype(np.int64)

    @property
    def count(self) -> int:
        return int(self.lens.size)

    @property
    def total(self) -> int:
        return int(self.lens.sum())


def batch(count: int, max_log2: int, lo: float, hi: float, seed: int) -> Batch:
    """Lengths first, then all angles uniform in [lo, hi), from one generator."""
    rng = np.random.default_rng(seed)
    lens = batch_lengths(count, max_log2, rng)
    angles = _uniform(rng, int(lens.sum()), lo, hi)
    return Batch(angles, lens)


@dataclass
class Differentiation:
    x: np.ndarray
    gs: np.ndarray
    gc: np.ndarray


def differentiation(n: int, lo: float, hi: float, seed: int) -> Differentiation:
    """Angles uniform in [lo, hi), then upstream gradients gs and gc ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    x = _uniform(rng, n, lo, hi)
    gs = rng.standard_normal(n, dtype=np.float32)
    gc = rng.standard_normal(n, dtype=np.float32)
    return Differentiation(x, gs, gc)


@dataclass
class Diffraction:
    """Observation points p (3 arrays of m), sources q (3 arrays of n), complex
    amplitudes a (n,) and the wavenumber k, in units of the wavelength."""
    p: tuple
    q: tuple
    a: np.ndarray
    k: float


def diffraction(grid: int = 512, half_width: float = 60.0, distance: float = 400.0,
                sources: int = 4096, radius: float = 20.0, seed: int = 5) -> Diffraction:
    """A grid x grid observation plane at z = distance spanning
    [-half_width, half_width]^2; `sources` points uniform in a disc of the
    given radius at z = 0 (pairs drawn uniform in the enclosing square, in
    batches, keeping those inside the disc in draw order); then complex
    Gaussian amplitudes.  Lengths in wavelengths, so k = 2 pi."""
    rng = np.random.default_rng(seed)
    g = np.linspace(-half_width, half_width, grid)
    gx, gy = np.meshgrid(g, g, indexing="xy")
    p = (gx.ravel().astype(np.float32), gy.ravel().astype(np.float32),
         np.full(grid * grid, distance, np.float32))
    xs, ys = [], []
    kept = 0
    while kept < sources:
        cand = rng.uniform(-radius, radius, (2 * sources, 2))
        inside = cand[(cand * cand).sum(axis=1) <= radius * radius]
        xs.append(inside[:, 0])
        ys.append(inside[:, 1])
        kept += inside.shape[0]
    q = (np.concatenate(xs)[:sources].astype(np.float32),
         np.concatenate(ys)[:sources].astype(np.float32), np.zeros(sources, np.float32))
    a = (rng.standard_normal(sources) + 1j * rng.standard_normal(sources)).astype(np.complex64)
    return Diffraction(p, q, a, float(np.float32(2.0 * np.pi)))


# -- the five workloads the path is measured and checked on --------------------

PLAIN_N = 1 << 20            # uniform in [-pi, pi), seed 0
BANDWIDTH_N = 1 << 28        # uniform in [-1000, 1000), seed 1
PRECISION_N = 1 << 26        # |x| log-uniform in [1e-3, 1e5], random sign, seed 2
BATCH_COUNT = 4096           # lengths log-uniform in [1, 2^20], angles in [-100, 100), seed 3
DIFF_N = 1 << 26             # uniform in [-50, 50), seed 4; gs, gc ~ N(0, 1)

WORKLOADS = {
    "plain_2p20": "2^20 angles U[-pi, pi), seed 0, f32 out, plain reduction",
    "bandwidth_2p28": "2^28 angles U[-1000, 1000), seed 1, f32 out, plain reduction",
    "precision_2p26": "2^26 angles |x|=10^U[-3,5] random sign, seed 2; plain/compensated f32, "
                      "bf16/f16",
    "batching_4096": "4096 arrays, len=clamp(round(2^(20U)),1,2^20), U[-100,100), seed 3",
    "differentiation_2p26": "2^26 angles U[-50, 50), seed 4; gs, gc ~ N(0,1) f32",
    "diffraction_512x512_4096": "512x512 observation grid at z=400 over [-60,60]^2, 4096 "
                                "sources uniform in a radius-20 disc, Gaussian amplitudes, "
                                "k=2pi, seed 5",
}


def plain(n: int = PLAIN_N) -> np.ndarray:
    return angles_uniform(n, -math.pi, math.pi, 0)


def bandwidth(n: int = BANDWIDTH_N) -> np.ndarray:
    return angles_uniform(n, -1000.0, 1000.0, 1)


def precision(n: int = PRECISION_N) -> np.ndarray:
    return angles_log_magnitude(n, -3.0, 5.0, 2)


def batching(count: int = BATCH_COUNT, max_log2: int = 20) -> Batch:
    return batch(count, max_log2, -100.0, 100.0, 3)


def differentiation_inputs(n: int = DIFF_N) -> Differentiation:
    return differentiation(n, -50.0, 50.0, 4)
