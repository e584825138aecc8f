"""Helpers shared by the GPU parity tests (marshalling and comparisons only)."""
from __future__ import annotations

import numpy as np
import torch

# The stated parity tolerance: 2 ulp of 1.0 (2.4e-7 absolute) against the oracle.
PARITY_ABS_TOL = 2.4e-7


def as_np(t: torch.Tensor) -> np.ndarray:
    t = t.detach().cpu()
    if t.dtype in (torch.bfloat16, torch.float16):
        return t.view(torch.int16).numpy().view(np.uint16)
    return t.numpy()


def assert_f32_parity(got: np.ndarray, want: np.ndarray, what: str = ""):
    """GPU binary32 results against the oracle's: NaN where the oracle has
    NaN, otherwise within the stated tolerance, and bit-identical."""
    got = np.asarray(got, np.float32)
    want = np.asarray(want, np.float32)
    assert got.shape == want.shape, what
    nan_w = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan_w), f"{what}: NaN positions differ"
    g, w = got[~nan_w], want[~nan_w]
    if g.size:
        diff = np.abs(g.astype(np.float64) - w.astype(np.float64))
        assert diff.max() <= PARITY_ABS_TOL, f"{what}: max |gpu - oracle| = {diff.max():.3g}"
    neq = np.flatnonzero(g.view(np.uint32) != w.view(np.uint32))
    assert neq.size == 0, (f"{what}: {neq.size} results differ in their bits "
                           f"(first at {neq[:5]}: {g[neq[:5]]} vs {w[neq[:5]]})")


def _isnan16(a: np.ndarray, bf16: bool) -> np.ndarray:
    if bf16:
        return ((a & 0x7f80) == 0x7f80) & ((a & 0x007f) != 0)
    return ((a & 0x7c00) == 0x7c00) & ((a & 0x03ff) != 0)


def assert_16_parity(got: np.ndarray, want: np.ndarray, bf16: bool, what: str = ""):
    """16-bit outputs: NaN in the same places, every other bit pattern equal."""
    got = np.asarray(got, np.uint16)
    want = np.asarray(want, np.uint16)
    assert got.shape == want.shape, what
    nan_w = _isnan16(want, bf16)
    assert np.array_equal(_isnan16(got, bf16), nan_w), f"{what}: NaN positions differ"
    neq = np.flatnonzero(got[~nan_w] != want[~nan_w])
    assert neq.size == 0, f"{what}: {neq.size} 16-bit results differ"


def special_angles() -> np.ndarray:
    """Edge inputs: zeros, subnormals, NaN, infinities, ties, huge magnitudes."""
    v = [0.0, -0.0, 1e-45, -1e-45, 1e-40, -1e-40, 1.1754942e-38, 2.0 ** -126,
         np.nan, np.inf, -np.inf, 3.4028235e38, -3.4028235e38, 2.0 ** 23, 2.0 ** 26,
         5.27e7, -5.27e7, 1e10, 1e-10, 0.5, 1.0, np.pi, -np.pi, np.pi / 2, 2 * np.pi,
         1e5, -1e5, 99999.99, 1000.0, -1000.0]
    return np.array(v, dtype=np.float32)


def mixed_angles(n: int, seed: int) -> np.ndarray:
    """Random angles over many magnitudes plus the edge inputs, shuffled."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-np.pi, np.pi, n // 2),
             (10.0 ** rng.uniform(-8, 8, n - n // 2)) * np.where(rng.random(n - n // 2) < 0.5, -1, 1)]
    x = np.concatenate(parts).astype(np.float32)
    sp = special_angles()
    k = min(sp.size, n)
    x[rng.choice(n, k, replace=False)] = sp[:k]
    return x


class forced_plan:
    """Use one launch plan for every size class of (op, dtype) inside a with
    block, restoring the previous plans afterwards."""

    def __init__(self, op: str, dtype: str, plan):
        self.op, self.dtype, self.plan = op, dtype, tuple(plan)

    def __enter__(self):
        from paper_cs_0406049_gb300 import api
        self.saved = [(b, api.sincos_plan_get(self.op, self.dtype, 1 << b)) for b in range(0, 41)]
        for b, _ in self.saved:
            api.sincos_plan_set(self.op, self.dtype, 1 << b, *self.plan)
        return self

    def __exit__(self, *exc):
        from paper_cs_0406049_gb300 import api
        for b, p in self.saved:
            api.sincos_plan_set(self.op, self.dtype, 1 << b, p["block"], p["unroll"],
                                p["ctas_per_sm"], p["vec_bytes"])


def pageable_access(device: int = 0) -> bool:
    """Whether the device reads pageable host memory through the host's page
    tables (cudaDevAttrPageableMemoryAccess), asked of the CUDA runtime."""
    import ctypes
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
        except OSError:
            continue
        v = ctypes.c_int(0)
        if rt.cudaDeviceGetAttribute(ctypes.byref(v), ctypes.c_int(88), ctypes.c_int(device)) == 0:
            return v.value == 1
    return False


class host_route:
    """sincos_host_route_set inside a with block, back to "auto" after it."""

    def __init__(self, policy: str):
        self.policy = policy

    def __enter__(self):
        from paper_cs_0406049_gb300 import api
        api.sincos_host_route_set(self.policy)
        return self

    def __exit__(self, *exc):
        from paper_cs_0406049_gb300 import api
        api.sincos_host_route_set("auto")
