"""CPU oracle for the branch-free sine-cosine pair method (Mendenhall, cs/0406049).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or runs it.

The arithmetic lives in ``sincos_oracle.c`` (plain binary32 C with explicit
``fmaf``, compiled with ``-ffp-contract=off``); this module only compiles it
with gcc and marshals numpy arrays through ctypes.  ``fp64_reference`` is the
FP64 sine/cosine used to *state* errors; it is never a parity target.

Parity status: every exported function is pinned by the CPU test suite
(``tests/test_oracle_pins.py``, ``tests/test_oracle_mutations.py``); none is
unpinned.  ``doublings.py`` is a study model of the method with n doublings
(no GPU counterpart), pinned bit for bit to this oracle at the paper's n = 2
(``tests/test_doubling_study.py``).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "sincos_oracle.c")
_LIB_NAME = "liboracle_sincos.so"

REDUCTIONS = {"plain": 0, "compensated": 1}
COEFS = {"normalized": 0, "dagger": 1}
GCC_FLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

_lock = threading.Lock()
_default = None


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source into a shared object (IEEE binary32, no contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *GCC_FLAGS, "-o", tmp, src, "-lm", "-lpthread"], check=True)
    os.replace(tmp, out)
    return out


def lib_path() -> str:
    return os.path.join(_HERE, _LIB_NAME)


def build(force: bool = False) -> str:
    """Build ``liboracle_sincos.so`` next to its source when missing or stale.

    A tag file next to the library holds the hash of the source it came from."""
    out = lib_path()
    tag_file = out + ".srctag"
    with open(SOURCE, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    if not force and os.path.exists(out) and os.path.exists(tag_file):
        with open(tag_file) as f:
            if f.read().strip() == tag:
                return out
    compile_source(SOURCE, out)
    with open(tag_file, "w") as f:
        f.write(tag)
    return out


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32).ravel()


class OracleLib:
    """ctypes view of one compiled oracle shared object."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        f32p = ctypes.POINTER(ctypes.c_float)
        u16p = ctypes.POINTER(ctypes.c_uint16)
        i64, cint = ctypes.c_int64, ctypes.c_int
        lib.oracle_sincos_f32.argtypes = [f32p, f32p, f32p, i64, cint, cint]
        lib.oracle_sincos_f32.restype = None
        lib.oracle_sincos_16.argtypes = [f32p, u16p, u16p, i64, cint, cint, cint]
        lib.oracle_sincos_16.restype = None
        lib.oracle_sincos_backward.argtypes = [f32p, f32p, f32p, f32p, f32p, i64]
        lib.oracle_sincos_backward.restype = None
        lib.oracle_sincos_f32_mt.argtypes = [f32p, f32p, f32p, i64, cint, cint, cint]
        lib.oracle_sincos_f32_mt.restype = cint
        lib.oracle_round_16.argtypes = [f32p, u16p, i64, cint]
        lib.oracle_round_16.restype = None
        lib.oracle_huygens.argtypes = [f32p, f32p, f32p, i64, f32p, f32p, f32p, f32p, f32p, i64,
                                       ctypes.c_float, cint, f32p]
        lib.oracle_huygens.restype = None
        self.path = path
        self._lib = lib

    def sincos(self, x, reduction: str = "plain", coef: str = "normalized", out: str = "f32"):
        """(s, c) for every binary32 angle of ``x``: Section "Methodology", Fig. 1.

        ``out`` is "f32", or "bf16" / "f16" for the binary32 result rounded to
        nearest-even and returned as raw uint16 bit patterns."""
        x = _f32(x)
        n = x.size
        red, cf = REDUCTIONS[reduction], COEFS[coef]
        if out == "f32":
            s = np.empty(n, np.float32)
            c = np.empty(n, np.float32)
            self._lib.oracle_sincos_f32(_ptr(x, ctypes.c_float), _ptr(s, ctypes.c_float),
                                        _ptr(c, ctypes.c_float), n, red, cf)
            return s, c
        kind = {"bf16": 1, "f16": 2}[out]
        s = np.empty(n, np.uint16)
        c = np.empty(n, np.uint16)
        self._lib.oracle_sincos_16(_ptr(x, ctypes.c_float), _ptr(s, ctypes.c_uint16),
                                   _ptr(c, ctypes.c_uint16), n, red, cf, kind)
        return s, c

    def sincos_mt(self, x, s, c, reduction: str = "plain", coef: str = "normalized",
                  threads: int = 1) -> int:
        """Threaded binary32 forward into caller arrays: ``oracle_sincos_f32`` on
        contiguous sub-ranges, one per thread, so the results are those of
        ``sincos``.  Used for the CPU timing and the exhaustive GPU comparison.
        Returns the number of threads used."""
        for a in (x, s, c):
            assert a.dtype == np.float32 and a.flags.c_contiguous
        return self._lib.oracle_sincos_f32_mt(
            _ptr(x, ctypes.c_float), _ptr(s, ctypes.c_float), _ptr(c, ctypes.c_float), x.size,
            REDUCTIONS[reduction], COEFS[coef], int(threads))

    def backward(self, gs, gc, s, c):
        """gx = gs*c - gc*s on the forward's outputs; ``None`` for an all-zero gradient."""
        s, c = _f32(s), _f32(c)
        gs_a = None if gs is None else _f32(gs)
        gc_a = None if gc is None else _f32(gc)
        gx = np.empty(s.size, np.float32)
        self._lib.oracle_sincos_backward(
            None if gs_a is None else _ptr(gs_a, ctypes.c_float),
            None if gc_a is None else _ptr(gc_a, ctypes.c_float),
            _ptr(s, ctypes.c_float), _ptr(c, ctypes.c_float), _ptr(gx, ctypes.c_float), s.size)
        return gx

    def huygens(self, p, q, a, k: float, reduction: str = "compensated") -> np.ndarray:
        """Field sum at points p (3 x m) of sources q (3 x n) with complex
        amplitudes a (n, complex): sum_j a_j exp(i k r_ij) / r_ij, every
        phase factor from the method, summed in source order in binary32.
        Returns complex64 (m,)."""
        px, py, pz = (_f32(v) for v in p)
        qx, qy, qz = (_f32(v) for v in q)
        a = np.asarray(a, np.complex64).ravel()
        ar, ai = _f32(a.real), _f32(a.imag)
        m, n = px.size, qx.size
        u = np.zeros(2 * m, np.float32)
        f = lambda v: _ptr(v, ctypes.c_float)
        self._lib.oracle_huygens(f(px), f(py), f(pz), m, f(qx), f(qy), f(qz), f(ar), f(ai), n,
                                 float(np.float32(k)), REDUCTIONS[reduction], f(u))
        return u.view(np.complex64)

    def round16(self, v, kind: str) -> np.ndarray:
        """Binary32 -> bf16 or fp16 bit patterns, round to nearest even."""
        v = _f32(v)
        out = np.empty(v.size, np.uint16)
        self._lib.oracle_round_16(_ptr(v, ctypes.c_float), _ptr(out, ctypes.c_uint16), v.size,
                                  {"bf16": 1, "f16": 2}[kind])
        return out


def default() -> OracleLib:
    global _default
    with _lock:
        if _default is None:
            _default = OracleLib(build())
        return _default


def sincos(x, reduction: str = "plain", coef: str = "normalized", out: str = "f32"):
    return default().sincos(x, reduction, coef, out)


def sincos_mt(x, s, c, reduction: str = "plain", coef: str = "normalized", threads: int = 1):
    return default().sincos_mt(x, s, c, reduction, coef, threads)


def backward(gs, gc, s, c):
    return default().backward(gs, gc, s, c)


def to_bf16_bits(v) -> np.ndarray:
    return default().round16(v, "bf16")


def to_f16_bits(v) -> np.ndarray:
    return default().round16(v, "f16")


def huygens(p, q, a, k: float, reduction: str = "compensated"):
    return default().huygens(p, q, a, k, reduction)


def huygens_fp64(p, q, a, k: float) -> np.ndarray:
    """The same field sum in FP64 with libm sin/cos (error statement only)."""
    P = np.stack([np.asarray(v, np.float32).astype(np.float64) for v in p], axis=1)
    Q = np.stack([np.asarray(v, np.float32).astype(np.float64) for v in q], axis=1)
    a = np.asarray(a, np.complex64).astype(np.complex128)
    out = np.empty(P.shape[0], np.complex128)
    kd = float(np.float32(k))
    for i0 in range(0, P.shape[0], 256):
        d = P[i0:i0 + 256, None, :] - Q[None, :, :]
        r = np.sqrt((d * d).sum(axis=2))
        out[i0:i0 + 256] = (a[None, :] * np.exp(1j * kd * r) / r).sum(axis=1)
    return out


def fp64_reference(x):
    """FP64 sin and cos of the binary32 angles promoted to double (error statement only)."""
    xd = np.asarray(x, dtype=np.float32).astype(np.float64)
    return np.sin(xd), np.cos(xd)


def error_stats(x, s, c) -> dict:
    """Errors of a binary32 pair against FP64, in the paper's measures and in ulp.

    euclid  = sqrt((c - cos x)^2 + (s - sin x)^2)  (the paper's error measure)
    amp     = |1 - sqrt(c^2 + s^2)|                  (the paper's amplitude error)
    max_abs = max(|s - sin x|, |c - cos x|); ``max_abs_ulp1`` is it in units of
    2^-23 (one ulp of 1.0); ``max_ulp_rel_ge_2m4`` is |y - ref| / ulp(ref) over
    results with |ref| >= 2^-4 (the method is absolutely, not relatively,
    accurate, so a per-result ulp near a zero of sin or cos says nothing)."""
    x = np.asarray(x, np.float32)
    s64 = np.asarray(s, np.float64)
    c64 = np.asarray(c, np.float64)
    rs, rc = fp64_reference(x)
    finite = np.isfinite(rs) & np.isfinite(s64) & np.isfinite(c64)
    ds = np.abs(s64 - rs)[finite]
    dc = np.abs(c64 - rc)[finite]
    eu = np.sqrt(ds * ds + dc * dc)
    amp = np.abs(1.0 - np.sqrt(s64[finite] ** 2 + c64[finite] ** 2))
    ref = np.concatenate([rs[finite], rc[finite]])
    got = np.concatenate([s64[finite], c64[finite]])
    big = np.abs(ref) >= 2.0 ** -4
    ulp = np.spacing(np.abs(ref[big]).astype(np.float32)).astype(np.float64)
    rel = np.abs(got[big] - ref[big]) / ulp if big.any() else np.zeros(1)
    max_abs = float(max(ds.max(initial=0.0), dc.max(initial=0.0)))
    return {
        "n": int(finite.sum()),
        "rms_euclid": float(np.sqrt(np.mean(eu * eu))) if eu.size else 0.0,
        "max_euclid": float(eu.max(initial=0.0)),
        "max_amp": float(amp.max(initial=0.0)),
        "max_abs": max_abs,
        "max_abs_ulp1": max_abs / 2.0 ** -23,
        "max_ulp_rel_ge_2m4": float(rel.max(initial=0.0)),
    }
