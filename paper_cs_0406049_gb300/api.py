"""Python binding of the C ABI, with the same names, plus the torch front end.

The functions here only marshal arguments (device pointers, sizes, the
current CUDA stream) into ``libsincos_gb300.so``; every step of the method
runs in its CUDA kernels.  PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check

_DTYPES = {torch.float32: _lib.F32, torch.bfloat16: _lib.BF16, torch.float16: _lib.F16}
_DTYPE_NAMES = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
_REDUCTIONS = {"plain": _lib.RED_PLAIN, "compensated": _lib.RED_COMPENSATED}
_COEFS = {"normalized": _lib.COEF_NORMALIZED, "dagger": _lib.COEF_DAGGER}
_OPS = {"pairs": _lib.OP_PAIRS, "backward": _lib.OP_BACKWARD, "batched": _lib.OP_BATCHED,
        "expi": _lib.OP_EXPI, "huygens": _lib.OP_HUYGENS}


_loaded = None


def lib():
    global _loaded
    if _loaded is None:
        _loaded = _lib.load()
    return _loaded


def _torch_dtype(d) -> torch.dtype:
    return _DTYPE_NAMES[d] if isinstance(d, str) else d


# The raw handle of a device's current stream.  PyTorch's own accessor for it
# avoids building a Stream object on every call (2 us of host time per call,
# as much as the rest of a small launch); the public route is the fallback.
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream, device) -> int:
    if stream is None:
        index = device.index if isinstance(device, torch.device) else device
        if _raw_stream is not None and index is not None:
            return _raw_stream(index)
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class _on_device:
    """Make `device` current for a library call (the C ABI acts on the
    calling thread's current device); switches only when it is not current
    already, which costs far less than torch.cuda.device's full context."""

    __slots__ = ("index", "prev")

    def __init__(self, device):
        self.index = device.index if isinstance(device, torch.device) else device

    def __enter__(self):
        self.prev = torch.cuda.current_device()
        if self.index is not None and self.index != self.prev:
            torch.cuda.set_device(self.index)
        return self

    def __exit__(self, *exc):
        if self.index is not None and self.index != self.prev:
            torch.cuda.set_device(self.prev)


def _dev(t: torch.Tensor, name: str, dtype=None) -> int:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def _host(t: torch.Tensor, name: str, dtype=None) -> int:
    if t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


# -----------------------------------------------------------------------------
# C ABI, one function each
# -----------------------------------------------------------------------------

def sincos_pairs(x: torch.Tensor, s: torch.Tensor, c: torch.Tensor, stream=None) -> None:
    """s, c = sin(x), cos(x): binary32, plain reduction, normalized set."""
    n = x.numel()
    if s.numel() != n or c.numel() != n:
        raise ValueError("x, s and c must have the same number of elements")
    with _on_device(x.device):
        check(lib().sincos_pairs(_dev(x, "x", torch.float32), _dev(s, "s", torch.float32),
                                 _dev(c, "c", torch.float32), n, _stream(stream, x.device)),
              "sincos_pairs")


def sincos_pairs_ex(x: torch.Tensor, s: torch.Tensor, c: torch.Tensor, reduction: str = "plain",
                    coef: str = "normalized", stream=None) -> None:
    """General forward; the output dtype is that of s and c (f32, bf16 or f16)."""
    n = x.numel()
    if s.numel() != n or c.numel() != n or s.dtype != c.dtype:
        raise ValueError("s and c must match x in size and each other in dtype")
    with _on_device(x.device):
        check(lib().sincos_pairs_ex(_dev(x, "x", torch.float32), _dev(s, "s"), _dev(c, "c"), n,
                                    _DTYPES[s.dtype], _REDUCTIONS[reduction], _COEFS[coef],
                                    _stream(stream, x.device)),
              "sincos_pairs_ex")


def sincos_expi(x: torch.Tensor, z: torch.Tensor, reduction: str = "plain",
                coef: str = "normalized", stream=None) -> None:
    """z = exp(i x) as interleaved (cos, sin): a complex64 tensor of x's size
    or a float32 tensor of twice its size."""
    n = x.numel()
    zf = torch.view_as_real(z) if z.is_complex() else z
    if zf.dtype != torch.float32 or zf.numel() != 2 * n:
        raise ValueError("z must be complex64 with x's size, or float32 with twice it")
    with _on_device(x.device):
        check(lib().sincos_expi(_dev(x, "x", torch.float32), _dev(zf, "z"), n,
                                _REDUCTIONS[reduction], _COEFS[coef], _stream(stream, x.device)),
              "sincos_expi")


def expi(x: torch.Tensor, reduction: str = "plain", coef: str = "normalized") -> torch.Tensor:
    """exp(i x) as a new complex64 tensor shaped like x."""
    z = torch.empty(x.shape, dtype=torch.complex64, device=x.device)
    sincos_expi(x.contiguous(), z, reduction, coef)
    return z


def _huygens_args(p, q, a, u):
    px, py, pz = p
    qx, qy, qz = q
    a = a if a.is_complex() else torch.complex(a, torch.zeros_like(a))
    af = torch.view_as_real(a.contiguous())
    ar, ai = af[:, 0].contiguous(), af[:, 1].contiguous()
    uf = torch.view_as_real(u) if u.is_complex() else u
    m, n = px.numel(), qx.numel()
    if uf.numel() != 2 * m:
        raise ValueError("u must be complex64 with m elements or float32 with 2m")
    ptrs = [_dev(t, name, torch.float32) for t, name in
            ((px, "px"), (py, "py"), (pz, "pz"), (qx, "qx"), (qy, "qy"), (qz, "qz"),
             (ar, "ar"), (ai, "ai"))]
    return ptrs, m, n, _dev(uf, "u", torch.float32), (ar, ai)


def sincos_huygens(p, q, a: torch.Tensor, k: float, u: torch.Tensor,
                   reduction: str = "compensated", stream=None) -> None:
    """u_i = sum_j a_j exp(i k |p_i - q_j|) / |p_i - q_j|; p and q are (x, y, z)
    triples of float32 CUDA tensors, a complex (or real) amplitudes."""
    ptrs, m, n, up, keep = _huygens_args(p, q, a, u)
    with _on_device(u.device):
        check(lib().sincos_huygens(ptrs[0], ptrs[1], ptrs[2], m, ptrs[3], ptrs[4], ptrs[5],
                                   ptrs[6], ptrs[7], n, float(k), _REDUCTIONS[reduction], up,
                                   _stream(stream, u.device)), "sincos_huygens")
        del keep


def huygens(p, q, a: torch.Tensor, k: float, reduction: str = "compensated") -> torch.Tensor:
    """The Huygens field sum as a new complex64 tensor of the points' size."""
    u = torch.empty(p[0].numel(), dtype=torch.complex64, device=p[0].device)
    sincos_huygens(p, q, a, k, u, reduction)
    return u


def sincos_autotune_huygens(p, q, a, k: float, u, reduction: str = "compensated",
                            stream=None) -> dict:
    ptrs, m, n, up, keep = _huygens_args(p, q, a, u)
    plan = _lib.sincos_plan()
    with _on_device(u.device):
        check(lib().sincos_autotune_huygens(ptrs[0], ptrs[1], ptrs[2], m, ptrs[3], ptrs[4],
                                            ptrs[5], ptrs[6], ptrs[7], n, float(k),
                                            _REDUCTIONS[reduction], up,
                                            _stream(stream, u.device), ctypes.byref(plan)),
              "sincos_autotune_huygens")
        del keep
    return plan.as_dict()


def sincos_backward(gs, gc, s: torch.Tensor, c: torch.Tensor, gx: torch.Tensor,
                    stream=None) -> None:
    """gx = gs*c - gc*s; gs or gc may be None (an all-zero upstream gradient)."""
    n = gx.numel()
    for t in (gs, gc, s, c):
        if t is not None and t.numel() != n:
            raise ValueError("all arrays must have the same number of elements")
    with _on_device(gx.device):
        check(lib().sincos_backward(
            None if gs is None else _dev(gs, "gs", torch.float32),
            None if gc is None else _dev(gc, "gc", torch.float32),
            _dev(s, "s", torch.float32), _dev(c, "c", torch.float32),
            _dev(gx, "gx", torch.float32), n, _stream(stream, gx.device)),
            "sincos_backward")


def segments(x: torch.Tensor, s: torch.Tensor, c: torch.Tensor, offsets, lens):
    """Device descriptor and length arrays for segments packed in x, s, c.

    Segment i is elements [offsets[i], offsets[i] + lens[i]) of each of the
    three flat arrays.  Returns (segs, lens) device tensors for sincos_batched."""
    offsets = np.asarray(offsets, dtype=np.int64)
    lens_np = np.asarray(lens, dtype=np.int64)
    osz = s.element_size()
    desc = np.empty((offsets.size, 3), dtype=np.uint64)
    desc[:, 0] = np.uint64(_dev(x, "x", torch.float32)) + (offsets * 4).astype(np.uint64)
    desc[:, 1] = np.uint64(_dev(s, "s")) + (offsets * osz).astype(np.uint64)
    desc[:, 2] = np.uint64(_dev(c, "c")) + (offsets * osz).astype(np.uint64)
    segs_t = torch.from_numpy(desc.view(np.int64).reshape(-1)).to(x.device)
    lens_t = torch.from_numpy(lens_np).to(x.device)
    return segs_t, lens_t


def segments_from_lists(xs, ss, cs):
    """Device descriptor and length arrays for separate per-segment tensors."""
    desc = np.array([[_dev(a, "x", torch.float32), _dev(b, "s"), _dev(d, "c")]
                     for a, b, d in zip(xs, ss, cs)], dtype=np.uint64)
    lens_np = np.array([a.numel() for a in xs], dtype=np.int64)
    dev = xs[0].device
    return (torch.from_numpy(desc.view(np.int64).reshape(-1)).to(dev),
            torch.from_numpy(lens_np).to(dev))


def sincos_batched(segs: torch.Tensor, lens: torch.Tensor, out_dtype="f32",
                   reduction: str = "plain", coef: str = "normalized", stream=None) -> None:
    """All segments at once: one self-scheduling launch with the binary32
    default plan, a schedule kernel and a tile kernel with register plans."""
    count = lens.numel()
    with _on_device(lens.device):
        check(lib().sincos_batched_ex(_dev(segs, "segs"), _dev(lens, "lens", torch.int64), count,
                                      _DTYPES[_torch_dtype(out_dtype)], _REDUCTIONS[reduction],
                                      _COEFS[coef], _stream(stream, lens.device)),
              "sincos_batched_ex")


def sincos_batched_noalloc(segs: torch.Tensor, lens: torch.Tensor, out_dtype="f32",
                           reduction: str = "plain", coef: str = "normalized",
                           stream=None) -> None:
    """sincos_batched without any device allocation, for callers that must not
    allocate (its scratch is a fixed array inside the library, shared by all
    calls; at most ``NOALLOC_MAX_SEGMENTS`` arrays; calls must not overlap on
    the GPU)."""
    count = lens.numel()
    with _on_device(lens.device):
        check(lib().sincos_batched_noalloc(_dev(segs, "segs"), _dev(lens, "lens", torch.int64),
                                           count, _DTYPES[_torch_dtype(out_dtype)],
                                           _REDUCTIONS[reduction], _COEFS[coef],
                                           _stream(stream, lens.device)),
              "sincos_batched_noalloc")


def sincos_batched_release() -> None:
    check(lib().sincos_batched_release(), "sincos_batched_release")


class BatchedGraph:
    """sincos_batched_graph_*: the batched launch captured once, replayed by launch()."""

    def __init__(self, segs: torch.Tensor, lens: torch.Tensor, out_dtype="f32",
                 reduction: str = "plain", coef: str = "normalized"):
        self._keep = (segs, lens)
        self.device = lens.device
        self._h = ctypes.c_void_p()
        with _on_device(self.device):
            check(lib().sincos_batched_graph_create(
                _dev(segs, "segs"), _dev(lens, "lens", torch.int64), lens.numel(),
                _DTYPES[_torch_dtype(out_dtype)], _REDUCTIONS[reduction], _COEFS[coef],
                ctypes.byref(self._h)), "sincos_batched_graph_create")

    def launch(self, stream=None) -> None:
        with _on_device(self.device):
            check(lib().sincos_batched_graph_launch(self._h, _stream(stream, self.device)),
                  "sincos_batched_graph_launch")

    def close(self) -> None:
        if self._h:
            check(lib().sincos_batched_graph_destroy(self._h), "sincos_batched_graph_destroy")
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sincos_host_workspace_bytes(out_dtype, chunk_elems: int) -> int:
    return int(lib().sincos_host_workspace_bytes(_DTYPES[_torch_dtype(out_dtype)], chunk_elems))


def sincos_pairs_host(x_host: torch.Tensor, s_host: torch.Tensor, c_host: torch.Tensor,
                      workspace: torch.Tensor, reduction: str = "plain",
                      coef: str = "normalized", stream=None) -> None:
    """Forward on host tensors through a caller-provided device workspace."""
    n = x_host.numel()
    if s_host.numel() != n or c_host.numel() != n or s_host.dtype != c_host.dtype:
        raise ValueError("s_host and c_host must match x_host in size and each other in dtype")
    ws = _dev(workspace, "workspace")
    with _on_device(workspace.device):
        check(lib().sincos_pairs_host(
            _host(x_host, "x_host", torch.float32), _host(s_host, "s_host"),
            _host(c_host, "c_host"), n, _DTYPES[s_host.dtype], _REDUCTIONS[reduction],
            _COEFS[coef], ws, workspace.numel() * workspace.element_size(),
            _stream(stream, workspace.device)), "sincos_pairs_host")


_HOST_PATHS = {_lib.HOST_PATH_NONE: "none", _lib.HOST_PATH_ZERO_COPY: "zero-copy",
               _lib.HOST_PATH_PIPELINE: "pipeline",
               _lib.HOST_PATH_ZERO_COPY_PAGEABLE: "zero-copy-pageable"}
_HOST_ROUTES = {"auto": _lib.HOST_ROUTE_AUTO, "pipeline": _lib.HOST_ROUTE_PIPELINE}


def sincos_host_last_path() -> str:
    """The route of this thread's last sincos_pairs_host call: "zero-copy"
    (one kernel on page-locked host buffers), "zero-copy-pageable" (one kernel,
    pageable memory through the host's page tables), "pipeline" (chunked
    copies) or "none"."""
    return _HOST_PATHS[lib().sincos_host_last_path()]


def sincos_host_route_set(policy: str) -> None:
    """"auto" (zero-copy whenever the device can reach the buffers) or
    "pipeline" (always chunked copies), for the whole process."""
    check(lib().sincos_host_route_set(_HOST_ROUTES[policy]), "sincos_host_route_set")


# -----------------------------------------------------------------------------
# Plans and the autotuner
# -----------------------------------------------------------------------------

def sincos_plan_get(op: str, out_dtype, n: int) -> dict:
    p = _lib.sincos_plan()
    check(lib().sincos_plan_get(_OPS[op], _DTYPES[_torch_dtype(out_dtype)], n, ctypes.byref(p)),
          "sincos_plan_get")
    return p.as_dict()


def sincos_plan_set(op: str, out_dtype, n: int, block: int, unroll: int, ctas_per_sm: int,
                    vec_bytes: int = 32):
    p = _lib.sincos_plan(block, unroll, ctas_per_sm, vec_bytes)
    check(lib().sincos_plan_set(_OPS[op], _DTYPES[_torch_dtype(out_dtype)], n, ctypes.byref(p)),
          "sincos_plan_set")


def sincos_autotune_pairs(x, s, c, reduction: str = "plain", coef: str = "normalized",
                          stream=None) -> dict:
    p = _lib.sincos_plan()
    with _on_device(x.device):
        check(lib().sincos_autotune_pairs(
            _dev(x, "x", torch.float32), _dev(s, "s"), _dev(c, "c"), x.numel(),
            _DTYPES[s.dtype], _REDUCTIONS[reduction], _COEFS[coef], _stream(stream, x.device),
            ctypes.byref(p)), "sincos_autotune_pairs")
    return p.as_dict()


def sincos_autotune_expi(x, z, reduction: str = "plain", coef: str = "normalized",
                         stream=None) -> dict:
    p = _lib.sincos_plan()
    zf = torch.view_as_real(z) if z.is_complex() else z
    with _on_device(x.device):
        check(lib().sincos_autotune_expi(_dev(x, "x", torch.float32), _dev(zf, "z"), x.numel(),
                                         _REDUCTIONS[reduction], _COEFS[coef],
                                         _stream(stream, x.device), ctypes.byref(p)),
              "sincos_autotune_expi")
    return p.as_dict()


def sincos_autotune_backward(gs, gc, s, c, gx, stream=None) -> dict:
    p = _lib.sincos_plan()
    with _on_device(gx.device):
        check(lib().sincos_autotune_backward(
            None if gs is None else _dev(gs, "gs", torch.float32),
            None if gc is None else _dev(gc, "gc", torch.float32),
            _dev(s, "s", torch.float32), _dev(c, "c", torch.float32),
            _dev(gx, "gx", torch.float32), gx.numel(), _stream(stream, gx.device),
            ctypes.byref(p)), "sincos_autotune_backward")
    return p.as_dict()


def sincos_autotune_batched(segs, lens, out_dtype="f32", reduction: str = "plain",
                            coef: str = "normalized", stream=None) -> dict:
    p = _lib.sincos_plan()
    with _on_device(lens.device):
        check(lib().sincos_autotune_batched(
            _dev(segs, "segs"), _dev(lens, "lens", torch.int64), lens.numel(),
            _DTYPES[_torch_dtype(out_dtype)], _REDUCTIONS[reduction], _COEFS[coef],
            _stream(stream, lens.device), ctypes.byref(p)), "sincos_autotune_batched")
    return p.as_dict()


def sincos_plan_cache_save(path: str) -> None:
    check(lib().sincos_plan_cache_save(path.encode()), "sincos_plan_cache_save")


def sincos_plan_cache_load(path: str) -> None:
    check(lib().sincos_plan_cache_load(path.encode()), "sincos_plan_cache_load")


def sincos_device_wait_timeouts() -> int:
    """Bounded waits that gave up in bulk-path kernels since the last call."""
    return int(lib().sincos_device_wait_timeouts())


def sincos_device_bad_segments() -> int:
    """Batched arrays skipped for a null or misaligned descriptor since the
    last call."""
    return int(lib().sincos_device_bad_segments())


def sincos_seg_check(x: int, s: int, c: int, length: int, out_dtype="f32") -> bool:
    """The batched kernels' descriptor check on the host, for raw addresses."""
    seg = _lib.sincos_seg(x, s, c)
    return lib().sincos_seg_check(ctypes.byref(seg), int(length),
                                  _DTYPES[_torch_dtype(out_dtype)]) == _lib.OK


def sincos_launch_count() -> int:
    return int(lib().sincos_launch_count())


def sincos_version() -> int:
    return int(lib().sincos_version())


# -----------------------------------------------------------------------------
# Torch front end
# -----------------------------------------------------------------------------

def sincos(x: torch.Tensor, out_dtype=torch.float32, reduction: str = "plain",
           coef: str = "normalized"):
    """(sin x, cos x) as two new tensors shaped like x."""
    out_dtype = _torch_dtype(out_dtype)
    xc = x.contiguous()
    s = torch.empty(x.shape, dtype=out_dtype, device=x.device)
    c = torch.empty(x.shape, dtype=out_dtype, device=x.device)
    sincos_pairs_ex(xc, s, c, reduction, coef)
    return s, c


class SinCosFn(torch.autograd.Function):
    """(s, c) = (sin x, cos x) with the hand-written backward gx = gs*c - gc*s."""

    @staticmethod
    def forward(ctx, x, reduction="plain", coef="normalized"):
        s, c = sincos(x, torch.float32, reduction, coef)
        ctx.save_for_backward(s, c)
        return s, c

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gs, gc):
        # The kernel's gradient carries no graph of its own, so a second
        # derivative is refused rather than silently taken as zero.
        s, c = ctx.saved_tensors
        gs = None if gs is None else gs.contiguous()
        gc = None if gc is None else gc.contiguous()
        gx = torch.empty_like(s)
        sincos_backward(gs, gc, s, c, gx)
        return gx, None, None


def sincos_autograd(x: torch.Tensor, reduction: str = "plain", coef: str = "normalized"):
    return SinCosFn.apply(x, reduction, coef)
