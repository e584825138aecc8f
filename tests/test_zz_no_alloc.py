"""The allocation-free batched entry point, through the C ABI.

`sincos_batched_noalloc` serves callers that may not allocate device memory:
a plug-in whose host program owns all GPU memory, a real-time thread that
cannot afford the device synchronization cudaMalloc may cause, code with a
memory budget fixed at start-up.  Its schedule scratch is a fixed array inside
the library, which only register plans (vec_bytes 16 or 32) use: the ring
kernel of the binary32 default plan schedules itself.  So most checks here run
under register plans (forced; the defaults for 16-bit outputs are such plans),
where the launch counter moves by two per call (schedule kernel + tile
kernel), which shows the scratch array was written and read.

Every check makes two calls in a row, the second with fewer arrays than the
first, so the second call's schedule sits at other offsets of the shared
array than the first's and stale entries would show.  Each call's results are
compared element by element with the oracle, and with the existing entry
point `sincos_batched_ex` on the same plan.  The file is named to be collected
last.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

import oracle
from gpu_util import as_np, assert_16_parity, assert_f32_parity, forced_plan, mixed_angles
from paper_cs_0406049_gb300 import _lib, api

pytestmark = pytest.mark.gpu

DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
CODE = {"f32": _lib.F32, "bf16": _lib.BF16, "f16": _lib.F16}
REGISTER_PLANS = {"reg16": (1024, 2, 1, 16), "reg32": (256, 4, 8, 32)}
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _packed(lens, seed, dtype):
    lens = np.asarray(lens, np.int64)
    total = int(np.clip(lens, 0, None).sum())
    x = mixed_angles(total, seed)
    offs = np.concatenate([[0], np.cumsum(np.clip(lens, 0, None))[:-1]]).astype(np.int64)
    return x, torch.from_numpy(x).cuda(), offs, lens


def _check(x, s, c, dtype, red, coef, what):
    want_s, want_c = oracle.sincos(x, reduction=red, coef=coef, out=dtype)
    if dtype == "f32":
        assert_f32_parity(as_np(s), want_s, what + " s")
        assert_f32_parity(as_np(c), want_c, what + " c")
    else:
        assert_16_parity(as_np(s), want_s, dtype == "bf16", what + " s")
        assert_16_parity(as_np(c), want_c, dtype == "bf16", what + " c")


def _run_both(lib, lens, seed, dtype="f32", red="plain", coef="normalized", kernels=None):
    """One no-alloc call and one sincos_batched_ex call on the same arrays:
    each against the oracle, and the two bit for bit."""
    x, xt, offs, lens = _packed(lens, seed, dtype)
    n = xt.numel()
    s_ref = torch.full((n,), 5.0, device="cuda").to(DT[dtype])
    c_ref = torch.full((n,), 5.0, device="cuda").to(DT[dtype])
    s_new = torch.full((n,), 9.0, device="cuda").to(DT[dtype])
    c_new = torch.full((n,), 9.0, device="cuda").to(DT[dtype])
    segs_ref, lens_t = api.segments(xt, s_ref, c_ref, offs, lens)
    segs_new, _ = api.segments(xt, s_new, c_new, offs, lens)
    stream = torch.cuda.current_stream().cuda_stream
    args = (lens.size, CODE[dtype], api._REDUCTIONS[red], api._COEFS[coef], stream)
    before = lib.sincos_launch_count()
    assert lib.sincos_batched_noalloc(segs_new.data_ptr(), lens_t.data_ptr(), *args) == _lib.OK
    launched = lib.sincos_launch_count() - before
    torch.cuda.synchronize()
    if kernels is not None:
        assert launched == kernels, f"no-alloc call launched {launched} kernels, not {kernels}"
    assert lib.sincos_batched_ex(segs_ref.data_ptr(), lens_t.data_ptr(), *args) == _lib.OK
    torch.cuda.synchronize()
    _check(x, s_new, c_new, dtype, red, coef, f"no-alloc {dtype} {red}/{coef}")
    _check(x, s_ref, c_ref, dtype, red, coef, f"batched_ex {dtype} {red}/{coef}")
    assert torch.equal(s_new.view(torch.int16 if dtype != "f32" else torch.int32),
                       s_ref.view(torch.int16 if dtype != "f32" else torch.int32))
    assert torch.equal(c_new.view(torch.int16 if dtype != "f32" else torch.int32),
                       c_ref.view(torch.int16 if dtype != "f32" else torch.int32))
    assert api.sincos_device_wait_timeouts() == 0


def _two_calls(lib, dtype="f32", red="plain", coef="normalized", kernels=None):
    rng = np.random.default_rng(77)
    first = rng.integers(1, 20000, 3000)
    first[::97] = 0
    _run_both(lib, first, seed=1, dtype=dtype, red=red, coef=coef, kernels=kernels)
    second = rng.integers(1, 5000, 41)
    _run_both(lib, second, seed=2, dtype=dtype, red=red, coef=coef, kernels=kernels)


@pytest.mark.parametrize("plan", sorted(REGISTER_PLANS))
def test_noalloc_register_plans_two_calls(cuda_lib, plan):
    """Binary32 under a forced register plan: the scratch array is used."""
    with forced_plan("batched", "f32", REGISTER_PLANS[plan]):
        _two_calls(cuda_lib, kernels=2)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_noalloc_16bit_register_plans_two_calls(cuda_lib, dtype):
    """16-bit outputs under register plans (their defaults; forced here so
    that a plan tuned earlier in the same process cannot change the path)."""
    with forced_plan("batched", dtype, REGISTER_PLANS["reg32"]):
        _two_calls(cuda_lib, dtype=dtype, red="compensated", kernels=2)


def test_noalloc_dagger_register_plan(cuda_lib):
    with forced_plan("batched", "f32", REGISTER_PLANS["reg16"]):
        _two_calls(cuda_lib, red="compensated", coef="dagger", kernels=2)


def test_noalloc_ring_plan_two_calls(cuda_lib):
    """The binary32 bulk plan runs the ring kernel alone (one launch, no scratch)."""
    with forced_plan("batched", "f32", (512, 2, 1, 0)):
        _two_calls(cuda_lib, kernels=1)


def test_noalloc_limits(cuda_lib):
    lib = cuda_lib
    n = _lib.NOALLOC_MAX_SEGMENTS + 1
    lens = torch.ones(n, dtype=torch.int64, device="cuda")
    segs = torch.zeros(3 * n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    before = lib.sincos_launch_count()
    assert lib.sincos_batched_noalloc(segs.data_ptr(), lens.data_ptr(), n, _lib.F32,
                                      _lib.RED_PLAIN, _lib.COEF_NORMALIZED,
                                      stream) == _lib.EUNSUPPORTED
    assert b"SINCOS_NOALLOC_MAX_SEGMENTS" in lib.sincos_last_error()
    assert lib.sincos_batched_noalloc(None, None, 0, _lib.F32, _lib.RED_PLAIN,
                                      _lib.COEF_NORMALIZED, stream) == _lib.OK
    assert lib.sincos_launch_count() == before


@pytest.mark.parametrize("plan", sorted(REGISTER_PLANS))
def test_noalloc_at_the_maximum_count(cuda_lib, plan):
    """Exactly SINCOS_NOALLOC_MAX_SEGMENTS arrays of 1..7 angles each under a
    register plan (the whole array in use), then a small batch after it."""
    lens = (np.arange(_lib.NOALLOC_MAX_SEGMENTS) % 7 + 1).astype(np.int64)
    with forced_plan("batched", "f32", REGISTER_PLANS[plan]):
        _run_both(cuda_lib, lens, seed=3, kernels=2)
        _run_both(cuda_lib, [5, 0, 9000, 1], seed=4, kernels=2)


_FIRST_CALL_UNDER_CAPTURE = textwrap.dedent("""
    import sys
    import torch
    sys.path.insert(0, {root!r})
    from paper_cs_0406049_gb300 import _lib, api, build
    build.build()
    lib = _lib.load()
    api.sincos_plan_get("batched", "f32", 8)          # device facts, outside any capture
    x = torch.zeros(64, device="cuda")
    s, c = torch.empty_like(x), torch.empty_like(x)
    segs, lens = api.segments(x, s, c, [0, 32], [32, 32])
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        x.add_(0.0)                                     # keep the graph non-empty
        rc = lib.sincos_batched_noalloc(segs.data_ptr(), lens.data_ptr(), 2, _lib.F32,
                                        _lib.RED_PLAIN, _lib.COEF_NORMALIZED,
                                        side.cuda_stream)
    torch.cuda.synchronize()
    print("RC", rc)
""")


def test_noalloc_first_call_under_capture_is_refused(cuda_lib):
    """A fresh process whose first no-alloc call comes on a capturing stream
    gets SINCOS_ECAPTURE and nothing is enqueued (the address lookup would
    have run inside the capture)."""
    code = _FIRST_CALL_UNDER_CAPTURE.format(root=ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr
    assert f"RC {_lib.ECAPTURE}" in r.stdout, r.stdout + r.stderr
