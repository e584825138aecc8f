"""GPU forward against the CPU oracle, element by element, through the C ABI.

Tolerance: |gpu - oracle| <= 2.4e-7 (2 ulp of 1.0) for binary32 results; the
design (same operation tree, explicit roundings, no contraction, no flush to
zero) also makes them bit-identical, which is asserted too.  16-bit outputs
must equal the oracle's round-to-nearest-even bit patterns.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import (PARITY_ABS_TOL, as_np, assert_16_parity, assert_f32_parity,
                      forced_plan, mixed_angles, special_angles)
from paper_cs_0406049_gb300 import api, workloads

pytestmark = pytest.mark.gpu

DTYPES = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
VARIANTS = [(d, r, c) for d in DTYPES for r in ("plain", "compensated")
            for c in ("normalized", "dagger")]
SIZES = [1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 33, 63, 65, 255, 257, 1023, 1025, 4095, 4097,
         65535, 65537, 262147, (1 << 20) + 5]
GUARD = 64
SENTINEL32 = np.uint32(0x7fa5a5a5)     # a NaN pattern no kernel writes
SENTINEL16 = np.uint16(0x7da5)


def oracle_out(x, dtype, red, coef):
    return oracle.sincos(x, reduction=red, coef=coef, out=dtype)


def check(dtype, got_s, got_c, want_s, want_c, what):
    if dtype == "f32":
        assert_f32_parity(got_s, want_s, what + " s")
        assert_f32_parity(got_c, want_c, what + " c")
    else:
        assert_16_parity(got_s, want_s, dtype == "bf16", what + " s")
        assert_16_parity(got_c, want_c, dtype == "bf16", what + " c")


def run_guarded(x, dtype, red, coef, offs):
    """Forward on sub-ranges of guard-padded device buffers; returns (s, c)
    and asserts that no element outside [0, n) of any buffer was written."""
    n = x.size
    ox, os_, oc = offs
    tdt = DTYPES[dtype]
    xb = torch.zeros(n + 2 * GUARD, dtype=torch.float32, device="cuda")
    xb[GUARD + ox:GUARD + ox + n] = torch.from_numpy(x).cuda()
    if dtype == "f32":
        fill = torch.tensor(SENTINEL32.view(np.int32)).item()
        sb = torch.full((n + 2 * GUARD,), fill, dtype=torch.int32, device="cuda").view(tdt)
        cb = sb.clone()
    else:
        fill = int(SENTINEL16.view(np.int16))
        sb = torch.full((n + 2 * GUARD,), fill, dtype=torch.int16, device="cuda").view(tdt)
        cb = sb.clone()
    xs = xb[GUARD + ox:GUARD + ox + n]
    ss = sb[GUARD + os_:GUARD + os_ + n]
    cs = cb[GUARD + oc:GUARD + oc + n]
    api.sincos_pairs_ex(xs, ss, cs, red, coef)
    torch.cuda.synchronize()
    for buf, o in ((sb, os_), (cb, oc)):
        raw = as_np(buf)
        if dtype == "f32":
            raw = raw.view(np.uint32)
            sent = SENTINEL32
        else:
            sent = SENTINEL16
        assert np.all(raw[:GUARD + o] == sent), "write before the output range"
        assert np.all(raw[GUARD + o + n:] == sent), "write after the output range"
    return as_np(ss), as_np(cs)


# Element offsets (x, s, c) into guard-padded buffers.  Equal offsets share a
# 128-byte line grid (line-aligned vector path after a scalar head); (0, 1, 2),
# (3, 0, 1) in f32 still share a 16-byte grid for some heads or none; for
# 16-bit outputs (1, 5, 5), (2, 4, 4) and (0, 1, 3) admit no common vector
# alignment (element-wise path).
OFFSETS = {
    "f32": [(0, 0, 0), (1, 1, 1), (2, 2, 2), (3, 3, 3), (0, 1, 2), (3, 0, 1)],
    "bf16": [(0, 0, 0), (1, 1, 1), (3, 3, 3), (1, 5, 5), (2, 4, 4), (0, 1, 3)],
    "f16": [(0, 0, 0), (1, 1, 1), (3, 3, 3), (1, 5, 5), (2, 4, 4), (0, 1, 3)],
}


PATHS = {"bulk": (512, 2, 1, 0), "bulk_small": (256, 2, 2, 0), "reg16": (256, 8, 4, 16),
         "reg32": (256, 4, 4, 32)}


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("dtype,red,coef", VARIANTS)
def test_ragged_sizes_and_alignments(cuda_lib, dtype, red, coef, path):
    with forced_plan("pairs", dtype, PATHS[path]):
        for n in SIZES:
            x = mixed_angles(n, seed=n)
            want_s, want_c = oracle_out(x, dtype, red, coef)
            for offs in OFFSETS[dtype]:
                if n > 70000 and offs != (0, 0, 0) and offs != OFFSETS[dtype][1]:
                    continue
                s, c = run_guarded(x, dtype, red, coef, offs)
                check(dtype, s, c, want_s, want_c,
                      f"{path} {dtype}/{red}/{coef} n={n} offs={offs}")
    assert api.sincos_device_wait_timeouts() == 0


BULK_SIZES = [8191, 8192, 8193, 8192 + 31, 8192 + 33, 2 * 8192, 3 * 8192 + 5, 152 * 8192,
              152 * 8192 + 8191, 153 * 8192 - 1, 1000 * 8192 + 4099]


@pytest.mark.parametrize("block", [128, 256, 512, 1024])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_bulk_path_chunk_boundaries(cuda_lib, dtype, block):
    """Whole chunks, partial tails and heads around the 8192-angle chunk and
    the 152-CTA grid, on line-aligned and offset pointers."""
    with forced_plan("pairs", dtype, (block, 2, 1, 0)):
        for n in BULK_SIZES:
            x = mixed_angles(n, seed=n + block)
            want_s, want_c = oracle_out(x, dtype, "plain", "normalized")
            for offs in OFFSETS[dtype][:2]:
                s, c = run_guarded(x, dtype, "plain", "normalized", offs)
                check(dtype, s, c, want_s, want_c, f"bulk{block} {dtype} n={n} offs={offs}")
    assert api.sincos_device_wait_timeouts() == 0


SMALL_BULK_SIZES = [4095, 4096, 4097, 4096 + 31, 2 * 4096 + 5, 456 * 4096, 456 * 4096 + 4095,
                    457 * 4096 - 1, 2000 * 4096 + 2049]


@pytest.mark.parametrize("block", [128, 256, 512])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_small_stage_bulk_path_chunk_boundaries(cuda_lib, dtype, block):
    """The 4096-angle-stage variant (several CTAs per SM): whole chunks, tails
    and heads around its chunk and its larger grid."""
    with forced_plan("pairs", dtype, (block, 2, 2, 0)):
        for n in SMALL_BULK_SIZES:
            x = mixed_angles(n, seed=n + block + 1)
            want_s, want_c = oracle_out(x, dtype, "compensated", "normalized")
            for offs in OFFSETS[dtype][:2]:
                s, c = run_guarded(x, dtype, "compensated", "normalized", offs)
                check(dtype, s, c, want_s, want_c,
                      f"small bulk{block} {dtype} n={n} offs={offs}")
    assert api.sincos_device_wait_timeouts() == 0


def test_plain_entry_point_on_the_plain_workload(cuda_lib):
    """sincos_pairs on 2^20 angles U[-pi, pi) (seed 0): every element."""
    x = workloads.plain()
    xt = torch.from_numpy(x).cuda()
    s = torch.empty_like(xt)
    c = torch.empty_like(xt)
    api.sincos_pairs(xt, s, c)
    torch.cuda.synchronize()
    want_s, want_c = oracle.sincos(x)
    assert_f32_parity(as_np(s), want_s, "s")
    assert_f32_parity(as_np(c), want_c, "c")
    st = oracle.error_stats(x, as_np(s), as_np(c))
    # the paper's first-method statistics hold for the GPU results as well
    assert st["rms_euclid"] <= 1.3e-7 and st["max_amp"] <= 2e-7


def test_special_values(cuda_lib):
    x = np.tile(special_angles(), 37)
    for dtype, red, coef in VARIANTS:
        s, c = run_guarded(x, dtype, red, coef, (0, 0, 0))
        want_s, want_c = oracle_out(x, dtype, red, coef)
        check(dtype, s, c, want_s, want_c, f"special {dtype}/{red}/{coef}")


def test_every_float_in_a_binade(cuda_lib):
    """All 2^23 binary32 values in [2, 4): the range that wraps at pi."""
    x = np.arange(np.float32(2.0).view(np.int32), np.float32(4.0).view(np.int32),
                  dtype=np.int32).view(np.float32)
    xt = torch.from_numpy(x).cuda()
    for red in ("plain", "compensated"):
        s = torch.empty_like(xt)
        c = torch.empty_like(xt)
        api.sincos_pairs_ex(xt, s, c, red)
        want_s, want_c = oracle.sincos(x, reduction=red)
        assert_f32_parity(as_np(s), want_s, red + " s")
        assert_f32_parity(as_np(c), want_c, red + " c")


@pytest.mark.parametrize("path", sorted(PATHS))
def test_in_place(cuda_lib, path):
    with forced_plan("pairs", "f32", PATHS[path]):
        _in_place()


def _in_place():
    x = mixed_angles(100003, seed=5)
    want_s, want_c = oracle.sincos(x)
    buf = torch.from_numpy(x.copy()).cuda()
    c = torch.empty_like(buf)
    api.sincos_pairs(buf, buf, c)          # sines overwrite the angles
    assert_f32_parity(as_np(buf), want_s, "in-place s")
    assert_f32_parity(as_np(c), want_c, "in-place c")
    buf = torch.from_numpy(x.copy()).cuda()
    s = torch.empty_like(buf)
    api.sincos_pairs(buf, s, buf)          # cosines overwrite the angles
    assert_f32_parity(as_np(s), want_s, "in-place s2")
    assert_f32_parity(as_np(buf), want_c, "in-place c2")


def test_zero_length_enqueues_nothing(cuda_lib):
    x = torch.empty(0, device="cuda")
    before = api.sincos_launch_count()
    api.sincos_pairs(x, x, x)
    assert api.sincos_launch_count() == before


def _sampled_parity(x_np, xt, dtype, red, coef, n_sample=1 << 20, seed=0):
    s = torch.empty(xt.numel(), dtype=DTYPES[dtype], device="cuda")
    c = torch.empty_like(s)
    api.sincos_pairs_ex(xt, s, c, red, coef)
    torch.cuda.synchronize()
    n = x_np.size
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([np.arange(4096), np.arange(n - 4096, n),
                                    rng.integers(0, n, n_sample)]))
    it = torch.from_numpy(idx).cuda()
    gs, gc = as_np(s[it]), as_np(c[it])
    want_s, want_c = oracle_out(x_np[idx], dtype, red, coef)
    check(dtype, gs, gc, want_s, want_c, f"{dtype}/{red}/{coef} sampled")
    return idx, gs, gc


def test_bandwidth_workload_full_size(cuda_lib):
    """2^28 angles U[-1000, 1000) (seed 1), the launch the benchmark times:
    sampled outputs against the oracle, and the plain-reduction error bound."""
    x = workloads.bandwidth()
    xt = torch.from_numpy(x).cuda()
    idx, s, c = _sampled_parity(x, xt, "f32", "plain", "normalized")
    st = oracle.error_stats(x[idx], s, c)
    assert st["max_abs"] < 1.2e-4      # 2 pi |x1| 2^-23 at |x| = 1000, plus the method's 5e-7


@pytest.mark.parametrize("dtype,red", [("f32", "plain"), ("f32", "compensated"),
                                       ("bf16", "compensated"), ("f16", "compensated")])
def test_precision_workload_full_size(cuda_lib, dtype, red):
    """2^26 angles, |x| log-uniform in [1e-3, 1e5] (seed 2)."""
    x = workloads.precision()
    xt = torch.from_numpy(x).cuda()
    idx, s, c = _sampled_parity(x, xt, dtype, red, "normalized")
    if dtype == "f32" and red == "compensated":
        assert oracle.error_stats(x[idx], s, c)["max_abs"] <= 7e-7
