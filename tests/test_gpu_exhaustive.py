"""Every binary32 input: all 2^32 bit patterns through the GPU kernel and the
oracle, in chunks of 2^28, compared bit for bit (NaN results compared as NaN:
their payloads are not part of the method).

The oracle side is the threaded driver of the pinned per-element function;
16-bit results are its binary32 results through the oracle's own
round-to-nearest-even conversion, exactly as its 16-bit entry point does."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_cs_0406049_gb300 import api

pytestmark = pytest.mark.gpu

CHUNK = 1 << 28
DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def _nan_bits(v: np.ndarray, out: str) -> np.ndarray:
    if out == "f32":
        return np.isnan(v.view(np.float32))
    if out == "bf16":
        return ((v & 0x7f80) == 0x7f80) & ((v & 0x007f) != 0)
    return ((v & 0x7c00) == 0x7c00) & ((v & 0x03ff) != 0)


@pytest.mark.parametrize("reduction,coef,out", [
    ("plain", "normalized", "f32"),
    ("compensated", "normalized", "f32"),
    ("plain", "dagger", "f32"),
    ("compensated", "normalized", "bf16"),
    ("compensated", "normalized", "f16"),
])
def test_every_binary32_input(cuda_lib, reduction, coef, out):
    lib = oracle.default()
    threads = len(os.sched_getaffinity(0))
    xg = torch.empty(CHUNK, dtype=torch.float32, device="cuda")
    sg = torch.empty(CHUNK, dtype=DT[out], device="cuda")
    cg = torch.empty_like(sg)
    so = np.empty(CHUNK, np.float32)
    co = np.empty(CHUNK, np.float32)
    ubits = np.uint32 if out == "f32" else np.uint16
    nan_results = 0
    for k in range((1 << 32) // CHUNK):
        bits = np.arange(k * CHUNK, (k + 1) * CHUNK, dtype=np.uint32)
        x = bits.view(np.float32)
        xg.copy_(torch.from_numpy(x))
        api.sincos_pairs_ex(xg, sg, cg, reduction, coef)
        lib.sincos_mt(x, so, co, reduction=reduction, coef=coef, threads=threads)
        torch.cuda.synchronize()
        for name, got_t, want32 in (("s", sg, so), ("c", cg, co)):
            got = got_t.cpu().view(torch.int32 if out == "f32" else torch.int16).numpy()
            got = got.view(ubits)
            want = want32.view(np.uint32) if out == "f32" else lib.round16(want32, out)
            diff = np.flatnonzero(got != want)
            if diff.size:
                both_nan = _nan_bits(got[diff], out) & _nan_bits(want[diff], out)
                bad = diff[~both_nan]
                assert bad.size == 0, (
                    f"{reduction}/{coef}/{out} {name}: {bad.size} inputs differ, first at bit "
                    f"patterns {[hex(v) for v in bits[bad[:4]]]}: gpu "
                    f"{[hex(v) for v in got[bad[:4]]]} oracle {[hex(v) for v in want[bad[:4]]]}")
                nan_results += int(both_nan.sum())
    # only NaN and infinite inputs give NaN: 2^24 patterns of each sign, two outputs
    assert nan_results <= 2 * (1 << 24) * 2
    assert api.sincos_device_wait_timeouts() == 0
