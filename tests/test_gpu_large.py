"""Arrays past 2^31 elements: 64-bit indexing in every kernel, sampled against
the oracle (the angles are generated on the device; the sampled ones are
copied back for the oracle)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import as_np, assert_f32_parity, forced_plan
from paper_cs_0406049_gb300 import api

pytestmark = pytest.mark.gpu

N = (1 << 31) + 4099


def big_angles(n):
    """Deterministic angles in [-500, 500) without a host copy of the array."""
    i = torch.arange(n, device="cuda", dtype=torch.int64)
    return ((i * 7919) % 100003).to(torch.float32) * 0.01 - 500.0


def sample_idx(n):
    rng = np.random.default_rng(1)
    edge = np.concatenate([np.arange(64), np.arange((1 << 31) - 64, (1 << 31) + 64),
                           np.arange(n - 64, n)])
    idx = np.unique(np.concatenate([edge, rng.integers(0, n, 1 << 16)]))
    return idx[(idx >= 0) & (idx < n)]


@pytest.mark.parametrize("plan", [(512, 2, 1, 0), (256, 8, 4, 16)])
def test_forward_past_2_31(cuda_lib, plan):
    x = big_angles(N)
    s = torch.empty_like(x)
    c = torch.empty_like(x)
    with forced_plan("pairs", "f32", plan):
        api.sincos_pairs(x, s, c)
    torch.cuda.synchronize()
    idx = sample_idx(N)
    it = torch.from_numpy(idx).cuda()
    ws, wc = oracle.sincos(as_np(x[it]))
    assert_f32_parity(as_np(s[it]), ws, f"big s {plan}")
    assert_f32_parity(as_np(c[it]), wc, f"big c {plan}")
    assert api.sincos_device_wait_timeouts() == 0


def test_backward_and_expi_past_2_31(cuda_lib):
    n = (1 << 31) + 5
    x = big_angles(n)
    idx = sample_idx(n)
    it = torch.from_numpy(idx).cuda()
    z = torch.empty(n, dtype=torch.complex64, device="cuda")
    api.sincos_expi(x, z)
    torch.cuda.synchronize()
    ws, wc = oracle.sincos(as_np(x[it]))
    zr = torch.view_as_real(z)[it].cpu().numpy()
    assert_f32_parity(zr[:, 0].copy(), wc, "big expi c")
    assert_f32_parity(zr[:, 1].copy(), ws, "big expi s")
    del z
    s = torch.empty_like(x)
    c = torch.empty_like(x)
    api.sincos_pairs(x, s, c)
    gx = x                                  # in place over the angles
    gs = torch.ones_like(x)
    api.sincos_backward(gs, None, s, c, gx)
    torch.cuda.synchronize()
    want = oracle.backward(np.ones(idx.size, np.float32), None, as_np(s[it]), as_np(c[it]))
    assert_f32_parity(as_np(gx[it]), want, "big backward")


@pytest.mark.parametrize("plan", [(512, 2, 1, 0), (1024, 2, 1, 16)])
def test_batched_segment_past_2_31(cuda_lib, plan):
    lens = [1000, (1 << 31) + 3, 77]
    total = sum(lens)
    x = big_angles(total)
    s = torch.empty_like(x)
    c = torch.empty_like(x)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    segs, lens_t = api.segments(x, s, c, offs, lens)
    with forced_plan("batched", "f32", plan):
        api.sincos_batched(segs, lens_t)
    torch.cuda.synchronize()
    idx = sample_idx(total)
    it = torch.from_numpy(idx).cuda()
    ws, wc = oracle.sincos(as_np(x[it]))
    assert_f32_parity(as_np(s[it]), ws, f"big batched s {plan}")
    assert_f32_parity(as_np(c[it]), wc, f"big batched c {plan}")
