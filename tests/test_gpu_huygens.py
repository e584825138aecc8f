"""Huygens field sum on the GPU against the oracle (same per-term operation
order and the same source-order summation, so the sums are bit-identical)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import as_np, assert_f32_parity, forced_plan
from paper_cs_0406049_gb300 import api, workloads
import pins

pytestmark = pytest.mark.gpu


def to_dev(p, q, a):
    P = tuple(torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in p)
    Q = tuple(torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in q)
    return P, Q, torch.from_numpy(a).cuda()


def gpu_field(p, q, a, k, red):
    P, Q, A = to_dev(p, q, a)
    u = api.huygens(P, Q, A, k, red)
    torch.cuda.synchronize()
    return torch.view_as_real(u).cpu().numpy().reshape(-1)


@pytest.mark.parametrize("plan", [(256, 2, 8, 16), (128, 1, 8, 16), (512, 4, 8, 16),
                                  (256, 4, 8, 16), (256, 1, 8, 32), (128, 2, 8, 32),
                                  (512, 4, 8, 32)])
@pytest.mark.parametrize("red", ["compensated", "plain"])
def test_huygens_ragged(cuda_lib, plan, red):
    with forced_plan("huygens", "f32", plan):
        for m, n in [(1, 1), (3, 5), (255, 2047), (257, 2049), (1000, 777), (4097, 4100),
                     (513, 0)]:
            p, q, a, k = pins.huygens_case(m=m, n=n, seed=m + n)
            want = oracle.huygens(p, q, a, k, red).view(np.float32)
            assert_f32_parity(gpu_field(p, q, a, k, red), want, f"huygens {plan} {red} {m}x{n}")


@pytest.mark.parametrize("plan", [(256, 1, 8, 16), (256, 1, 8, 32), (128, 4, 8, 32)])
@pytest.mark.parametrize("red", ["compensated", "plain"])
def test_huygens_one_term_per_point(cuda_lib, plan, red):
    """One source and 2^20 + 3 points: every output is a single term
    w (a exp(i k r)), so each phase factor (and each packed pair of them) is
    compared on its own, not inside a sum.  Distances from 1e-3 to 3e3 at
    k = 37.7 put k r across 1.8e4 revolutions and every reduced angle."""
    m = (1 << 20) + 3
    rng = np.random.default_rng(17)
    d = np.exp(rng.uniform(np.log(1e-3), np.log(3e3), m))
    u = rng.standard_normal((m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    p = tuple((d[:, None] * u)[:, i].astype(np.float32) for i in range(3))
    q = tuple(np.array([v], np.float32) for v in (0.25, -0.5, 0.125))
    a = np.array([0.75 - 1.25j], np.complex64)
    k = float(np.float32(37.7))
    with forced_plan("huygens", "f32", plan):
        got = gpu_field(p, q, a, k, red)
    want = oracle.huygens(p, q, a, k, red).view(np.float32)
    assert_f32_parity(got, want, f"one-term huygens {plan} {red}")


def test_huygens_diffraction_workload_sampled(cuda_lib):
    """512 x 512 points x 4096 sources; 1024 sampled points against the oracle."""
    w = workloads.diffraction()
    P, Q, A = to_dev(w.p, w.q, w.a)
    u = torch.view_as_real(api.huygens(P, Q, A, w.k)).cpu().numpy()
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, len(w.p[0]) - 1], rng.integers(0, len(w.p[0]), 1024)]))
    sub = tuple(v[idx] for v in w.p)
    want = oracle.huygens(sub, w.q, w.a, w.k).view(np.float32).reshape(-1, 2)
    assert_f32_parity(u[idx].reshape(-1), want.reshape(-1), "diffraction sample")


def test_huygens_autotune(cuda_lib):
    p, q, a, k = pins.huygens_case(m=20000, n=1500, seed=3)
    P, Q, A = to_dev(p, q, a)
    u = torch.empty(20000, dtype=torch.complex64, device="cuda")
    best = api.sincos_autotune_huygens(P, Q, A, k, u)
    assert api.sincos_plan_get("huygens", "f32", 20000) == best
    u.zero_()
    api.sincos_huygens(P, Q, A, k, u)
    torch.cuda.synchronize()
    want = oracle.huygens(p, q, a, k).view(np.float32)
    assert_f32_parity(torch.view_as_real(u).cpu().numpy().reshape(-1), want, "tuned huygens")
