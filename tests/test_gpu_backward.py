"""GPU backward (through torch.autograd and through the C ABI) against the
oracle, FP64 central finite differences and the analytic FP64 gradient."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import as_np, assert_f32_parity
from paper_cs_0406049_gb300 import api, workloads

pytestmark = pytest.mark.gpu


def test_autograd_differentiation_workload(cuda_lib):
    """2^26 angles U[-50, 50) (seed 4), gs, gc ~ N(0, 1): forward and backward
    through SinCosFn; every gradient element against the oracle."""
    w = workloads.differentiation_inputs()
    x = torch.from_numpy(w.x).cuda().requires_grad_(True)
    gs = torch.from_numpy(w.gs).cuda()
    gc = torch.from_numpy(w.gc).cuda()
    s, c = api.sincos_autograd(x)
    torch.autograd.backward([s, c], [gs, gc])
    torch.cuda.synchronize()
    so, co = oracle.sincos(w.x)
    assert_f32_parity(as_np(s), so, "forward s")
    assert_f32_parity(as_np(c), co, "forward c")
    want = oracle.backward(w.gs, w.gc, so, co)
    assert_f32_parity(as_np(x.grad), want, "gx")

    # FP64 checks on the first 4096 elements: central differences (h = 1e-3)
    # of L = gs sin x + gc cos x, and the analytic gs cos x - gc sin x.
    k = 4096
    xd = w.x[:k].astype(np.float64)
    gsd, gcd = w.gs[:k].astype(np.float64), w.gc[:k].astype(np.float64)
    gx = as_np(x.grad)[:k].astype(np.float64)
    h = 1e-3
    L = lambda t: gsd * np.sin(t) + gcd * np.cos(t)
    fd = (L(xd + h) - L(xd - h)) / (2 * h)
    scale = np.abs(gsd) + np.abs(gcd)
    assert np.all(np.abs(gx - fd) <= 1e-4 * scale)
    analytic = gsd * np.cos(xd) - gcd * np.sin(xd)
    assert np.all(np.abs(gx - analytic) <= 1e-4 * scale)


def test_one_output_used(cuda_lib):
    """Only s feeds the loss, so autograd passes no gc: gx = gs * c."""
    rng = np.random.default_rng(21)
    xn = rng.uniform(-50, 50, 300007).astype(np.float32)
    x = torch.from_numpy(xn).cuda().requires_grad_(True)
    s, c = api.sincos_autograd(x)
    (3.0 * s).sum().backward()
    so, co = oracle.sincos(xn)
    want = oracle.backward(np.full(xn.size, 3.0, np.float32), None, so, co)
    assert_f32_parity(as_np(x.grad), want, "gx (gs only)")

    x.grad = None
    s, c = api.sincos_autograd(x)
    (2.0 * c).sum().backward()
    want = oracle.backward(None, np.full(xn.size, 2.0, np.float32), so, co)
    assert_f32_parity(as_np(x.grad), want, "gx (gc only)")


@pytest.mark.parametrize("n", [1, 3, 4, 5, 17, 1023, 4097, 65537, (1 << 20) + 3])
@pytest.mark.parametrize("offset", [0, 1, 3])
def test_abi_backward_ragged(cuda_lib, n, offset):
    rng = np.random.default_rng(n + offset)
    xn = rng.uniform(-50, 50, n).astype(np.float32)
    gsn = rng.standard_normal(n).astype(np.float32)
    gcn = rng.standard_normal(n).astype(np.float32)
    so, co = oracle.sincos(xn)
    pad = lambda a, o: torch.from_numpy(np.concatenate([np.zeros(o, np.float32), a])).cuda()[o:]
    gs_t, gc_t = pad(gsn, offset), pad(gcn, offset)
    s_t, c_t = pad(so, offset), pad(co, (offset + 1) % 4)   # c misaligned differently
    gx = pad(np.zeros(n, np.float32), offset)
    for gs_use, gc_use in ((True, True), (True, False), (False, True), (False, False)):
        api.sincos_backward(gs_t if gs_use else None, gc_t if gc_use else None, s_t, c_t, gx)
        want = oracle.backward(gsn if gs_use else None, gcn if gc_use else None, so, co)
        assert_f32_parity(as_np(gx), want, f"gx n={n} gs={gs_use} gc={gc_use}")


def test_backward_in_place(cuda_lib):
    rng = np.random.default_rng(3)
    n = 100001
    xn = rng.uniform(-5, 5, n).astype(np.float32)
    gsn = rng.standard_normal(n).astype(np.float32)
    gcn = rng.standard_normal(n).astype(np.float32)
    so, co = oracle.sincos(xn)
    want = oracle.backward(gsn, gcn, so, co)
    gs_t = torch.from_numpy(gsn).cuda()
    api.sincos_backward(gs_t, torch.from_numpy(gcn).cuda(), torch.from_numpy(so).cuda(),
                        torch.from_numpy(co).cuda(), gs_t)
    assert_f32_parity(as_np(gs_t), want, "in-place gx")


def test_second_derivative_is_refused(cuda_lib):
    """The hand-written backward is differentiable once: asking for a second
    derivative raises instead of silently returning zero."""
    x = torch.linspace(-3.0, 3.0, 1000, device="cuda").requires_grad_(True)
    s, c = api.sincos_autograd(x)
    (gx,) = torch.autograd.grad(s.sum() + 2.0 * c.sum(), x, create_graph=True)
    with pytest.raises(RuntimeError):
        torch.autograd.grad(gx.sum(), x)
