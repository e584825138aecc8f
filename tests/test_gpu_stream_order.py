"""Stream order between consecutive launches of the bulk kernels, which run
with programmatic dependent launch: a launch may start while the previous one
drains, and must still see every write of the kernels before it and must not
overwrite what they still read.  Chains of dependent calls are enqueued with
no synchronization between them and checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import as_np, assert_f32_parity, mixed_angles
from paper_cs_0406049_gb300 import api

pytestmark = pytest.mark.gpu

N = (1 << 22) + 7          # many bulk chunks per CTA and a ragged tail


def test_read_after_write_chain(cuda_lib):
    """Each call reads the sines the previous call wrote (s_i -> x_{i+1})."""
    x = mixed_angles(N, seed=41)
    bufs = [torch.from_numpy(x).cuda()] + [torch.empty(N, device="cuda") for _ in range(6)]
    cs = [torch.empty(N, device="cuda") for _ in range(6)]
    for i in range(6):
        api.sincos_pairs(bufs[i], bufs[i + 1], cs[i])
    torch.cuda.synchronize()
    want = x
    for i in range(6):
        ws, wc = oracle.sincos(want)
        assert_f32_parity(as_np(bufs[i + 1]), ws, f"chain step {i} s")
        assert_f32_parity(as_np(cs[i]), wc, f"chain step {i} c")
        want = ws


def test_write_after_read(cuda_lib):
    """A call that overwrites the previous call's input must not change what
    that call read: call 1 reads x, call 2 writes its sines into x."""
    x = mixed_angles(N, seed=42)
    z = mixed_angles(N, seed=43)
    xt = torch.from_numpy(x).cuda()
    zt = torch.from_numpy(z).cuda()
    s1, c1, c2 = (torch.empty(N, device="cuda") for _ in range(3))
    for _ in range(3):
        xt.copy_(torch.from_numpy(x))
        api.sincos_pairs(xt, s1, c1)          # reads x
        api.sincos_pairs(zt, xt, c2)          # writes x
        torch.cuda.synchronize()
        ws, wc = oracle.sincos(x)
        assert_f32_parity(as_np(s1), ws, "first call s")
        assert_f32_parity(as_np(c1), wc, "first call c")
        zs, zc = oracle.sincos(z)
        assert_f32_parity(as_np(xt), zs, "second call s")


def test_exp_ix_after_forward(cuda_lib):
    """exp(ix) of the sines the forward kernel wrote just before, and a
    forward of the real parts exp(ix) wrote, without synchronization."""
    x = mixed_angles(N, seed=44)
    xt = torch.from_numpy(x).cuda()
    s, c = torch.empty(N, device="cuda"), torch.empty(N, device="cuda")
    z = torch.empty(N, dtype=torch.complex64, device="cuda")
    re = torch.empty(N, device="cuda")
    s2, c2 = torch.empty(N, device="cuda"), torch.empty(N, device="cuda")
    api.sincos_pairs(xt, s, c)
    api.sincos_expi(s, z)
    re.copy_(torch.view_as_real(z)[:, 0])
    api.sincos_pairs(re, s2, c2)
    torch.cuda.synchronize()
    ws, wc = oracle.sincos(x)
    zs, zc = oracle.sincos(ws)
    zr = torch.view_as_real(z).cpu().numpy()
    assert_f32_parity(zr[:, 0].copy(), zc, "exp(ix) real")
    assert_f32_parity(zr[:, 1].copy(), zs, "exp(ix) imag")
    ts, tc = oracle.sincos(zc)
    assert_f32_parity(as_np(s2), ts, "third call s")
    assert_f32_parity(as_np(c2), tc, "third call c")
    assert api.sincos_device_wait_timeouts() == 0


def test_dependent_chain_in_a_cuda_graph(cuda_lib):
    """The read-after-write chain captured into a CUDA graph (the bulk
    launches become programmatic dependencies of the graph) and replayed
    twice with new angles copied in between."""
    x = mixed_angles(N, seed=45)
    x2 = mixed_angles(N, seed=46)
    src = torch.from_numpy(x).cuda()
    bufs = [torch.empty(N, device="cuda") for _ in range(4)]
    cs = [torch.empty(N, device="cuda") for _ in range(3)]
    bufs[0].copy_(src)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for i in range(3):                     # warm-up outside the capture
            api.sincos_pairs(bufs[i], bufs[i + 1], cs[i])
        side.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            for i in range(3):
                api.sincos_pairs(bufs[i], bufs[i + 1], cs[i])
    torch.cuda.synchronize()
    for angles in (x, x2):
        bufs[0].copy_(torch.from_numpy(angles))
        g.replay()
        torch.cuda.synchronize()
        want = angles
        for i in range(3):
            ws, wc = oracle.sincos(want)
            assert_f32_parity(as_np(bufs[i + 1]), ws, f"graph chain step {i} s")
            assert_f32_parity(as_np(cs[i]), wc, f"graph chain step {i} c")
            want = ws
