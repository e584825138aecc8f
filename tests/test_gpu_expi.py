"""exp(i x) as interleaved complex64 against the oracle's (cos, sin) pairs."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import as_np, assert_f32_parity, forced_plan, mixed_angles
from paper_cs_0406049_gb300 import api

pytestmark = pytest.mark.gpu

PATHS = {"bulk256": (256, 2, 1, 0), "bulk512": (512, 2, 1, 0), "reg16": (256, 8, 4, 16),
         "reg32": (256, 4, 4, 32)}
SIZES = [1, 3, 4, 5, 31, 33, 1023, 8191, 8192, 8193, 8192 * 3 + 37, 152 * 8192 + 4099,
         (1 << 20) + 5]
GUARD = 64
SENT = np.uint32(0x7fa5a5a5)


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("red,coef", [("plain", "normalized"), ("compensated", "dagger")])
def test_expi_ragged(cuda_lib, path, red, coef):
    with forced_plan("expi", "f32", PATHS[path]):
        for n in SIZES:
            x = mixed_angles(n, seed=n)
            ws, wc = oracle.sincos(x, reduction=red, coef=coef)
            want = np.empty(2 * n, np.float32)
            want[0::2], want[1::2] = wc, ws
            for ox, oz in ((0, 0), (1, 2), (3, 6), (2, 1), (1, 0)):
                xb = torch.zeros(n + 8, device="cuda")
                xb[ox:ox + n] = torch.from_numpy(x).cuda()
                fill = int(SENT.view(np.int32))
                zb = torch.full((2 * n + 2 * GUARD,), fill, dtype=torch.int32,
                                device="cuda").view(torch.float32)
                z = zb[GUARD + oz:GUARD + oz + 2 * n]
                api.sincos_expi(xb[ox:ox + n], z, red, coef)
                torch.cuda.synchronize()
                raw = as_np(zb).view(np.uint32)
                assert np.all(raw[:GUARD + oz] == SENT) and np.all(raw[GUARD + oz + 2 * n:] == SENT)
                assert_f32_parity(as_np(z), want, f"expi {path} {red} n={n} offs={ox},{oz}")
    assert api.sincos_device_wait_timeouts() == 0


def test_expi_autotune(cuda_lib):
    n = (1 << 22) + 3
    x = mixed_angles(n, seed=8)
    xt = torch.from_numpy(x).cuda()
    z = torch.empty(n, dtype=torch.complex64, device="cuda")
    best = api.sincos_autotune_expi(xt, z)
    assert api.sincos_plan_get("expi", "f32", n) == best
    z.zero_()
    api.sincos_expi(xt, z)
    ws, wc = oracle.sincos(x)
    zr = torch.view_as_real(z).cpu().numpy().reshape(-1)
    assert_f32_parity(zr[0::2], wc, "tuned expi c")
    assert_f32_parity(zr[1::2], ws, "tuned expi s")


def test_expi_complex_tensor(cuda_lib):
    x = torch.from_numpy(mixed_angles(100000, seed=3)).cuda()
    z = api.expi(x)
    assert z.dtype == torch.complex64 and z.shape == x.shape
    s, c = api.sincos(x)
    assert torch.equal(z.real.contiguous().view(torch.int32), c.view(torch.int32))
    assert torch.equal(z.imag.contiguous().view(torch.int32), s.view(torch.int32))
