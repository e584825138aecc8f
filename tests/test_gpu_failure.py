"""The bulk kernels' bounded waits: a wait that runs out is counted and the
device stays usable (no fault, trap or hang is provoked)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import as_np, assert_f32_parity, mixed_angles
from paper_cs_0406049_gb300 import api

pytestmark = pytest.mark.gpu


def test_wait_that_runs_out_is_reported(cuda_lib):
    lib = api.lib()
    assert api.sincos_device_wait_timeouts() == 0          # nothing pending
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.sincos_selftest_wait_timeout(4096, stream) == 0
    torch.cuda.synchronize()
    assert api.sincos_device_wait_timeouts() == 1
    assert api.sincos_device_wait_timeouts() == 0          # reading clears
    # the context is still usable: a bulk-path forward right after is exact
    x = mixed_angles((1 << 20) + 3, seed=17)
    xt = torch.from_numpy(x).cuda()
    s, c = api.sincos(xt)
    ws, wc = oracle.sincos(x)
    assert_f32_parity(as_np(s), ws, "after timeout s")
    assert_f32_parity(as_np(c), wc, "after timeout c")
    assert api.sincos_device_wait_timeouts() == 0
