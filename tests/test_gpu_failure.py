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
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    assert lib.sincos_selftest_wait_timeout(5000, stream) == 0     # gives up after 5 ms
    ev1.record()
    torch.cuda.synchronize()
    # the limit is wall-clock time: the wait lasted at least its 5 ms, and
    # ended long before the kernels' own 1 s limit
    assert 4.5 <= ev0.elapsed_time(ev1) < 500.0, ev0.elapsed_time(ev1)
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
