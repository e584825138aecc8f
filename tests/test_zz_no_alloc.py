"""The allocation-free batched entry point, through the C ABI.

`sincos_batched_noalloc` serves callers that may not allocate device memory
(a plug-in whose host program owns all GPU memory, a real-time thread that
cannot afford the device synchronization cudaMalloc may cause, code with a
memory budget fixed at start-up).  Its scratch is a fixed array inside the
library.  These checks compare it with `sincos_batched` on two calls in a
row, the second smaller than the first, so stale scratch contents from the
first call would show up in the second.  The file is named to be collected
last.
"""
import numpy as np
import pytest
import torch

from gpu_util import as_np, assert_f32_parity, mixed_angles
from paper_cs_0406049_gb300 import _lib, api

pytestmark = pytest.mark.gpu


def _packed(lens, seed):
    lens = np.asarray(lens, np.int64)
    total = int(np.clip(lens, 0, None).sum())
    x = torch.from_numpy(mixed_angles(total, seed)).cuda()
    offs = np.concatenate([[0], np.cumsum(np.clip(lens, 0, None))[:-1]]).astype(np.int64)
    return x, offs, lens


def _run_both(lib, lens, seed):
    x, offs, lens = _packed(lens, seed)
    s_ref, c_ref = torch.empty_like(x), torch.empty_like(x)
    s_new, c_new = torch.full_like(x, 9.0), torch.full_like(x, 9.0)
    segs_ref, lens_t = api.segments(x, s_ref, c_ref, offs, lens)
    segs_new, _ = api.segments(x, s_new, c_new, offs, lens)
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.sincos_batched_ex(segs_ref.data_ptr(), lens_t.data_ptr(), lens.size, _lib.F32,
                                 _lib.RED_PLAIN, _lib.COEF_NORMALIZED, stream) == _lib.OK
    assert lib.sincos_batched_noalloc(segs_new.data_ptr(), lens_t.data_ptr(), lens.size, _lib.F32,
                                      _lib.RED_PLAIN, _lib.COEF_NORMALIZED, stream) == _lib.OK
    torch.cuda.synchronize()
    # NaN where the existing entry point has NaN (NaN and infinite angles are
    # among the inputs), elsewhere within 2.4e-7 and bit-identical
    assert_f32_parity(as_np(s_new), as_np(s_ref), "no-alloc s")
    assert_f32_parity(as_np(c_new), as_np(c_ref), "no-alloc c")


def test_noalloc_matches_batched_on_two_calls(cuda_lib):
    lib = cuda_lib
    rng = np.random.default_rng(77)
    first = rng.integers(1, 70000, 3000)
    first[::97] = 0
    _run_both(lib, first, seed=1)
    second = rng.integers(1, 5000, 41)
    _run_both(lib, second, seed=2)


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
    assert lib.sincos_batched_noalloc(None, None, 0, _lib.F32, _lib.RED_PLAIN,
                                      _lib.COEF_NORMALIZED, stream) == _lib.OK
    assert lib.sincos_launch_count() == before


def test_noalloc_at_the_maximum_count(cuda_lib):
    """Exactly SINCOS_NOALLOC_MAX_SEGMENTS arrays of 1..7 angles each."""
    lens = (np.arange(_lib.NOALLOC_MAX_SEGMENTS) % 7 + 1).astype(np.int64)
    _run_both(cuda_lib, lens, seed=3)
