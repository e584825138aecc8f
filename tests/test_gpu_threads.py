"""Concurrent callers: host threads, each on its own stream and buffers,
calling the forward, the backward and the batched forward at the same time
(ctypes releases the GIL around every library call).  Every result must equal
the single-threaded one bit for bit."""
import threading

import numpy as np
import pytest
import torch

import oracle
from gpu_util import as_np, assert_f32_parity, mixed_angles
from paper_cs_0406049_gb300 import api

pytestmark = pytest.mark.gpu

THREADS = 8
ROUNDS = 15


def test_concurrent_calls_on_separate_streams(cuda_lib):
    n = (1 << 20) + 5
    x = mixed_angles(n, seed=31)
    want_s, want_c = oracle.sincos(x)
    rng = np.random.default_rng(31)
    gs = rng.standard_normal(n).astype(np.float32)
    gc = rng.standard_normal(n).astype(np.float32)
    want_gx = oracle.backward(gs, gc, want_s, want_c)
    lens = [1000, 0, 70001, 3, 8192, 100000]
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    errors = []

    def worker(k):
        try:
            dev = torch.device("cuda", 0)
            stream = torch.cuda.Stream(device=dev)
            with torch.cuda.device(dev), torch.cuda.stream(stream):
                xt = torch.from_numpy(x).to(dev)
                gst = torch.from_numpy(gs).to(dev)
                gct = torch.from_numpy(gc).to(dev)
                s = torch.empty_like(xt)
                c = torch.empty_like(xt)
                gx = torch.empty_like(xt)
                sb = torch.empty_like(xt)
                cb = torch.empty_like(xt)
                segs, lens_t = api.segments(xt, sb, cb, offs, lens)
                for _ in range(ROUNDS):
                    api.sincos_pairs(xt, s, c)
                    api.sincos_backward(gst, gct, s, c, gx)
                    api.sincos_batched(segs, lens_t)
                stream.synchronize()
                assert_f32_parity(as_np(s), want_s, f"thread {k} s")
                assert_f32_parity(as_np(c), want_c, f"thread {k} c")
                assert_f32_parity(as_np(gx), want_gx, f"thread {k} gx")
                m = int(sum(lens))
                assert_f32_parity(as_np(sb)[:m], want_s[:m], f"thread {k} batched s")
                assert_f32_parity(as_np(cb)[:m], want_c[:m], f"thread {k} batched c")
        except Exception as e:          # reported by the main thread
            errors.append(f"thread {k}: {e!r}")

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(THREADS)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in threads), "a worker did not finish"
    assert not errors, errors
    assert api.sincos_device_wait_timeouts() == 0
