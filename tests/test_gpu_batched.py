"""Batched forward (one prefix + persistent launch, and its CUDA graph)
against the oracle applied to each array."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import as_np, assert_16_parity, assert_f32_parity, forced_plan, mixed_angles
from paper_cs_0406049_gb300 import api, workloads

pytestmark = pytest.mark.gpu

DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def packed(lens, dtype, seed=0):
    """Segments packed back to back in one buffer (most start unaligned)."""
    lens = np.asarray(lens, np.int64)
    total = int(np.clip(lens, 0, None).sum())
    x = mixed_angles(max(total, 1), seed)[:total]
    offs = np.concatenate([[0], np.cumsum(np.clip(lens, 0, None))[:-1]]).astype(np.int64)
    xt = torch.from_numpy(x).cuda() if total else torch.empty(0, device="cuda")
    s = torch.full((max(total, 1),), 7.0, device="cuda").to(DT[dtype])[:total]
    c = torch.full((max(total, 1),), 7.0, device="cuda").to(DT[dtype])[:total]
    return x, xt, s, c, offs


def check_all(x, s, c, dtype, red, coef, what):
    want_s, want_c = oracle.sincos(x, reduction=red, coef=coef, out=dtype)
    if dtype == "f32":
        assert_f32_parity(as_np(s), want_s, what + " s")
        assert_f32_parity(as_np(c), want_c, what + " c")
    else:
        assert_16_parity(as_np(s), want_s, dtype == "bf16", what + " s")
        assert_16_parity(as_np(c), want_c, dtype == "bf16", what + " c")


EDGE_LENS = [1, 0, 3, 4095, 4096, 4097, 8191, 8192, 8193, 2, 65536 + 17, 5, 0, 0, 1, 1 << 20,
             31, 7, 8, 3 * 8192 + 63, 64, 65]
PATHS = {"bulk256": (256, 2, 1, 0), "bulk1024": (1024, 2, 1, 0), "bulksmall": (256, 2, 3, 0),
         "reg16": (1024, 2, 1, 16), "reg32": (256, 4, 8, 32)}


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("red,coef", [("plain", "normalized"), ("compensated", "dagger")])
def test_edge_lengths(cuda_lib, dtype, red, coef, path):
    x, xt, s, c, offs = packed(EDGE_LENS, dtype, seed=1)
    segs, lens = api.segments(xt, s, c, offs, EDGE_LENS)
    with forced_plan("batched", dtype, PATHS[path]):
        api.sincos_batched(segs, lens, dtype, red, coef)
    check_all(x, s, c, dtype, red, coef, f"batched {path} {dtype}")
    assert api.sincos_device_wait_timeouts() == 0
    assert api.sincos_device_bad_segments() == 0


@pytest.mark.parametrize("path", sorted(PATHS))
def test_all_lengths_empty(cuda_lib, path):
    """No elements at all: every CTA's run is empty and nothing is written."""
    lens = [0, -4, 0, -1]
    x = mixed_angles(64, 3)
    xt = torch.from_numpy(x).cuda()
    s = torch.full_like(xt, 7.0)
    c = torch.full_like(xt, 7.0)
    segs, lens_t = api.segments(xt, s, c, [0, 8, 16, 24], lens)
    with forced_plan("batched", "f32", PATHS[path]):
        api.sincos_batched(segs, lens_t)
    torch.cuda.synchronize()
    assert torch.all(s == 7.0) and torch.all(c == 7.0)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_one_long_segment_then_short_ones(cuda_lib, path):
    """Most CTA boundaries fall inside the first segment (at its head, inside
    tiles, at its end); the short segments after it share the last runs."""
    lens = [3 * (1 << 20) + 13] + [1, 0, 5, 33, 4097, 2, 0, 9000, 1, 1]
    x, xt, s, c, offs = packed(lens, "f32", seed=4)
    segs, lens_t = api.segments(xt, s, c, offs, lens)
    with forced_plan("batched", "f32", PATHS[path]):
        api.sincos_batched(segs, lens_t)
    check_all(x, s, c, "f32", "plain", "normalized", f"long then short {path}")


@pytest.mark.parametrize("path", sorted(PATHS))
def test_negative_and_empty_lengths(cuda_lib, path):
    lens = [5, -3, 0, 9, -100, 1, 20000, -1]
    x, xt, s, c, offs = packed(lens, "f32", seed=2)
    segs, lens_t = api.segments(xt, s, c, offs, lens)
    with forced_plan("batched", "f32", PATHS[path]):
        api.sincos_batched(segs, lens_t)
    check_all(x, s, c, "f32", "plain", "normalized", "negative lengths")


@pytest.mark.parametrize("path", sorted(PATHS))
def test_separate_tensors_mixed_alignment(cuda_lib, path):
    """Segments as separate tensors whose x, s and c start at different
    offsets modulo 16 bytes (the element-wise path inside tiles)."""
    rng = np.random.default_rng(4)
    xs, ss, cs, xn = [], [], [], []
    keep = []
    for i in range(40):
        n = int(rng.integers(1, 20000))
        a = mixed_angles(n, seed=100 + i)
        bx = torch.zeros(n + 4, device="cuda")
        bs = torch.zeros(n + 4, device="cuda")
        bc = torch.zeros(n + 4, device="cuda")
        ox, os_, oc = (int(v) for v in rng.integers(0, 4, 3))
        bx[ox:ox + n] = torch.from_numpy(a).cuda()
        xs.append(bx[ox:ox + n]); ss.append(bs[os_:os_ + n]); cs.append(bc[oc:oc + n])
        xn.append(a)
        keep += [bx, bs, bc]
    segs, lens = api.segments_from_lists(xs, ss, cs)
    with forced_plan("batched", "f32", PATHS[path]):
        api.sincos_batched(segs, lens)
    torch.cuda.synchronize()
    for i, a in enumerate(xn):
        want_s, want_c = oracle.sincos(a)
        assert_f32_parity(as_np(ss[i]), want_s, f"seg {i} s")
        assert_f32_parity(as_np(cs[i]), want_c, f"seg {i} c")


# kernels per batched call: the ring kernel alone, or the schedule kernel and
# the tile kernel of a register plan
GRAPH_CASES = {"default": (None, 1), "bulk256": (PATHS["bulk256"], 1),
               "reg16": (PATHS["reg16"], 2), "reg32": (PATHS["reg32"], 2)}


@pytest.mark.parametrize("case", sorted(GRAPH_CASES))
def test_graph_replay_bit_identical(cuda_lib, case):
    """The graph's results equal the oracle's on the first replay and the
    first replay's bits on the second; creating the graph leaves the launch
    counter where it was, and each replay adds the kernels the graph holds."""
    plan, kernels = GRAPH_CASES[case]
    lens = EDGE_LENS * 3
    if plan is None:       # whatever plan the library holds for this count now
        kernels = 1 if api.sincos_plan_get("batched", "f32", len(lens))["vec_bytes"] == 0 else 2
    x, xt, s, c, offs = packed(lens, "f32", seed=3)
    segs, lens_t = api.segments(xt, s, c, offs, lens)
    ctx = forced_plan("batched", "f32", plan) if plan else None
    if ctx:
        ctx.__enter__()
    try:
        before = api.sincos_launch_count()
        g = api.BatchedGraph(segs, lens_t)
        assert api.sincos_launch_count() == before, "capturing counted launches"
    finally:
        if ctx:
            ctx.__exit__(None, None, None)
    with g:
        g.launch()
        torch.cuda.synchronize()
        check_all(x, s, c, "f32", "plain", "normalized", f"graph replay 1 ({case})")
        first_s, first_c = as_np(s).copy(), as_np(c).copy()
        s.fill_(0)
        c.fill_(0)
        before = api.sincos_launch_count()
        g.launch()
        torch.cuda.synchronize()
        assert api.sincos_launch_count() == before + kernels
        assert np.array_equal(as_np(s).view(np.uint32), first_s.view(np.uint32))
        assert np.array_equal(as_np(c).view(np.uint32), first_c.view(np.uint32))


def test_batching_workload_full_size(cuda_lib):
    """4096 arrays, lengths log-uniform in [1, 2^20] (seed 3), packed back to
    back: the persistent launch, its graph replay and 4096 single-array
    launches agree bit for bit; the oracle checks the first and last 64 and
    64 random elements of every array."""
    b = workloads.batching()
    xt = torch.from_numpy(b.angles).cuda()
    s = torch.empty_like(xt)
    c = torch.empty_like(xt)
    segs, lens = api.segments(xt, s, c, b.offsets, b.lens)
    api.sincos_batched(segs, lens)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    idx = []
    for off, n in zip(b.offsets, b.lens):
        k = min(int(n), 64)
        idx.append(off + np.arange(k))
        idx.append(off + n - k + np.arange(k))
        idx.append(off + rng.integers(0, n, 64))
    idx = np.unique(np.concatenate(idx))
    it = torch.from_numpy(idx).cuda()
    want_s, want_c = oracle.sincos(b.angles[idx])
    assert_f32_parity(as_np(s[it]), want_s, "batched s")
    assert_f32_parity(as_np(c[it]), want_c, "batched c")

    s2 = torch.empty_like(xt)
    c2 = torch.empty_like(xt)
    segs2, _ = api.segments(xt, s2, c2, b.offsets, b.lens)
    with api.BatchedGraph(segs2, lens) as g:
        g.launch()
    torch.cuda.synchronize()
    assert torch.equal(s.view(torch.int32), s2.view(torch.int32))
    assert torch.equal(c.view(torch.int32), c2.view(torch.int32))

    s3 = torch.empty_like(xt)
    c3 = torch.empty_like(xt)
    for off, n in zip(b.offsets.tolist(), b.lens.tolist()):
        api.sincos_pairs(xt[off:off + n], s3[off:off + n], c3[off:off + n])
    torch.cuda.synchronize()
    assert torch.equal(s.view(torch.int32), s3.view(torch.int32))
    assert torch.equal(c.view(torch.int32), c3.view(torch.int32))


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_gaps_between_arrays_stay_untouched(cuda_lib, path, dtype):
    """Arrays placed in one buffer with sentinel-filled gaps of 1-40 elements
    between them (and 64 before and after): every gap element is unchanged
    after the call, every array element matches the oracle."""
    rng = np.random.default_rng(21)
    lens = [int(v) for v in rng.choice([1, 3, 7, 31, 100, 4097, 8191, 8192, 8195, 20000, 70001],
                                       200)]
    gaps = rng.integers(1, 41, len(lens))
    offs, pos = [], 64
    for n, g in zip(lens, gaps):
        offs.append(pos)
        pos += n + int(g)
    total = pos + 64
    x = mixed_angles(total, 8)
    xt = torch.from_numpy(x).cuda()
    if dtype == "f32":
        fill = torch.tensor(np.array([0x7fa5a5a5], np.uint32).view(np.int32)[0]).item()
        s = torch.full((total,), fill, dtype=torch.int32, device="cuda").view(torch.float32)
        c = s.clone()
        sent = np.uint32(0x7fa5a5a5)
    else:
        s = torch.full((total,), 0x7da5, dtype=torch.int16, device="cuda").view(torch.bfloat16)
        c = s.clone()
        sent = np.uint16(0x7da5)
    segs, lens_t = api.segments(xt, s, c, offs, lens)
    with forced_plan("batched", dtype, PATHS[path]):
        api.sincos_batched(segs, lens_t, dtype)
    torch.cuda.synchronize()
    inside = np.zeros(total, bool)
    for o, n in zip(offs, lens):
        inside[o:o + n] = True
    for name, t in (("s", s), ("c", c)):
        raw = as_np(t)
        raw = raw.view(np.uint32) if dtype == "f32" else raw
        assert np.all(raw[~inside] == sent), f"{path} {dtype}: {name} written outside the arrays"
    xs = np.concatenate([x[o:o + n] for o, n in zip(offs, lens)])
    sel = np.concatenate([np.arange(o, o + n) for o, n in zip(offs, lens)])
    check_all(xs, s[torch.from_numpy(sel).cuda()], c[torch.from_numpy(sel).cuda()], dtype,
              "plain", "normalized", f"gaps {path} {dtype}")


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("count", [5000, 20000, 65536])
def test_many_arrays(cuda_lib, path, count):
    """More arrays than the ring kernel's threads hold in one batch of
    metadata each (its prologue then reloads them for the second pass), with
    empty arrays, short ones and a few long ones, against the oracle."""
    rng = np.random.default_rng(count)
    lens = rng.integers(0, 40, count)
    lens[rng.integers(0, count, 12)] = rng.integers(8000, 60000, 12)
    lens[::53] = 0
    x, xt, s, c, offs = packed(lens, "f32", seed=5)
    segs, lens_t = api.segments(xt, s, c, offs, lens)
    with forced_plan("batched", "f32", PATHS[path]):
        api.sincos_batched(segs, lens_t)
    check_all(x, s, c, "f32", "plain", "normalized", f"{count} arrays {path}")
    assert api.sincos_device_wait_timeouts() == 0


def test_ring_plan_captures_without_a_prior_call(cuda_lib):
    """The ring kernel needs no scratch, so a binary32 batch can be captured
    into a CUDA graph on a stream the library has never seen, and the replay
    matches the oracle."""
    lens = [3, 8192, 0, 70001, 5, 4097]
    x, xt, s, c, offs = packed(lens, "f32", seed=9)
    segs, lens_t = api.segments(xt, s, c, offs, lens)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with forced_plan("batched", "f32", PATHS["bulk256"]):
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                api.sincos_batched(segs, lens_t)
        torch.cuda.current_stream().wait_stream(side)
        s.fill_(0)
        c.fill_(0)
        graph.replay()
    torch.cuda.synchronize()
    check_all(x, s, c, "f32", "plain", "normalized", "captured ring batch")


@pytest.mark.parametrize("path", sorted(PATHS))
def test_null_pointers_on_empty_arrays(cuda_lib, path):
    """Arrays of length <= 0 may carry null pointers (they are never used):
    the other arrays are exact and nothing is counted as skipped.  Only valid
    descriptors are launched here; the skip of invalid ones is checked on the
    host (the same predicate, tests/test_abi_cpu.py)."""
    lens = [5000, 0, 17, -3, 8193, 0]
    x, xt, s, c, offs = packed(lens, "f32", seed=6)
    segs, lens_t = api.segments(xt, s, c, offs, lens)
    segs = segs.view(-1, 3).clone()
    for i, n in enumerate(lens):
        if n <= 0:
            segs[i] = 0
    assert api.sincos_device_bad_segments() == 0
    with forced_plan("batched", "f32", PATHS[path]):
        api.sincos_batched(segs.view(-1), lens_t)
    check_all(x, s, c, "f32", "plain", "normalized", f"null empties {path}")
    assert api.sincos_device_bad_segments() == 0


def test_plan_change_takes_effect_on_the_next_call(cuda_lib):
    """A plan set between two calls of the same kind is used by the second
    (the library keeps each thread's last plan lookup until a plan changes):
    a register plan launches two kernels, the ring plan one."""
    lens = [7000, 3, 9000, 0, 12]
    x, xt, s, c, offs = packed(lens, "f32", seed=8)
    segs, lens_t = api.segments(xt, s, c, offs, lens)
    for plan, kernels in ((PATHS["reg16"], 2), (PATHS["bulksmall"], 1), (PATHS["reg32"], 2),
                          (PATHS["bulk256"], 1)):
        with forced_plan("batched", "f32", plan):
            before = api.sincos_launch_count()
            api.sincos_batched(segs, lens_t)
            torch.cuda.synchronize()
            assert api.sincos_launch_count() - before == kernels, plan
        check_all(x, s, c, "f32", "plain", "normalized", f"plan {plan}")
