"""bench.py's host logic on CPU: multi-rank timing over gloo (world size 2)
and the reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(world)
    d.init("gloo")
    elapsed = 10.0 * (rank + 1)          # rank 1 is the slow one
    m = d.max(elapsed)
    d.barrier()
    q.put((rank, m, bench.aggregate_value(d.world, 1 << 28, 20, m)))
    d.close()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [m for _, m, _ in out] == [20.0, 20.0]
    # whole-job throughput: both ranks' pairs over the slowest rank's time
    assert out[0][2] == pytest.approx(2 * (1 << 28) * 20 / 20e-3)


def _shard_worker(rank, world, port, n, q):
    """One rank of the split (strong-scaling) data plane on the CPU: the
    oracle stands in for the kernel on this rank's block of one seeded array;
    the blocks travel to rank 0 only for the check (the product path has no
    collective on the data)."""
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    import torch.distributed as dist

    import bench
    import oracle
    from paper_cs_0406049_gb300 import workloads
    d = bench.Dist(world)
    d.init("gloo")
    x = workloads.angles_uniform(n, -1000.0, 1000.0, seed=1)
    lo, hi = bench.shard_bounds(n, d.rank, d.world)
    s, c = oracle.sincos(x[lo:hi])
    got = [None] * world
    dist.all_gather_object(got, (d.rank, lo, hi, s.view(np.uint32).tobytes(),
                                 c.view(np.uint32).tobytes()))
    if d.rank == 0:
        got.sort()
        assert got[0][1] == 0 and got[-1][2] == n
        for a, b in zip(got, got[1:]):
            assert a[2] == b[1], "blocks leave a gap or overlap"
        assert max(h - l for _, l, h, _, _ in got) - min(h - l for _, l, h, _, _ in got) <= 1
        ws, wc = oracle.sincos(x)
        s_all = np.frombuffer(b"".join(g[3] for g in got), np.uint32)
        c_all = np.frombuffer(b"".join(g[4] for g in got), np.uint32)
        assert np.array_equal(s_all, ws.view(np.uint32))
        assert np.array_equal(c_all, wc.view(np.uint32))
    d.barrier()
    q.put(rank)
    d.close()


@pytest.mark.parametrize("world", [2, 3])
def test_split_data_plane_over_ranks(world):
    """bench.py --split cuts one array into contiguous per-rank blocks; over
    gloo ranks on the CPU the blocks tile the array, differ in size by at most
    one, and the per-rank results put together are the oracle's for the
    whole array, bit for bit (n = 1000003, so the blocks are ragged)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, 1000003, q))
             for r in range(world)]
    for p in procs:
        p.start()
    done = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert done == list(range(world))


def test_shard_bounds_tile_the_array():
    sys.path.insert(0, ROOT)
    import bench
    for n in (0, 1, 5, 1 << 28, (1 << 28) + 7):
        for world in (1, 2, 3, 4, 8):
            b = [bench.shard_bounds(n, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            sizes = [h - l for l, h in b]
            assert max(sizes) - min(sizes) <= 1


def test_reference_arm_on_other_ranks_does_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "pairs/s" and line["value"] > 0
    assert line["config"]["workload"] == "bandwidth_2p28"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_accuracy_statistics_of_known_errors():
    """The Euclidean and amplitude errors of results with planted errors: an
    exact pair gives zeros; s off by 3e-7 and c off by 4e-7 at x = 0 (s = 0,
    c = 1) give a Euclidean error of 5e-7 and an amplitude error of 4e-7."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    x = np.zeros(4, np.float32)
    st = bench.e1_stats(x, np.zeros(4), np.ones(4))
    assert st["rms_euclid"] == 0.0 and st["max_euclid"] == 0.0 and st["max_amplitude"] == 0.0
    assert st["max_euclid_reduced_angle"] == 0.0          # fl(0 * K) = 0
    s = np.array([0.0, 3e-7, 0.0, 0.0])
    c = np.array([1.0, 1.0 + 4e-7, 1.0, 1.0])
    st = bench.e1_stats(x, s, c)
    assert abs(st["max_euclid"] - 5e-7) < 1e-15
    assert abs(st["rms_euclid"] - 2.5e-7) < 1e-15          # sqrt(25e-14 / 4)
    assert abs(st["max_amplitude"] - 4e-7) < 1e-13         # hypot(3e-7, 1 + 4e-7) - 1
    # x = 1: the reduced angle 2 pi fl(K) differs from 1 by the rounding of K
    k32 = float(np.float32(1.0 / (2.0 * 3.1415926536)))
    a = 2 * np.pi * k32
    st = bench.e1_stats(np.ones(1, np.float32), np.array([np.sin(a)]), np.array([np.cos(a)]))
    assert st["max_euclid_reduced_angle"] == 0.0
    assert abs(st["max_euclid"] - abs(2 * np.sin((a - 1.0) / 2))) < 1e-16   # chord of a - 1


def test_cpulist_parsing():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()


def test_error_helpers_on_rounded_exact_values():
    """The bench's FP64 error statements: correctly rounded binary32 values
    of the exact results come out within half an ulp (and a planted error
    of one ulp of 1.0 comes out as one)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    rng = np.random.default_rng(5)
    x = rng.uniform(-50, 50, 1 << 16).astype(np.float32)
    xd = x.astype(np.float64)
    s = np.sin(xd).astype(np.float32).astype(np.float64)
    c = np.cos(xd).astype(np.float32).astype(np.float64)
    e = bench.fp64_errors(x, s, c)
    assert e["max_abs"] <= 2.0 ** -25 and e["max_abs_ulp1"] <= 0.5
    assert e["max_ulp_rel_ge_2m4"] <= 0.5 + 1e-9 and e["sample"] == x.size
    s_bad = s.copy()
    s_bad[7] += 2.0 ** -23
    assert bench.fp64_errors(x, s_bad, c)["max_abs_ulp1"] >= 0.75   # 1 ulp(1) less a rounding
    gs = rng.standard_normal(x.size).astype(np.float32)
    gc = rng.standard_normal(x.size).astype(np.float32)
    gx = (gs.astype(np.float64) * np.cos(xd) - gc.astype(np.float64) * np.sin(xd)).astype(np.float32)
    b = bench.backward_fp64_errors(x, gs, gc, gx)
    assert b["max_rel_to_abs_gs_plus_abs_gc"] <= 2.0 ** -24


def test_huygens_error_helper_and_batch_sample():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench

    class W:
        pass
    rng = np.random.default_rng(6)
    w = W()
    w.p = tuple(rng.uniform(-5, 5, 40).astype(np.float32) for _ in range(2)) + \
        (np.full(40, 30.0, np.float32),)
    w.q = tuple(rng.uniform(-2, 2, 25).astype(np.float32) for _ in range(3))
    w.a = (rng.standard_normal(25) + 1j * rng.standard_normal(25)).astype(np.complex64)
    w.k = float(np.float32(2 * np.pi))
    p = [v.astype(np.float64) for v in w.p]
    q = [v.astype(np.float64) for v in w.q]
    r = np.sqrt(sum((p[d][:, None] - q[d][None, :]) ** 2 for d in range(3)))
    exact = (w.a.astype(np.complex128)[None, :] * np.exp(1j * w.k * r) / r).sum(axis=1)
    u = np.stack([exact.real, exact.imag], axis=1).astype(np.float32)
    pts = np.arange(0, 40, 3)
    h = bench.huygens_fp64_errors(w, u, pts)
    assert h["sample"] == pts.size and h["max_rel_to_sum_abs_terms"] <= 2.0 ** -23
    offs, lens = np.array([0, 10, 500, 501]), np.array([10, 490, 1, 300])
    idx = bench.batch_sample(offs, lens)
    assert np.all(np.diff(idx) > 0) and idx.min() == 0 and idx.max() == 800
    for o, n in zip(offs, lens):
        k = min(n, 64)
        assert np.isin(np.arange(o, o + k), idx).all()
        assert np.isin(np.arange(o + n - k, o + n), idx).all()


def test_kernel_hash_ignores_comments_only():
    sys.path.insert(0, ROOT)
    import bench
    a = "int f(int x) { return x + 1; }  // one\n/* two\n three */\n"
    b = "// another comment\nint f(int x) { return x + 1; }\n\n"
    c = "int f(int x) { return x + 2; }\n"
    assert bench.code_only(a) == bench.code_only(b) != bench.code_only(c)
    assert bench.code_only('const char *s = "// not a comment";') == 'const char *s = "// not a comment";'
