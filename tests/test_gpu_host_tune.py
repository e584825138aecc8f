"""Host-buffer path, autotuner and plan cache, on the GPU."""
import os

import numpy as np
import pytest
import torch

import oracle
from gpu_util import (as_np, assert_16_parity, assert_f32_parity, host_route, mixed_angles,
                      pageable_access)
from paper_cs_0406049_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("route", ["auto", "pipeline"])
def test_host_path_chunks(cuda_lib, dtype, pinned, route):
    """Many chunks (a small workspace), a ragged last chunk, host arrays;
    every route: zero-copy on page-locked memory, zero-copy on pageable
    memory where the device reaches it through the host's page tables (the
    outputs are fresh, untouched pages), and the copy pipeline."""
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    n = (1 << 20) + 12345
    x = mixed_angles(n, seed=9)
    xh = torch.from_numpy(x)
    sh = torch.empty(n, dtype=tdt)
    ch = torch.empty(n, dtype=tdt)
    if pinned:
        xh, sh, ch = xh.pin_memory(), sh.pin_memory(), ch.pin_memory()
    ws = torch.empty(api.sincos_host_workspace_bytes(dtype, 100000), dtype=torch.uint8,
                     device="cuda")
    with host_route(route):
        api.sincos_pairs_host(xh, sh, ch, ws, "compensated")
        got = api.sincos_host_last_path()
    if route == "pipeline":
        assert got == "pipeline"
    elif pinned:
        assert got == "zero-copy"
    else:
        assert got == ("zero-copy-pageable" if pageable_access() else "pipeline")
    torch.cuda.synchronize()
    want_s, want_c = oracle.sincos(x, reduction="compensated", out=dtype)
    if dtype == "f32":
        assert_f32_parity(sh.numpy(), want_s, "host s")
        assert_f32_parity(ch.numpy(), want_c, "host c")
    else:
        assert_16_parity(as_np(sh), want_s, dtype == "bf16", "host s")
        assert_16_parity(as_np(ch), want_c, dtype == "bf16", "host c")


@pytest.mark.parametrize("route", ["auto", "pipeline"])
def test_host_path_mixed_memory_kinds(cuda_lib, route):
    """Page-locked x and c with a pageable s: zero-copy where the device
    reaches pageable memory (each buffer through its own address), the
    chunked copies otherwise; the results are the same."""
    n = (1 << 19) + 77
    x = mixed_angles(n, seed=10)
    xh = torch.from_numpy(x).pin_memory()
    sh = torch.empty(n)
    ch = torch.empty(n).pin_memory()
    ws = torch.empty(api.sincos_host_workspace_bytes("f32", 65536), dtype=torch.uint8,
                     device="cuda")
    with host_route(route):
        api.sincos_pairs_host(xh, sh, ch, ws)
        got = api.sincos_host_last_path()
    if route == "auto" and pageable_access():
        assert got == "zero-copy-pageable"
    else:
        assert got == "pipeline"
    torch.cuda.synchronize()
    want_s, want_c = oracle.sincos(x)
    assert_f32_parity(sh.numpy(), want_s, "mixed s")
    assert_f32_parity(ch.numpy(), want_c, "mixed c")


def test_host_path_zero_copy_in_place_and_overlap(cuda_lib):
    """Page-locked buffers: s may be x itself (binary32), a partial overlap is
    refused before anything runs."""
    n = (1 << 18) + 3
    x = mixed_angles(n, seed=11)
    buf = torch.from_numpy(x).pin_memory()
    ch = torch.empty(n).pin_memory()
    ws = torch.empty(api.sincos_host_workspace_bytes("f32", 4096), dtype=torch.uint8,
                     device="cuda")
    api.sincos_pairs_host(buf, buf, ch, ws)
    assert api.sincos_host_last_path() == "zero-copy"
    torch.cuda.synchronize()
    want_s, want_c = oracle.sincos(x)
    assert_f32_parity(buf.numpy(), want_s, "in-place s")
    assert_f32_parity(ch.numpy(), want_c, "in-place c")
    big = torch.from_numpy(mixed_angles(n + 1, seed=12)).pin_memory()
    before = big.clone()
    with pytest.raises(RuntimeError):
        api.sincos_pairs_host(big[:n], big[1:], ch, ws)
    assert api.sincos_host_last_path() == "none"
    torch.cuda.synchronize()
    assert torch.equal(big.view(torch.int32), before.view(torch.int32))   # bits: NaNs included


def test_autotune_pairs_and_plan_cache(cuda_lib, tmp_path):
    n = 1 << 22
    x = mixed_angles(n, seed=10)
    xt = torch.from_numpy(x).cuda()
    s = torch.empty_like(xt)
    c = torch.empty_like(xt)
    best = api.sincos_autotune_pairs(xt, s, c)
    assert best["block"] in (128, 256, 512, 1024)
    assert api.sincos_plan_get("pairs", "f32", n) == best
    s.zero_()
    c.zero_()
    api.sincos_pairs(xt, s, c)
    want_s, want_c = oracle.sincos(x)
    assert_f32_parity(as_np(s), want_s, "tuned s")
    assert_f32_parity(as_np(c), want_c, "tuned c")

    path = str(tmp_path / "plans.json")
    api.sincos_plan_cache_save(path)
    api.sincos_plan_set("pairs", "f32", n, 128, 1, 2, 16)
    assert api.sincos_plan_get("pairs", "f32", n) == {"block": 128, "unroll": 1, "ctas_per_sm": 2,
                                                      "vec_bytes": 16}
    api.sincos_plan_cache_load(path)
    assert api.sincos_plan_get("pairs", "f32", n) == best
    assert os.path.getsize(path) > 0


@pytest.mark.parametrize("plan", [(64, 1, 1, 16), (128, 8, 16, 32), (1024, 8, 2, 32),
                                  (96, 2, 3, 16), (256, 4, 4, 32), (128, 2, 1, 0),
                                  (1024, 2, 1, 0)])
def test_every_plan_shape_is_exact(cuda_lib, plan):
    """Odd plans (small grids, big unrolls, non-power-of-two blocks) change
    only the schedule, never the results."""
    n = 777777
    x = mixed_angles(n, seed=11)
    xt = torch.from_numpy(x).cuda()
    want_s, want_c = oracle.sincos(x)
    for op in ("pairs", "batched"):
        key = n if op == "pairs" else 3
        old = api.sincos_plan_get(op, "f32", key)
        api.sincos_plan_set(op, "f32", key, *plan)
        try:
            s = torch.empty_like(xt)
            c = torch.empty_like(xt)
            if op == "pairs":
                api.sincos_pairs(xt, s, c)
            else:
                offs = [0, 1000, 1001]
                lens = [1000, 1, n - 1001]
                segs, lens_t = api.segments(xt, s, c, offs, lens)
                api.sincos_batched(segs, lens_t)
            assert_f32_parity(as_np(s), want_s, f"{op} {plan} s")
            assert_f32_parity(as_np(c), want_c, f"{op} {plan} c")
        finally:
            api.sincos_plan_set(op, "f32", key, old["block"], old["unroll"], old["ctas_per_sm"],
                                old["vec_bytes"])


def test_autotune_backward_and_batched(cuda_lib):
    n = 1 << 21
    rng = np.random.default_rng(12)
    g = [torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda() for _ in range(4)]
    gx = torch.empty(n, device="cuda")
    p = api.sincos_autotune_backward(g[0], g[1], g[2], g[3], gx)
    assert p["unroll"] in (1, 2, 4, 8)
    lens = [1000, 50000, 3, 70000]
    total = sum(lens)
    x = mixed_angles(total, seed=13)
    xt = torch.from_numpy(x).cuda()
    s = torch.empty_like(xt)
    c = torch.empty_like(xt)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    segs, lens_t = api.segments(xt, s, c, offs, lens)
    p = api.sincos_autotune_batched(segs, lens_t)
    assert api.sincos_plan_get("batched", "f32", len(lens)) == p
    s.zero_()
    api.sincos_batched(segs, lens_t)
    want_s, _ = oracle.sincos(x)
    assert_f32_parity(as_np(s), want_s, "batched after tuning")


_DEFAULTS = """
import json, sys
sys.path.insert(0, {root!r})
from paper_cs_0406049_gb300 import api, build
build.build()
out = {{}}
for op in ("pairs", "expi", "backward", "batched"):
    for dt in ("f32", "bf16", "f16"):
        if op in ("expi", "backward") and dt != "f32":
            continue
        for lg in (0, 12, 20, 23, 24, 28):
            for n in ((1 << lg) - 1, 1 << lg):
                p = api.sincos_plan_get(op, dt, n)
                out[f"{{op}} {{dt}} {{n}}"] = [p["block"], p["unroll"], p["ctas_per_sm"],
                                            p["vec_bytes"]]
print("PLANS", json.dumps(out))
"""


def test_default_plans_by_size(cuda_lib):
    """A fresh process with no plan cache: single arrays below 2^24 angles
    default to the 4096-angle stages (256-thread CTAs, several per SM), from
    2^24 up to the large-array plans; the other operations' defaults do not
    depend on the size."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k != "SINCOS_TUNE_CACHE"}
    r = subprocess.run([sys.executable, "-c", _DEFAULTS.format(root=root)], capture_output=True,
                       text=True, timeout=300, cwd=root, env=env)
    assert r.returncode == 0, r.stdout + r.stderr
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("PLANS ")][0]
    plans = {k: tuple(v) for k, v in json.loads(line[6:]).items()}
    large = {"f32": (512, 2, 1, 0), "bf16": (512, 2, 3, 0), "f16": (512, 2, 3, 0)}
    for key, p in plans.items():
        op, dt, n = key.split()
        n = int(n)
        if op == "pairs":
            assert p == ((256, 2, 2, 0) if n < 1 << 24 else large[dt]), key
        elif op == "expi":
            assert p == (512, 2, 1, 0), key
        elif op == "backward":
            assert p == (512, 2, 2, 16), key
        else:
            assert p == ((512, 2, 2, 0) if dt == "f32" else (1024, 2, 1, 16)), key
