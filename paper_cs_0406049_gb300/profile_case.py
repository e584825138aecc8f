"""Run one kernel of the library a few times on a synthetic case, for profilers.

    python -m paper_cs_0406049_gb300.profile_case --op forward --log2n 26 --launches 3

Generates the inputs on the device (uniform angles in [-1000, 1000) or N(0, 1)
gradients from a seeded torch generator), launches the chosen entry point
``--launches`` times on the current stream and exits.  The sizes are meant for
profiler captures: large enough to exceed the L2 cache, small enough to keep
device memory and capture time modest.
"""
from __future__ import annotations

import argparse
import sys

import torch

from . import api, build


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--op", choices=["forward", "forward_bf16", "forward_compensated",
                                    "backward", "batched", "expi", "huygens"], default="forward")
    p.add_argument("--log2n", type=int, default=26)
    p.add_argument("--launches", type=int, default=3)
    p.add_argument("--plan", default="",
                   help="block,unroll,ctas_per_sm,vec_bytes to use instead of the default plan")
    p.add_argument("--reduction", choices=["plain", "compensated"], default=None,
                   help="reduction of the forward ops (default: compensated for "
                        "forward_compensated, else plain)")
    a = p.parse_args(argv)
    build.build()
    n = 1 << a.log2n
    plan = tuple(int(v) for v in a.plan.split(",")) if a.plan else None

    def use_plan(op, dt, key):
        if plan:
            api.sincos_plan_set(op, dt, key, *plan)

    g = torch.Generator(device="cuda").manual_seed(1)
    x = (torch.rand(n, device="cuda", generator=g) * 2000.0 - 1000.0).contiguous()
    if a.op.startswith("forward"):
        dt = torch.bfloat16 if a.op == "forward_bf16" else torch.float32
        red = a.reduction or ("compensated" if a.op == "forward_compensated" else "plain")
        s = torch.empty(n, dtype=dt, device="cuda")
        c = torch.empty_like(s)
        use_plan("pairs", dt, n)
        run = lambda: api.sincos_pairs_ex(x, s, c, red)
    elif a.op == "expi":
        z = torch.empty(n, dtype=torch.complex64, device="cuda")
        use_plan("expi", "f32", n)
        run = lambda: api.sincos_expi(x, z)
    elif a.op == "huygens":
        # n observation points on a plane at z = 400, 4096 sources in a disc
        pts = (x[:n] * 0.06, torch.flip(x[:n], [0]) * 0.06, torch.full((n,), 400.0, device="cuda"))
        src = (x[:4096] * 0.014, x[4096:8192] * 0.014, torch.zeros(4096, device="cuda"))
        amp = torch.complex(torch.randn(4096, device="cuda", generator=g),
                            torch.randn(4096, device="cuda", generator=g))
        u = torch.empty(n, dtype=torch.complex64, device="cuda")
        use_plan("huygens", "f32", n)
        run = lambda: api.sincos_huygens(pts, src, amp, 6.2831855, u)
    elif a.op == "backward":
        gs = torch.randn(n, device="cuda", generator=g)
        gc = torch.randn(n, device="cuda", generator=g)
        s = torch.empty_like(x)
        c = torch.empty_like(x)
        api.sincos_pairs(x, s, c)
        gx = torch.empty_like(x)
        use_plan("backward", "f32", n)
        run = lambda: api.sincos_backward(gs, gc, s, c, gx)
    else:
        # 4096 arrays packed back to back with the batching workload's
        # log-uniform lengths, clamp(round(2^(mU)), 1, 2^m) with m = log2n - 8
        # (m = 20 at log2n = 28 gives that workload's lengths exactly)
        import numpy as np
        from . import workloads
        lens = workloads.batch_lengths(4096, max(1, a.log2n - 8), np.random.default_rng(3))
        offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
        total = int(lens.sum())
        xb = (torch.rand(total, device="cuda", generator=g) * 200.0 - 100.0).contiguous()
        del x
        s = torch.empty_like(xb)
        c = torch.empty_like(xb)
        segs, lens_t = api.segments(xb, s, c, offs, lens)
        use_plan("batched", "f32", lens_t.numel())
        run = lambda: api.sincos_batched(segs, lens_t)
    for _ in range(a.launches):
        run()
    torch.cuda.synchronize()
    print(f"profile_case {a.op} n=2^{a.log2n} launches={a.launches} ok")
    return 0


if __name__ == "__main__":
    sys.exit(main())
