"""Run one solve of a seeded planted-CPCP workload through the C ABI and print
the solver report (for profiling a solve under a profiler or by hand).

    python -m paper_2206_13369_gb300.run_solve --m 2000 --n 2000 --rank 50 \\
        --levels 3 --max-iter 200 [--fp64] [--power-iters 1] [--tol 1e-6]

The workload is workloads.planted_cpcp(m, n, rank, corruption, observed, seed),
or with --config N one of the numbered workloads of workloads.config (3 is the
19200 x 400 video-shaped problem).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=2000)
    ap.add_argument("--n", type=int, default=2000)
    ap.add_argument("--rank", type=int, default=50)
    ap.add_argument("--corruption", type=float, default=0.10)
    ap.add_argument("--observed", type=float, default=0.8)
    ap.add_argument("--seed", type=int, default=2000)
    ap.add_argument("--levels", type=int, default=3)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iter", type=int, default=5000)
    ap.add_argument("--power-iters", type=int, default=1)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--profile", action="store_true")
    ap.add_argument("--config", type=int, default=0, help="use workloads.config(N) instead of planted_cpcp")
    args = ap.parse_args()

    import torch

    from paper_2206_13369_gb300 import cpcp, workloads
    if args.config:
        p = workloads.config(args.config)
    else:
        p = workloads.planted_cpcp(args.m, args.n, args.rank, args.corruption, args.observed, args.seed,
                                   levels=args.levels)
    dt = torch.float64 if args.fp64 else torch.float32
    D = torch.as_tensor(p["D"], dtype=dt).cuda()
    Q = None if p["mask"] is None else torch.as_tensor(cpcp.pack_mask(p["mask"])).cuda()
    with cpcp.Handle(0, max_iter=args.max_iter, power_iters=args.power_iters, profile=int(args.profile)) as h:
        for _ in range(args.repeat):
            _, _, info = h.solve(D, Q, p["lam"], p["mu"], levels=args.levels, tol=args.tol)
        torch.cuda.synchronize()
    print(json.dumps(info))
    return 0


if __name__ == "__main__":
    sys.exit(main())
