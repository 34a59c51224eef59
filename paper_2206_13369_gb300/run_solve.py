"""Run one solve of a seeded planted-CPCP workload through the C ABI and print
the solver report (for profiling a solve under a profiler or by hand).

    python -m paper_2206_13369_gb300.run_solve --m 2000 --n 2000 --rank 50 \\
        --levels 3 --max-iter 200 [--fp64] [--power-iters 1] [--tol 1e-6]
        [--precision 1] [--products-tc 1] [--unroll K --rho R]

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
    ap.add_argument("--pass-simt", action="store_true", help="fused fine pass on the SIMT cores")
    ap.add_argument("--plain-launches", action="store_true", help="no CUDA graph replay of iterations")
    ap.add_argument("--config", type=int, default=0, help="use workloads.config(N) instead of planted_cpcp")
    ap.add_argument("--precision", type=int, default=0, help="1: BF16 tensor-core contractions, then fp32")
    ap.add_argument("--products-tc", type=int, default=0,
                    help="subspace products M Omega, M^T Q: 1 tensor cores, -1 SIMT, 0 by height")
    ap.add_argument("--transfer", type=int, default=0,
                    help="1: an orthonormal basis of the range of R on the coarse levels")
    ap.add_argument("--unroll", type=int, default=0, help="K > 0: the K-step differentiable program and its "
                    "reverse sweep (loss ||L_K - L0||^2)")
    ap.add_argument("--rho", type=float, default=1100.0, help="continuation scale of the unrolled program")
    ap.add_argument("--option", action="append", default=[], metavar="NAME=VALUE",
                    help="any other cpcp_options field (integer or float), e.g. --option chol_form=1")
    ap.add_argument("--batched", type=int, default=0, help="N > 0: the first N instances of the 256-instance "
                    "workload in one cpcp_solve_batched call")
    args = ap.parse_args()

    import torch

    from paper_2206_13369_gb300 import cpcp, workloads
    if args.batched > 0:
        ps = workloads.config(4)[:args.batched]
        probs = []
        for q in ps:
            Dq = torch.as_tensor(q["D"], dtype=torch.float32).cuda()
            Qq = None if q["mask"] is None else torch.as_tensor(cpcp.pack_mask(q["mask"])).cuda()
            probs.append({"D": Dq, "Q": Qq, "lam": q["lam"], "mu": q["mu"], "levels": q["levels"]})
        with cpcp.Handle(0, max_iter=args.max_iter) as h:
            for _ in range(args.repeat):
                _, _, infos, st = h.solve_batched(probs, tol=args.tol)
            torch.cuda.synchronize()
        print(json.dumps({"status": st, "iters": [f["iters"] for f in infos],
                          "phase_ms": [f["phase_ms"] for f in infos]}))
        return 0
    if args.config:
        p = workloads.config(args.config)
    else:
        p = workloads.planted_cpcp(args.m, args.n, args.rank, args.corruption, args.observed, args.seed,
                                   levels=args.levels)
    dt = torch.float64 if args.fp64 else torch.float32
    D = torch.as_tensor(p["D"], dtype=dt).cuda()
    Q = None if p["mask"] is None else torch.as_tensor(cpcp.pack_mask(p["mask"])).cuda()
    opts = dict(max_iter=args.max_iter, power_iters=args.power_iters, profile=int(args.profile),
                pass_simt=int(args.pass_simt), plain_launches=int(args.plain_launches),
                precision=args.precision, transfer=args.transfer, products_tc=args.products_tc)
    for kv in args.option:
        name, val = kv.split("=", 1)
        opts[name] = float(val) if any(c in val for c in ".e") else int(val)
    if args.unroll > 0:
        opts.update(unroll=args.unroll, rho=args.rho)
    with cpcp.Handle(0, **opts) as h:
        for _ in range(args.repeat):
            L, _, info = h.solve(D, Q, p["lam"], p["mu"], levels=args.levels, tol=args.tol)
            if args.unroll > 0:
                _, dlam, dmu = h.backward(2.0 * (L - torch.as_tensor(p["L0"], dtype=torch.float32).cuda()))
                info["dlambda"], info["dmu"] = dlam, dmu
        torch.cuda.synchronize()
    print(json.dumps(info))
    return 0


if __name__ == "__main__":
    sys.exit(main())
