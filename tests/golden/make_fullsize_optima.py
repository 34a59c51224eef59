"""Writes sampled entries of the fp64 oracle's optimum of eq. (cpcp) for the
full-size CPCP workloads (the 2000 x 2000 rank-50 workload, the 19200 x 400
video-shaped workload and the 65536 x 128 hyperspectral-shaped workload), for
the full-size GPU parity tests and the benchmark's error columns.

Only ``oracle/`` computes anything here (``oracle.fista``, single level, the
plain full-SVD iteration; the optimum of the convex program does not depend on
the level schedule); ``workloads`` draws the seeded inputs.  D is rounded to
fp32 first, as the CUDA path stores it, so both sides solve the same program.

Output: ``cpcp_optimum_<name>.txt``: a header of ``#`` lines (workload,
oracle settings and report), then one line ``i j L_ij S_ij`` per sampled
entry: 1024 entries drawn uniformly (seeded) and 512 drawn from the support of
the oracle's S.

Run (takes tens of minutes on a few cores):
    python tests/golden/make_fullsize_optima.py [cpcp2000] [video] [hyperspectral]
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2206_13369_gb300 import workloads as W  # noqa: E402

TOL = 1e-9
WORKLOADS = {
    "cpcp2000": lambda: W.config(2),
    "video": lambda: W.config(3),
    "hyperspectral": lambda: W.config(6),
}


def write(name: str) -> str:
    p = WORKLOADS[name]()
    D = p["D"].astype(np.float32).astype(np.float64)
    mask = p["mask"]
    t0 = time.time()
    L, S, info = oracle.fista(D, mask, p["lam"], p["mu"], levels=1, tol=TOL)
    dt = time.time() - t0
    m, n = D.shape
    rng = np.random.default_rng(0x5A3)
    flat = rng.choice(m * n, size=1024, replace=False)
    supp = np.flatnonzero(S != 0)
    flat_s = rng.choice(supp, size=min(512, supp.size), replace=False)
    idx = np.concatenate([flat, flat_s])
    path = os.path.join(HERE, f"cpcp_optimum_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# fp64 oracle optimum of eq. (cpcp), sampled entries; workload {name}: m={m} n={n}\n")
        f.write(f"# lam={p['lam']!r} mu={p['mu']!r}; D rounded to fp32; oracle.fista levels=1 tol={TOL}\n")
        f.write(f"# status={info['status']} iters={info['iters']} relkkt={float(info['relkkt'])!r} "
                f"rank={info['rank']} objective={float(info['objective'])!r} seconds={dt:.0f}\n")
        f.write(f"# fro_L={float(np.linalg.norm(L))!r} fro_S={float(np.linalg.norm(S))!r} nnz_S={int(supp.size)}\n")
        f.write("# i j L S  (first 1024 uniform, then entries of supp(S))\n")
        for q in idx:
            i, j = divmod(int(q), n)
            f.write(f"{i} {j} {float(L[i, j])!r} {float(S[i, j])!r}\n")
    return path


if __name__ == "__main__":
    for nm in (sys.argv[1:] or list(WORKLOADS)):
        print(write(nm), flush=True)
