"""Full-size parity: the CUDA path on the 2000 x 2000 rank-50 workload (fp32,
3 levels), on the 19200 x 400 video-shaped workload (mixed BF16/fp32, 4
levels) and on the 65536 x 128 hyperspectral-shaped workload (fp32, 1 and 3
levels), in the launch configuration the benchmark times, against the fp64
oracle's optimum of eq. (cpcp).

The oracle needs tens of minutes per solve at these sizes, so its optimum is
stored as sampled entries (tests/golden/cpcp_optimum_*.txt, written by
tests/golden/make_fullsize_optima.py, which calls only the oracle): 1024
uniformly drawn entries and 512 from the support of S.  The GPU result is
compared at those entries (relative error over the sample, and the support of
S exactly where the shrink margin of the optimum exceeds 1e-3), and its fp64
residual is evaluated by the oracle over the whole matrix.

Tolerances: the mixed path within 1e-4; the fp32 path within 2e-6 (the
attainable error: its residual floor times the workload's sensitivity; the
values measured are printed); the hyperspectral workload, whose optimum moves
about 70x the residual, within the fp64 oracle's own distance at the same
tolerance.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2206_13369_gb300 import workloads as W  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_13369_gb300 import build
    build.build()
    from paper_2206_13369_gb300 import cpcp
    return cpcp


def load_golden(name):
    rows, hdr = [], {}
    with open(os.path.join(GOLDEN, f"cpcp_optimum_{name}.txt")) as f:
        for line in f:
            if line.startswith("#"):
                for tok in line[1:].replace(";", " ").split():
                    if "=" in tok:
                        k, v = tok.split("=", 1)
                        hdr[k] = v
                continue
            i, j, L, S = line.split()
            rows.append((int(i), int(j), float(L), float(S)))
    a = np.array(rows)
    return hdr, a[:, 0].astype(np.int64), a[:, 1].astype(np.int64), a[:, 2], a[:, 3]


def sampled_errors(p, L, S, name):
    hdr, ii, jj, Lr, Sr = load_golden(name)
    assert abs(float(hdr["mu"]) - p["mu"]) <= 1e-12 * p["mu"] and abs(float(hdr["lam"]) - p["lam"]) <= 1e-15
    eL = np.linalg.norm(L[ii, jj] - Lr) / np.linalg.norm(Lr)
    eS = np.linalg.norm(S[ii, jj] - Sr) / np.linalg.norm(Sr)
    # support of S where the optimum's shrink margin is safe: X = S - tau G, G = P_Q[L + S - D]
    D = p["D"].astype(np.float32).astype(np.float64)[ii, jj]
    obs = np.ones(len(ii), bool) if p["mask"] is None else p["mask"][ii, jj]
    X = Sr - 0.5 * np.where(obs, Lr + Sr - D, 0.0)
    th = 0.5 * p["lam"] * p["mu"]
    safe = np.abs(np.abs(X) - th) > 1e-3 * th
    supp_ok = np.array_equal((S[ii, jj] != 0)[safe], (Sr != 0)[safe])
    return eL, eS, supp_ok, int(safe.sum())


@pytest.mark.parametrize("ptc", [-1, 1])
def test_cpcp2000_fp32_matches_oracle_optimum(cp, ptc):
    # solved to 7e-7, just above the fp32 path's residual floor on this workload
    # (6.5e-7 measured); the optimum moves about 2x the residual here, so the
    # attainable error is about 1.3e-6: held to 2e-6.  ptc: the subspace
    # products on the SIMT (-1) or tensor (1) cores
    p = W.config(2)
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0, max_iter=600, products_tc=ptc) as h:
        L, S, info = h.solve(D, Q, p["lam"], p["mu"], levels=3, tol=7e-7)
    assert info["status"] in (0, 5) and info["relkkt"] <= 7.5e-7, info
    L, S = L.double().cpu().numpy(), S.double().cpu().numpy()
    eL, eS, supp_ok, nsafe = sampled_errors(p, L, S, "cpcp2000")
    print(f"cpcp2000 fp32 ptc={ptc}: sampled rel err L {eL:.3e} S {eS:.3e} relkkt {info['relkkt']:.3e} "
          f"iters {info['iters']}")
    assert eL <= 2e-6 and eS <= 2e-6
    assert supp_ok and nsafe > 1400
    assert np.all(S[~p["mask"]] == 0)
    # the oracle's fp64 residual of the fp32 result, over the whole matrix
    assert oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], L, S) <= 1e-6


def test_cpcp2000_bench_tolerance_error(cp):
    # the benchmark's own solve (rel-KKT 1e-6): its error against the optimum
    p = W.config(2)
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0) as h:
        L, S, info = h.solve(D, Q, p["lam"], p["mu"], levels=3, tol=1e-6)
    assert info["status"] == 0
    eL, eS, supp_ok, _ = sampled_errors(p, L.double().cpu().numpy(), S.double().cpu().numpy(), "cpcp2000")
    print(f"cpcp2000 fp32 at 1e-6: sampled rel err L {eL:.3e} S {eS:.3e} relkkt {info['relkkt']:.3e}")
    assert eL <= 3e-6 and eS <= 3e-6 and supp_ok


@pytest.mark.parametrize("precision,transfer,tol,bar,ptc", [(1, 0, 1e-6, 1e-4, 0), (1, 1, 1e-6, 1e-4, 0),
                                                            (0, 0, 4e-7, 2e-6, 0), (0, 0, 4e-7, 2e-6, -1)])
def test_video_matches_oracle_optimum(cp, precision, transfer, tol, bar, ptc):
    # the mixed path (this workload's precision pattern) at the benchmark's tolerance,
    # within 1e-4; the fp32 path solved to 4e-7, near its residual floor of about
    # 3.5e-7, where this workload's optimum moves about 4x the residual (measured
    # 1.4e-6), within 2e-6.  ptc 0: the default choice of product kernels (the
    # tensor cores at this height), -1: SIMT
    p = W.config(3)
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0, precision=precision, transfer=transfer, max_iter=1500, products_tc=ptc) as h:
        L, S, info = h.solve(D, Q, p["lam"], p["mu"], levels=4, tol=tol)
    assert info["status"] in (0, 5) and info["relkkt"] <= 1.25 * tol, info
    L, S = L.double().cpu().numpy(), S.double().cpu().numpy()
    eL, eS, supp_ok, _ = sampled_errors(p, L, S, "video")
    print(f"video precision={precision} transfer={transfer} ptc={ptc}: sampled rel err L {eL:.3e} S {eS:.3e} "
          f"relkkt {info['relkkt']:.3e} iters {info['iters']}")
    assert eL <= bar and eS <= bar
    assert oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], L, S) <= 2e-6


@pytest.mark.parametrize("levels,transfer", [(1, 0), (3, 1)])
def test_hyperspectral_matches_oracle_optimum(cp, levels, transfer):
    # the 65536 x 128 rank-8 hyperspectral-shaped workload at the benchmark's
    # tolerance, single-level and 3 levels with the orthonormal transfer (R24),
    # against the oracle's stored optimum.  This workload is sensitive: the
    # fp64 oracle itself, stopped at rel-KKT 9.6e-7 (190 iterations), is at
    # relative distance 6.9e-5 (L) and 1.21e-4 (S) from its rel-KKT-1e-9
    # optimum at these entries, so a result at the same tolerance is held to
    # that distance; the oracle's own fp64 residual of the result to 2e-6
    p = W.config(6)
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0, transfer=transfer, max_iter=3000) as h:
        L, S, info = h.solve(D, Q, p["lam"], p["mu"], levels=levels, tol=1e-6)
    assert info["status"] == 0, info
    L, S = L.double().cpu().numpy(), S.double().cpu().numpy()
    eL, eS, supp_ok, nsafe = sampled_errors(p, L, S, "hyperspectral")
    print(f"hyperspectral levels={levels} transfer={transfer}: sampled rel err L {eL:.3e} S {eS:.3e} "
          f"relkkt {info['relkkt']:.3e} iters {info['iters']}")
    assert eL <= 7e-5 and eS <= 1.25e-4
    assert supp_ok and nsafe > 1400
    assert np.all(S[~p["mask"]] == 0)
    assert oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], L, S) <= 2e-6
