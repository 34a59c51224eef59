"""The fused fine pass on the tensor cores (tcgen05 kind::tf32, each factor
entry split into three TF32 parts, six products, small and large terms in
separate fp32 accumulators) against the SIMT fp32 pass and the fp64 oracle.

Both passes compute the same iteration (momentum, masked gradient, shrink,
M = L-hat - tau G); they differ only in the rounding of the rank-K
contraction L-hat (fp32 accumulation either way; the split represents each
factor to 2^-33).  Solves through either reach the tolerance in about the
same number of iterations and land on the same optimum to the accuracy the
tolerance fixes; the oracle's own fp64 rel-KKT of each result is the
arbiter.  (A two-term split, or one accumulator shared by all six products,
left a rel-KKT floor near 1.7e-6 on the 2000 x 2000 workload: the
momentum step (1 + beta) L_k - beta L_{k-1} cancels most of L-hat.)"""
import numpy as np
import pytest

import oracle
from paper_2206_13369_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_13369_gb300 import build
    build.build()
    from paper_2206_13369_gb300 import cpcp
    return cpcp


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _solve(cp, p, levels, tol, simt, max_iter=600):
    # simt = 1: the SIMT pass; 0: the tensor-core pass
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = None if p["mask"] is None else torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0, max_iter=max_iter, pass_simt=simt) as h:
        L, S, info = h.solve(D, Q, p["lam"], p["mu"], levels=levels, tol=tol)
    return L.double().cpu().numpy(), S.double().cpu().numpy(), info


@pytest.mark.parametrize("m,n,rank,obs,levels", [
    (300, 260, 8, 0.8, 1),     # ragged tiles in both dimensions (260 = 4 x 64 + 4)
    (640, 512, 16, 0.8, 2),    # several tiles per SM, multilevel
    (512, 384, 10, 1.0, 1),    # unmasked, exact tile multiples
])
def test_tc_pass_solve_matches_simt_and_oracle(cp, m, n, rank, obs, levels):
    p = W.planted_cpcp(m, n, rank, 0.1, obs, seed=m + n + rank, levels=levels)
    Lt, St, it = _solve(cp, p, levels, 1e-6, 0)
    Ls, Ss, is_ = _solve(cp, p, levels, 1e-6, 1)
    assert it["status"] == 0 and is_["status"] == 0, (it, is_)
    # the oracle's fp64 residual of each fp32 result
    rt = oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], Lt, St)
    rs = oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], Ls, Ss)
    assert rt <= 2e-6 and rs <= 2e-6, (rt, rs)
    # same iteration count within a check interval, same optimum to the tolerance's accuracy
    assert abs(it["iters"] - is_["iters"]) <= 20
    assert _rel(Lt, Ls) <= 1e-4 and _rel(St, Ss) <= 1e-4
    if p["mask"] is not None:
        assert np.all(St[~p["mask"]] == 0)


def test_tc_pass_bench_workload(cp):
    # the 2000 x 2000 rank-50 bench workload, three levels, to 1e-6: the same
    # iteration count and optimum as through the SIMT pass
    p = W.config(2)
    Lt, St, it = _solve(cp, p, 3, 1e-6, 0, max_iter=400)
    Ls, Ss, is_ = _solve(cp, p, 3, 1e-6, 1, max_iter=400)
    assert it["status"] == 0 and is_["status"] == 0, (it, is_)
    assert it["rank"] == 50 and abs(it["iters"] - is_["iters"]) <= 10
    assert _rel(Lt, Ls) <= 1e-4 and _rel(St, Ss) <= 1e-4


def test_tc_pass_unaligned_falls_back(cp):
    # n = 130: rows of D are 520 bytes, not a multiple of 16, so the pass
    # runs on the SIMT cores; pass_simt makes no difference to the result
    p = W.planted_cpcp(150, 130, 4, 0.1, 0.8, seed=5, levels=1)
    L0, S0, i0 = _solve(cp, p, 1, 1e-6, 0)
    L1, S1, i1 = _solve(cp, p, 1, 1e-6, 1)
    assert i0["iters"] == i1["iters"]
    assert np.array_equal(L0, L1) and np.array_equal(S0, S1)
