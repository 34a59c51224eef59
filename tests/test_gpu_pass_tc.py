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
    (640, 512, 16, 0.8, 2),    # 20 tiles of 128 x 128, multilevel
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


def _padded(x, ld):
    """device fp32 copy of x (rows x r) inside a zero rows x ld array, returned as
    the rows x r view (leading dimension ld: the TMA rules want a multiple of 4)"""
    out = torch.zeros((x.shape[0], ld), dtype=torch.float32, device="cuda")
    out[:, :x.shape[1]] = torch.as_tensor(x, dtype=torch.float32)
    return out[:, :x.shape[1]]


@pytest.mark.parametrize("m,n,hv_exact", [
    (41037, 120, True),   # 321 row tiles of 128 (ragged tail of 77 rows), ragged columns: every CTA takes >= 2 tiles
    (20513, 260, False),  # 161 x 3 = 483 tiles, ragged in both dimensions
])
def test_tc_step_many_tiles_matches_oracle(cp, m, n, hv_exact):
    # one fine-level step (halvings 0) through cpcp_step, whose fine pass is the
    # persistent tensor-core kernel: with more tiles than twice the SM count every
    # CTA walks at least two tiles (TMEM double buffers, buffer-parity hand-off);
    # element by element against the fp64 oracle step
    rng = np.random.default_rng(m + n)
    p = W.planted_cpcp(m, n, 5, 0.1, 0.8, seed=m + n)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    rk, rp, beta = 6, 5, 0.4
    Ak, Bk = rng.normal(size=(m, rk)), rng.normal(size=(n, rk))
    Ap, Bp = rng.normal(size=(m, rp)), rng.normal(size=(n, rp))
    Sk = np.where(mask & (rng.random((m, n)) < 0.2), rng.normal(size=(m, n)) * 3, 0.0)
    Sp = np.where(mask & (rng.random((m, n)) < 0.2), rng.normal(size=(m, n)) * 3, 0.0)
    mu_k = 0.25 * np.linalg.norm(np.where(mask, D, 0.0), 2)
    S_ref, L_ref, r_ref = oracle.step(D, mask, lam, mu_k, beta, 0, Sk, Sp, Ak @ Bk.T, Ap @ Bp.T)
    k = n if hv_exact else 128  # full width: the SVD is exact
    Qb = torch.as_tensor(cp.pack_mask(mask)).cuda()
    Dd = torch.as_tensor(D, dtype=torch.float32).cuda()
    args = (Dd, Qb, lam, mu_k, beta, 0, torch.as_tensor(Sk, dtype=torch.float32).cuda(),
            torch.as_tensor(Sp, dtype=torch.float32).cuda(), _padded(Ak, 8), _padded(Bk, 8), rk,
            _padded(Ap, 8), _padded(Bp, 8), rp)
    outs = {}
    for simt in (0, 1):
        with cp.Handle(0, pass_simt=simt) as h:
            outs[simt] = h.step(*args, k=k, q=2)
    S_tc = outs[0][0].double().cpu().numpy()
    S_si = outs[1][0].double().cpu().numpy()
    # the two passes round the rank-11 contraction differently: different kernels ran
    assert not np.array_equal(S_tc, S_si)
    th = 0.5 * lam * mu_k
    Lh, Sh = Ak @ Bk.T + beta * (Ak @ Bk.T - Ap @ Bp.T), Sk + beta * (Sk - Sp)
    X = Sh - 0.5 * np.where(mask, Lh + Sh - D, 0.0)
    safe = np.abs(np.abs(X) - th) > 1e-3 * th
    for S1 in (S_tc, S_si):
        assert _rel(S1, S_ref) <= 2e-6
        assert np.array_equal((S1 != 0)[safe], (S_ref != 0)[safe])
        assert np.all(S1[~mask] == 0)
    if hv_exact:
        S1, A1, B1, r, _ = outs[0]
        L1 = A1.double().cpu().numpy() @ B1.double().cpu().numpy().T
        assert r == r_ref
        assert _rel(L1, L_ref) <= 2e-5
