"""Pins for the fp64 oracle: each test checks it against something other than
itself -- closed forms, a library routine on the same inputs, the paper's
worked example, invariants and optimality conditions of eq. (cpcp).

The oracle is the test-suite's reference for the CUDA path, so every part of
it is pinned here before any GPU parity claim is made.
"""
import math
import os

import numpy as np
import scipy.linalg
import pytest

import oracle
from paper_2206_13369_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


# ----------------------------------------------------------------------------
# shrink (Sec. 2.1, Alg. 1; Alg. 3 thresholding step)
# ----------------------------------------------------------------------------

def test_shrink_closed_form_scalars():
    x = np.array([3.0, -3.0, 0.5, -0.5, 1.0, -1.0, 0.0, 1.0000001])
    y = oracle.shrink(x, 1.0)
    assert y.tolist()[:6] == [2.0, -2.0, 0.0, 0.0, 0.0, 0.0]
    assert y[6] == 0.0
    assert abs(y[7] - 1e-7) < 1e-15
    # ties and signed zeros: |x| == theta maps to a signed zero
    assert math.copysign(1.0, y[5]) == -1.0


def test_shrink_moreau_identity():
    rng = np.random.default_rng(1)
    x = rng.normal(size=1000) * 3
    th = 0.7
    # x = prox_{th |.|_1}(x) + projection onto the inf-ball of radius th
    assert np.allclose(oracle.shrink(x, th) + np.clip(x, -th, th), x, atol=1e-15, rtol=0)


# ----------------------------------------------------------------------------
# Jacobi SVD vs LAPACK (library routine on the same fp64 input)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["random", "tall", "wide", "rankdef", "repeated", "diag", "zero_col"])
def test_svd_matches_lapack(kind):
    rng = np.random.default_rng(2)
    if kind == "random":
        A = rng.normal(size=(40, 40))
    elif kind == "tall":
        A = rng.normal(size=(90, 25))
    elif kind == "wide":
        A = rng.normal(size=(17, 53))
    elif kind == "rankdef":
        A = rng.normal(size=(60, 3)) @ rng.normal(size=(3, 30))
    elif kind == "repeated":
        Q1, _ = np.linalg.qr(rng.normal(size=(30, 30)))
        Q2, _ = np.linalg.qr(rng.normal(size=(20, 20)))
        s = np.array([5.0] * 4 + [2.0] * 6 + list(np.linspace(1, 0.1, 10)))
        A = Q1[:, :20] @ np.diag(s) @ Q2.T
    elif kind == "diag":
        A = np.diag([3.0, -1.0, 7.0, 0.0, 2.5])
    else:
        A = rng.normal(size=(30, 12))
        A[:, 4] = 0.0
    U, s, V = oracle.svd(A)
    s_ref = np.linalg.svd(A, compute_uv=False)
    s1 = max(s_ref[0], 1.0)
    assert np.all(np.diff(s) <= 1e-14 * s1)
    assert np.max(np.abs(s - s_ref)) <= 1e-12 * s1
    assert np.max(np.abs(U @ np.diag(s) @ V.T - A)) <= 1e-12 * s1
    p = min(A.shape)
    nz = s > 1e-10 * s1
    assert np.max(np.abs((U[:, nz].T @ U[:, nz]) - np.eye(nz.sum()))) < 1e-12
    assert np.max(np.abs(V.T @ V - np.eye(p))) < 1e-12


def test_svd_warm_start_same_result():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(50, 30))
    Q, _ = np.linalg.qr(rng.normal(size=(30, 30)))
    _, s0, _ = oracle.svd(A)
    U, s, V = oracle.svd(A, V0=Q)
    assert np.max(np.abs(s - s0)) < 1e-12 * s0[0]
    assert np.max(np.abs(U @ np.diag(s) @ V.T - A)) < 1e-12 * s0[0]


# ----------------------------------------------------------------------------
# SVT (Sec. 2.1, Alg. 1; coarse minimiser of Sec. 3.2)
# ----------------------------------------------------------------------------

def test_svt_diagonal_closed_form():
    d = np.array([5.0, 3.0, 1.0, 0.5, 0.0])
    L, r, nuc = oracle.svt(np.diag(d), 1.0)
    assert r == 2
    assert np.allclose(L, np.diag(np.maximum(d - 1.0, 0.0)), atol=1e-14)
    assert abs(nuc - 6.0) < 1e-13


def test_svt_2x2_rotated():
    c, s = math.cos(0.3), math.sin(0.3)
    U = np.array([[c, -s], [s, c]])
    c2, s2 = math.cos(1.1), math.sin(1.1)
    V = np.array([[c2, -s2], [s2, c2]])
    M = U @ np.diag([4.0, 0.5]) @ V.T
    L, r, _ = oracle.svt(M, 1.5)
    assert r == 1
    assert np.allclose(L, 2.5 * np.outer(U[:, 0], V[:, 0]), atol=1e-14)


def test_svt_moreau_identity_and_prox_optimality():
    rng = np.random.default_rng(4)
    M = rng.normal(size=(30, 20))
    th = 2.0
    L, r, _ = oracle.svt(M, th)
    Uq, sq, Vqt = np.linalg.svd(M, full_matrices=False)
    proj = Uq @ np.diag(np.minimum(sq, th)) @ Vqt  # projection onto the spectral ball
    assert np.max(np.abs(L + proj - M)) < 1e-12
    # optimality of prox_{th ||.||_*}: (M - L)/th = U_r V_r^T + W, ||W||_2 <= 1
    Ur, Vr = Uq[:, :r], Vqt[:r].T
    Wm = (M - L) / th - Ur @ Vr.T
    assert np.linalg.norm(Wm, 2) <= 1 + 1e-12
    assert np.max(np.abs(Ur.T @ Wm)) < 1e-12 and np.max(np.abs(Wm @ Vr)) < 1e-12


# ----------------------------------------------------------------------------
# restriction / interpolation (Sec. 3.1)
# ----------------------------------------------------------------------------

def test_interp_worked_example():
    RT2 = _load_golden("interp_R6x3.txt")
    R = oracle.interp_level(6)
    assert np.array_equal(2 * R.T, RT2)
    LH = np.ones((4, 3))
    assert np.array_equal(LH @ R.T, np.ones((4, 6)))


def test_interp_printed_head_rows():
    head = _load_golden("interp_Rx_head.txt")
    for n in (6, 8, 10, 40):
        R = oracle.interp_level(n)
        assert np.array_equal(2 * R[:5, :3], head)
        assert np.all(R[:5, 3:] == 0)
        # the worked example fixes the last row as e_{n/2}
        e = np.zeros(n // 2)
        e[-1] = 1.0
        assert np.array_equal(R[-1], e)


def test_interp_odd_rule():
    R = oracle.interp_level(5)
    ref = np.array([[1, 0, 0], [.5, .5, 0], [0, 1, 0], [0, .5, .5], [0, 0, 1]])
    assert np.array_equal(R, ref)


def _hat_closed_form(n, h):
    """Piecewise-linear interpolation with coarse node j at fine index j 2^h
    (1-based) and constant extension below the first node; n = nH 2^h."""
    step = 2 ** h
    nh = n // step
    R = np.zeros((n, nh))
    for i in range(1, n + 1):
        if i <= step:
            R[i - 1, 0] = 1.0
            continue
        s = i / step
        j = int(math.floor(s))
        w = s - j
        R[i - 1, j - 1] += 1 - w
        if w > 0:
            R[i - 1, j] += w
    return R


@pytest.mark.parametrize("n,h", [(8, 2), (200, 1), (400, 3), (1024, 2), (16, 3), (96, 2)])
def test_composite_is_piecewise_linear(n, h):
    R, _ = oracle.restriction(n, h, scaled=False)
    assert np.array_equal(R, _hat_closed_form(n, h))
    # unit row sums (normalised interpolation) and full column rank (Assumption 1)
    assert np.allclose(R.sum(1), 1.0, atol=0, rtol=0)
    assert np.linalg.matrix_rank(R) == R.shape[1]
    # R^T R is tridiagonal
    G = R.T @ R
    assert np.all(np.triu(G, 2) == 0)


def test_composite_mixed_parity_is_product_and_banded():
    # 2000 -> 1000 -> 500 and 75 -> 38 -> 19 -> 10 (odd sizes on the way)
    for n, h in ((2000, 2), (75, 3), (301, 2)):
        R, _ = oracle.restriction(n, h, scaled=False)
        P = np.eye(n)
        cur = n
        for _ in range(h):
            Rl = oracle.interp_level(cur)
            P = P @ Rl
            cur = Rl.shape[1]
        assert np.allclose(R, P, atol=1e-15)
        assert np.all((R != 0).sum(1) <= 2)
        assert np.allclose(R.sum(1), 1.0, atol=1e-15)


def _kappa_closed_form(n, h):
    """Threshold of the coarse-gradient test from the closed-form rows of the
    composite R (Sec. 3.1; node j at fine index j 2^h): ||R||_F^2, the column
    sums 1^T R and the tridiagonal R^T R accumulated row by row, the unit-norm
    scale from R^T R's largest eigenvalue (LAPACK), then
    kappa = sqrt(||R||_F / sqrt(n) * ||1^T R|| / sqrt(n)) for R / ||R||_2."""
    step = 2 ** h
    nh = n // step
    fro2, cs = 0.0, np.zeros(nh)
    d, e = np.zeros(nh), np.zeros(max(nh - 1, 0))
    for i in range(1, n + 1):
        if i <= step:
            ws = [(0, 1.0)]
        else:
            j = i // step
            w = i / step - j
            ws = [(j - 1, 1.0 - w)] + ([(j, w)] if w > 0 else [])
        for c, wc in ws:
            fro2 += wc * wc
            cs[c] += wc
            d[c] += wc * wc
        if len(ws) == 2:
            e[ws[0][0]] += ws[0][1] * ws[1][1]
    lam = scipy.linalg.eigvalsh_tridiagonal(d, e)[-1]
    return math.sqrt(math.sqrt(fro2 / n) * math.sqrt(float(cs @ cs) / n)) / math.sqrt(lam), fro2, cs, d, e


@pytest.mark.parametrize("n,h", [(6, 1), (200, 1), (2000, 1), (8, 2), (1024, 2), (2000, 2), (16, 3), (400, 3),
                                 (2000, 3)])
def test_restriction_kappa_closed_form(n, h):
    kap, fro2, cs, d, e = _kappa_closed_form(n, h)
    if h == 1:
        # one halving, n = 2 n_H: rows e_1, e_j (n_H of them) and (e_j + e_{j+1})/2
        # (n_H - 1): ||R||_F^2 = (3 n_H + 1)/2; column sums 5/2, 2, ..., 2, 3/2;
        # R^T R = tridiag(1/4; 9/4, 3/2, ..., 3/2, 5/4; 1/4)
        nh = n // 2
        assert fro2 == (3 * nh + 1) / 2
        assert cs[0] == 2.5 and cs[-1] == 1.5 and np.all(cs[1:-1] == 2.0)
        assert d[0] == 2.25 and d[-1] == 1.25 and np.all(d[1:-1] == 1.5) and np.all(e == 0.25)
    assert abs(oracle.restriction_kappa(n, h) - kap) <= 1e-12 * kap
    if n == 6:
        # worked example of Sec. 3.1 by hand: ||R||_F^2 = 5, ||1^T R||^2 = 12.5,
        # R^T R = [[9/4, 1/4, 0], [1/4, 3/2, 1/4], [0, 1/4, 5/4]]
        lam = np.linalg.eigvalsh(np.array([[2.25, .25, 0], [.25, 1.5, .25], [0, .25, 1.25]]))[-1]
        assert abs(kap - math.sqrt(math.sqrt(5 / 6 * 12.5 / 6)) / math.sqrt(lam)) <= 1e-14
    if n == 2000:
        # the values the level rule uses on the 2000-column workloads
        assert abs(kap - {1: 0.7246, 2: 0.5728, 3: 0.4693}[h]) < 5e-5


def test_single_level_sigma_ratio_at_most_two():
    # Sec. 3.2: sigma_1(R) / sigma_{n_H}(R) <= 2 for the interpolation operator
    for n in (6, 20, 200, 201):
        s = np.linalg.svd(oracle.interp_level(n), compute_uv=False)
        assert s[0] / s[-1] <= 2.0 + 1e-12


def test_scaled_restriction_unit_norm():
    for n, h in ((200, 1), (96, 2), (75, 3)):
        R, sc = oracle.restriction(n, h, scaled=True)
        R0, _ = oracle.restriction(n, h, scaled=False)
        s = np.linalg.svd(R0, compute_uv=False)
        assert abs(sc - 1.0 / s[0]) < 1e-13
        assert abs(np.linalg.svd(R, compute_uv=False)[0] - 1.0) < 1e-13


def test_theorem_nuclear_norm_preservation():
    # Theorem (LH-eps), Sec. 3.2: ||L_H R^T||_* >= ||L_H||_* - eps, and
    # ||L_H R^T||_* <= ||L_H||_* when ||R||_2 <= 1.
    rng = np.random.default_rng(5)
    for n, h in ((64, 1), (96, 2)):
        R0, _ = oracle.restriction(n, h, scaled=False)
        R1, _ = oracle.restriction(n, h, scaled=True)
        nh = R0.shape[1]
        sR = np.linalg.svd(R0, compute_uv=False)
        for r in (1, 3, 8):
            LH = rng.normal(size=(150, r)) @ rng.normal(size=(r, nh))
            sL = np.linalg.svd(LH, compute_uv=False)[:r]
            eps = sum(sL[k] * (1 - sR[nh - 1 - k]) for k in range(r))
            assert oracle.nuclear_norm(LH @ R0.T) >= oracle.nuclear_norm(LH) - eps - 1e-9
            assert oracle.nuclear_norm(LH @ R1.T) <= oracle.nuclear_norm(LH) + 1e-9


# ----------------------------------------------------------------------------
# gradient / objective, eq. (cpcp) and eq. (cpcp-grad-LS)
# ----------------------------------------------------------------------------

def test_grad_and_objective_small():
    D = np.array([[1.0, 2.0], [3.0, np.nan]])
    mask = np.array([[1, 1], [1, 0]], dtype=bool)
    L = np.array([[0.5, 0.0], [0.0, 9.0]])
    S = np.array([[0.0, 1.0], [0.0, 0.0]])
    G = oracle.grad(D, mask, L, S)
    assert np.array_equal(G, np.array([[-0.5, -1.0], [-3.0, 0.0]]))
    lam, mu = 0.3, 2.0
    f = oracle.objective(D, mask, lam, mu, L, S)
    nuc = np.linalg.svd(L, compute_uv=False).sum()
    ref = 0.5 * (0.25 + 1.0 + 9.0) + mu * nuc + lam * mu * 1.0
    assert abs(f - ref) < 1e-12


# ----------------------------------------------------------------------------
# solver: optimality of the fixed point, level independence, uniqueness
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg1_solutions():
    p = W.config(1)
    out = {}
    for lv in (1, 2):
        out[lv] = oracle.fista(p["D"], p["mask"], p["lam"], p["mu"], levels=lv, tol=1e-10)
    return p, out


def _subgradient_certificate(D, mask, lam, mu, L, S, relkkt):
    """Optimality of eq. (cpcp) checked with numpy only:
    -G/mu in d||L||_* and -G/(lam mu) in d||S||_1, up to the residual scale.

    A gradient-mapping residual rel * ||P_Q D||_F bounds the error of G in
    these conditions by a small multiple of it (step 1/2)."""
    obs = np.ones(D.shape, bool) if mask is None else mask
    G = np.where(obs, L + S - D, 0.0)
    tolG = 20.0 * max(relkkt, 1e-14) * np.linalg.norm(np.where(obs, D, 0.0))
    U, s, Vt = np.linalg.svd(L, full_matrices=False)
    r = int((s > 1e-9 * max(s[0], 1e-300)).sum())
    Ur, Vr = U[:, :r], Vt[:r].T
    Wm = -G / mu - Ur @ Vr.T
    assert np.linalg.norm(Wm, 2) <= 1 + tolG / mu
    assert np.max(np.abs(Ur.T @ Wm)) < tolG / mu and np.max(np.abs(Wm @ Vr)) < tolG / mu
    on = S != 0
    assert np.max(np.abs(G[on] + lam * mu * np.sign(S[on]))) < tolG
    assert np.max(np.abs(G[~on])) <= lam * mu + tolG
    assert np.all(S[~obs] == 0)
    return r


def test_fista_fixed_point_certificate(cfg1_solutions):
    p, sols = cfg1_solutions
    for lv, (L, S, info) in sols.items():
        assert info["status"] == 0 and info["relkkt"] <= 1e-10
        assert info["final_level"] == 0
        r = _subgradient_certificate(p["D"], p["mask"], p["lam"], p["mu"], L, S, info["relkkt"])
        assert r == info["rank"]


def test_single_level_equals_multilevel(cfg1_solutions):
    _, sols = cfg1_solutions
    L1, S1, _ = sols[1]
    L2, S2, i2 = sols[2]
    assert i2["level_iters"][1] > 0  # the multilevel run did use the coarse level
    assert np.linalg.norm(L2 - L1) <= 1e-8 * np.linalg.norm(L1)
    assert np.linalg.norm(S2 - S1) <= 1e-8 * np.linalg.norm(S1)


def test_optimum_independent_of_trajectory(cfg1_solutions):
    p, sols = cfg1_solutions
    L1, S1, _ = sols[1]
    L3, S3, info = oracle.fista(p["D"], None, p["lam"], p["mu"], levels=1, tol=1e-10, eta=0.7,
                                mu0=3.0 * p["mu"])
    assert info["status"] == 0
    assert np.linalg.norm(L3 - L1) <= 1e-8 * np.linalg.norm(L1)
    assert np.linalg.norm(S3 - S1) <= 1e-8 * np.linalg.norm(S1)


def test_masked_cpcp_certificate_and_levels():
    p = W.planted_cpcp(72, 64, 3, 0.08, 0.75, seed=11, levels=3)
    D = p["D"].copy()
    D[~p["mask"]] = np.nan  # unobserved entries are never read
    L1, S1, i1 = oracle.fista(D, p["mask"], p["lam"], p["mu"], levels=1, tol=1e-10)
    L3, S3, i3 = oracle.fista(D, p["mask"], p["lam"], p["mu"], levels=3, tol=1e-10)
    assert i1["status"] == 0 and i3["status"] == 0
    assert np.all(np.isfinite(L1)) and np.all(np.isfinite(S1))
    _subgradient_certificate(np.nan_to_num(D), p["mask"], p["lam"], p["mu"], L1, S1, i1["relkkt"])
    assert np.linalg.norm(L3 - L1) <= 1e-7 * np.linalg.norm(L1)
    assert np.linalg.norm(S3 - S1) <= 1e-7 * np.linalg.norm(S1)


def test_wide_problem_solved_transposed():
    p = W.planted_cpcp(40, 70, 2, 0.05, 0.9, seed=12, levels=2)
    L, S, info = oracle.fista(p["D"], p["mask"], p["lam"], p["mu"], levels=2, tol=1e-10)
    Lt, St, _ = oracle.fista(p["D"].T, p["mask"].T, p["lam"], p["mu"], levels=2, tol=1e-10)
    assert info["status"] == 0
    assert np.allclose(L, Lt.T, atol=1e-12) and np.allclose(S, St.T, atol=1e-12)
    assert oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], L, S) <= 1e-10


def test_relkkt_zero_iff_optimal(cfg1_solutions):
    p, sols = cfg1_solutions
    L, S, _ = sols[1]
    assert oracle.relkkt(p["D"], None, p["lam"], p["mu"], L, S) <= 1e-10
    rng = np.random.default_rng(6)
    Lb = L + 1e-4 * rng.normal(size=L.shape)
    assert oracle.relkkt(p["D"], None, p["lam"], p["mu"], Lb, S) > 1e-6


def test_fista_rate_on_objective_gap():
    # fixed weight (no continuation), full SVD at level 0: FISTA gives
    # F(x_k) - F* <= 2 Lf ||x_0 - x*||^2 / (k+1)^2 with Lf = 2 (Sec. 2.3); the
    # paper's Frank-Wolfe bound 2 Lf D^2 / (k+2) is weaker for k >= 1.
    p = W.planted_cpcp(30, 24, 2, 0.05, 1.0, seed=13)
    lam, mu = p["lam"], p["mu"] * 20
    Ls, Ss, inf = oracle.fista(p["D"], None, lam, mu, tol=1e-13, mu0=mu, max_iter=50000)
    Fstar = oracle.objective(p["D"], None, lam, mu, Ls, Ss)
    R2 = np.linalg.norm(Ls) ** 2 + np.linalg.norm(Ss) ** 2
    for k in (1, 2, 5, 10, 20, 40, 80):
        Lk, Sk, _ = oracle.fista(p["D"], None, lam, mu, mu0=mu, fixed_iters=k)
        gap = oracle.objective(p["D"], None, lam, mu, Lk, Sk) - Fstar
        assert gap >= -1e-10
        assert gap <= 2 * 2.0 * R2 / (k + 1) ** 2 + 1e-12


# ----------------------------------------------------------------------------
# paper-literal IALM (Alg. 1) and ML-IALM (Alg. 4)
# ----------------------------------------------------------------------------

def test_ialm_exact_recovery_planted():
    # PCP recovers a planted low-rank + sparse pair (Sec. 1 and 2, eq. (rpca))
    p = W.planted_pcp(40, 40, 2, 0.05, seed=14, factor_var=1.0 / 40)
    L, S, it, fg = oracle.ialm(p["D"], 1.0 / math.sqrt(40), max_iter=20000, tol=1e-9)
    assert fg[-1] <= 1e-9
    assert np.linalg.norm(L - p["L0"]) <= 1e-6 * np.linalg.norm(p["L0"])
    assert np.linalg.norm(S - p["S0"]) <= 1e-6 * np.linalg.norm(p["S0"])


def test_cpcp_approaches_pcp_as_mu_shrinks():
    p = W.planted_pcp(40, 40, 2, 0.05, seed=14, factor_var=1.0 / 40)
    lam = 1.0 / math.sqrt(40)
    Lp, _, _, _ = oracle.ialm(p["D"], lam, max_iter=20000, tol=1e-10)
    errs = []
    for mu in (4e-3, 2e-3, 1e-3):
        L, S, info = oracle.fista(p["D"], None, lam, mu, tol=1e-11, max_iter=50000)
        assert info["status"] == 0
        errs.append(np.linalg.norm(L - Lp))
    assert errs[0] > errs[1] > errs[2]
    # linear in mu: halving mu roughly halves the distance
    assert 1.5 < errs[0] / errs[1] < 2.5 and 1.5 < errs[1] / errs[2] < 2.5


def test_ml_ialm_is_only_approximate():
    # Theorem 3: literal ML-IALM reaches an (eps + delta)-approximate solution of
    # eq. (rpca) when the solution is not of the form L_H R^T (Assumption 3
    # violated): nearly feasible, but with a larger objective than IALM's.
    p = W.planted_pcp(60, 40, 3, 0.05, seed=15)
    lam = p["lam"]
    L1, S1, _, fg1 = oracle.ialm(p["D"], lam, levels=1, max_iter=400, tol=1e-9)
    L2, S2, _, fg2 = oracle.ialm(p["D"], lam, levels=2, max_iter=400, tol=1e-9)
    f1 = oracle.nuclear_norm(L1) + lam * np.abs(S1).sum()
    f2 = oracle.nuclear_norm(L2) + lam * np.abs(S2).sum()
    assert fg1[-1] <= 1e-9 and fg2[-1] <= 1e-4
    assert f2 > 1.05 * f1
    assert np.linalg.norm(L1 - p["L0"]) <= 1e-6 * np.linalg.norm(p["L0"])


# ----------------------------------------------------------------------------
# single step (the hot path of one iteration)
# ----------------------------------------------------------------------------

def test_step_fixed_point_at_optimum(cfg1_solutions):
    # the optimum of eq. (cpcp) is a fixed point of the fine-level prox step
    p, sols = cfg1_solutions
    L, S, _ = sols[1]
    S1, L1, r = oracle.step(p["D"], None, p["lam"], p["mu"], 0.0, 0, S, S, L, L)
    assert np.linalg.norm(L1 - L) <= 1e-8 * np.linalg.norm(L)
    assert np.linalg.norm(S1 - S) <= 1e-8 * np.linalg.norm(S)
    assert r == sols[1][2]["rank"]


def test_step_coarse_prox_optimality():
    # S_out and L_out solve their prox subproblems: S_out minimises
    # th_S ||s||_1 + 1/2 ||s - X_S||^2 and L_H minimises
    # th_L ||L_H||_* + 1/2 ||L_H - M R||^2 with L_out = L_H R^T (Alg. 4).
    rng = np.random.default_rng(21)
    m, n, h = 48, 40, 2
    p = W.planted_cpcp(m, n, 3, 0.1, 0.8, seed=22)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    mu_k, beta = 0.3, 0.4
    Sk, Sp = rng.normal(size=(m, n)) * mask, rng.normal(size=(m, n)) * mask
    Lk, Lp = rng.normal(size=(m, 3)) @ rng.normal(size=(3, n)), rng.normal(size=(m, 2)) @ rng.normal(size=(2, n))
    S1, L1, r = oracle.step(D, mask, lam, mu_k, beta, h, Sk, Sp, Lk, Lp)
    Lh, Sh = Lk + beta * (Lk - Lp), Sk + beta * (Sk - Sp)
    G = np.where(mask, Lh + Sh - D, 0.0)
    XS, M = Sh - 0.5 * G, Lh - 0.5 * G
    thS, thL = 0.5 * lam * mu_k, 0.5 * mu_k
    on = S1 != 0
    assert np.allclose((XS - S1)[on], thS * np.sign(S1[on]), atol=1e-12)
    assert np.all(np.abs(XS[~on]) <= thS + 1e-12)
    R, _ = oracle.restriction(n, h, scaled=True)
    LH = L1 @ R @ np.linalg.inv(R.T @ R)
    assert np.allclose(LH @ R.T, L1, atol=1e-10)  # L_out lies in the prolongation range
    U, s, Vt = np.linalg.svd(LH, full_matrices=False)
    rr = int((s > 1e-10).sum())
    assert rr == r
    Wm = (M @ R - LH) / thL - U[:, :rr] @ Vt[:rr]
    assert np.linalg.norm(Wm, 2) <= 1 + 1e-9
    assert np.max(np.abs(U[:, :rr].T @ Wm)) < 1e-9 and np.max(np.abs(Wm @ Vt[:rr].T)) < 1e-9
