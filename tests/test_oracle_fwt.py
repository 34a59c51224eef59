"""Pins of the oracle's Frank-Wolfe Thresholding (Alg. 3) and ML-FWT (Alg. 6)
for eq. (cpcp), against facts fixed outside the oracle: brute force for the
two-segment line search, the optimum of the same program reached by the
oracle's independent proximal-gradient solver (its own stopping rule, a
different algorithm), the closed-form zero solution for large weights, and
the descent property of exact line search."""
import numpy as np
import pytest

import oracle
from paper_2206_13369_gb300 import workloads as W


def _q(A, B, C, ga, gb, a, b):
    return 0.5 * (A * a * a + 2 * C * a * b + B * b * b) + ga * a + gb * b


@pytest.mark.parametrize("seed", range(12))
def test_line_search_is_the_box_minimiser(seed):
    rng = np.random.default_rng(seed)
    P = rng.normal(size=(2, 2))
    H = P @ P.T
    if seed % 4 == 1:
        H[0, 0], H[0, 1], H[1, 0] = 0.0, 0.0, 0.0  # no curvature along the L segment
    if seed % 4 == 2:
        v = rng.normal(size=2)
        H = np.outer(v, v)  # singular: a line of minimisers
    g = rng.normal(size=2) * rng.choice([0.1, 1.0, 10.0])
    A, B, C = H[0, 0], H[1, 1], H[0, 1]
    a, b = oracle.fw_line_search(A, B, C, g[0], g[1])
    assert 0.0 <= a <= 1.0 and 0.0 <= b <= 1.0
    grid = np.linspace(0.0, 1.0, 401)
    aa, bb = np.meshgrid(grid, grid, indexing="ij")
    qmin = _q(A, B, C, g[0], g[1], aa, bb).min()
    assert _q(A, B, C, g[0], g[1], a, b) <= qmin + 1e-12
    # first-order optimality on the box
    da = A * a + C * b + g[0]
    db = C * a + B * b + g[1]
    for x, d in ((a, da), (b, db)):
        if 0.0 < x < 1.0:
            assert abs(d) <= 1e-9 * (1 + abs(g).max())
        elif x == 0.0:
            assert d >= -1e-9 * (1 + abs(g).max())
        else:
            assert d <= 1e-9 * (1 + abs(g).max())


def test_zero_solution_for_large_weights():
    # lambda_L >= ||P_Q D||_2 and lambda_S >= max |P_Q D|: (0, 0) is optimal
    # (0 lies in both subdifferentials), and FW-T must not leave it
    p = W.planted_cpcp(40, 30, 2, 0.1, 0.8, seed=3, levels=1)
    D, mask = p["D"], p["mask"]
    PD = np.where(mask, D, 0.0)
    mu = 1.01 * np.linalg.svd(PD, compute_uv=False)[0]
    lam = 1.01 * np.abs(PD).max() / mu
    L, S, it, ft, (tl, ts) = oracle.fwt(D, mask, lam, mu, max_iter=5, tol=0.0)
    assert np.abs(L).max() == 0.0 and np.abs(S).max() == 0.0 and tl == 0.0 and ts == 0.0
    assert np.allclose(ft, 0.5 * np.sum(PD ** 2), rtol=1e-15)


@pytest.fixture(scope="module")
def small_cpcp():
    p = W.planted_cpcp(60, 40, 3, 0.1, 0.8, seed=5, levels=1)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    mu = 0.05 * np.linalg.svd(np.where(mask, D, 0.0), compute_uv=False)[0]
    Lf, Sf, _ = oracle.fista(D, mask, lam, mu, levels=1, tol=1e-11)
    return D, mask, lam, mu, oracle.objective(D, mask, lam, mu, Lf, Sf)


def test_fwt_descends_and_approaches_the_optimum(small_cpcp):
    D, mask, lam, mu, fstar = small_cpcp
    L, S, it, ft, (tl, ts) = oracle.fwt(D, mask, lam, mu, max_iter=600, tol=0.0)
    assert it == 600
    # exact line search and the thresholding step (a prox step) never increase f
    assert np.all(np.diff(ft) <= 1e-12 * ft[:-1])
    # f is an upper bound of the objective of eq. (cpcp) at the iterate
    # (t_L >= ||L||_*, t_S = ||S||_1), and both approach f*
    F = oracle.objective(D, mask, lam, mu, L, S)
    assert fstar <= F <= ft[-1] * (1 + 1e-12)
    gaps = (ft - fstar) / fstar
    assert gaps[99] < gaps[9] and gaps[-1] < gaps[99] and gaps[-1] <= 0.03
    assert (F - fstar) / fstar <= 0.02
    # the O(1/k) bound of the FW analysis: f_k - f* <= 2 Lip Diam^2 / (k + 2) with the
    # 2-Lipschitz gradient and Diam <= sqrt(5) sqrt(U_L^2 + U_S^2) at the initial bounds
    f0 = 0.5 * np.sum(np.where(mask, D, 0.0) ** 2)
    diam2 = 5.0 * ((f0 / mu) ** 2 + (f0 / (lam * mu)) ** 2)
    k = np.arange(1, it + 1)
    assert np.all(ft - fstar <= 4.0 * diam2 / (k + 2))


@pytest.mark.parametrize("levels", [2, 3])
def test_ml_fwt_matches_fwt_when_the_solution_is_coarse(levels):
    # static video background: the optimum's L lies (to 0.6%) in the coarse range,
    # so ML-FWT (Theorem 5) reaches the accuracy of FW-T on the program's objective
    p = W.video_cpcp(11, h=12, w=16, frames=64, rank=1, blocks=3, block=3, obs=0.8, levels=levels)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    mu = 0.05 * np.linalg.svd(np.where(mask, D, 0.0), compute_uv=False)[0]
    Lf, Sf, _ = oracle.fista(D, mask, lam, mu, levels=1, tol=1e-11)
    fstar = oracle.objective(D, mask, lam, mu, Lf, Sf)
    L1, S1, _, ft1, _ = oracle.fwt(D, mask, lam, mu, levels=1, max_iter=300, tol=0.0)
    Lm, Sm, _, ftm, _ = oracle.fwt(D, mask, lam, mu, levels=levels, max_iter=300, tol=0.0)
    g1 = (oracle.objective(D, mask, lam, mu, L1, S1) - fstar) / fstar
    gm = (oracle.objective(D, mask, lam, mu, Lm, Sm) - fstar) / fstar
    assert np.all(np.diff(ftm) <= 1e-12 * ftm[:-1])
    assert 0.0 <= gm <= max(2.0 * g1, 5e-3), (gm, g1)


def test_stopping_rule_relative_decrease(small_cpcp):
    D, mask, lam, mu, _ = small_cpcp
    _, _, it, ft, _ = oracle.fwt(D, mask, lam, mu, max_iter=1000, tol=1e-3)
    assert it < 1000
    assert abs(ft[-2] - ft[-1]) <= 1e-3 * ft[-2]
    assert np.all(np.abs(np.diff(ft[:-1])) > 1e-3 * ft[:-2])


@pytest.mark.parametrize("levels", [2, 3])
def test_ml_fwt_orthonormal_transfer_tracks_fwt(levels):
    # with R (R^T R)^{-1/2} the lifted nuclear-ball vertex -u (R_o v_H)^T has nuclear
    # norm 1, as the fine LMO's does; on data whose solution lies near the coarse
    # range, ML-FWT then follows FW-T's objective iteration for iteration, while the
    # unit-norm R (vertices inside the ball, ||R v_H|| < 1) lags behind
    p = W.video_cpcp(11, h=12, w=16, frames=64, rank=1, blocks=3, block=3, obs=0.8, levels=levels)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    mu = 0.05 * np.linalg.svd(np.where(mask, D, 0.0), compute_uv=False)[0]
    Lf, Sf, _ = oracle.fista(D, mask, lam, mu, levels=1, tol=1e-11)
    fstar = oracle.objective(D, mask, lam, mu, Lf, Sf)
    _, _, _, f1, _ = oracle.fwt(D, mask, lam, mu, levels=1, max_iter=300, tol=0.0)
    _, _, _, fo, _ = oracle.fwt(D, mask, lam, mu, levels=levels, max_iter=300, tol=0.0, transfer="orth")
    _, _, _, fu, _ = oracle.fwt(D, mask, lam, mu, levels=levels, max_iter=300, tol=0.0, transfer="unit")
    g1, go, gu = (f1[-1] - fstar) / fstar, (fo[-1] - fstar) / fstar, (fu[-1] - fstar) / fstar
    assert np.all(np.diff(fo) <= 1e-12 * fo[:-1])
    assert go <= 1.1 * g1, (go, g1)
    assert gu >= 3.0 * go, (gu, go)
