"""Pins of the unrolled-iteration oracle and its adjoint (CPU only).

The forward is checked against K calls of the C oracle's step (a separate
Jacobi SVD); the SVT adjoint and the full reverse sweep against central
finite differences in fp64; a diagonal one-step problem against its closed
form.  A dropped term or sign in the adjoint moves at least one of these."""
import numpy as np
import pytest

import oracle
from oracle import unrolled as U
from paper_2206_13369_gb300 import workloads as W


def _problem(m, n, rank, seed, obs=0.8):
    # rho puts mu_0 10% above ||P_Q D||_2: at exactly ||P_Q D||_2 the first
    # single-level step thresholds tau P_Q D at its top singular value, a kink
    p = W.planted_cpcp(m, n, rank, 0.1, obs, seed=seed)
    rho = 1.1 * oracle.spectral_norm(np.where(p["mask"], p["D"], 0.0) if p["mask"] is not None else p["D"]) / p["mu"]
    return p, rho


@pytest.mark.parametrize("halvings", [0, 1, 2])
def test_forward_equals_repeated_step(halvings):
    p, rho = _problem(48, 32, 3, 11 + halvings)
    K, eta = 7, 0.9
    L, S = U.forward(p["D"], p["mask"], p["lam"], p["mu"], rho, eta, halvings, K)
    m, n = p["D"].shape
    Lk = Lp = Sk = Sp = np.zeros((m, n))
    betas = U.momentum(K)
    mus, _ = U.weights(p["mu"], rho, eta, K)
    for k in range(K):
        Sn, Ln, _ = oracle.step(p["D"], p["mask"], p["lam"], mus[k], betas[k], halvings, Sk, Sp, Lk, Lp)
        Lp, Lk, Sp, Sk = Lk, Ln, Sk, Sn
    assert np.allclose(L, Lk, rtol=0, atol=1e-10 * np.abs(Lk).max())
    assert np.allclose(S, Sk, rtol=0, atol=1e-10 * max(np.abs(Sk).max(), 1.0))


def test_momentum_and_weights():
    b = U.momentum(4)
    assert b[0] == 0.0
    t1 = 0.5 * (1 + np.sqrt(5.0))
    t2 = 0.5 * (1 + np.sqrt(1 + 4 * t1 * t1))
    assert np.isclose(b[1], (t1 - 1) / t2)
    mus, d = U.weights(2.0, 3.0, 0.5, 4)
    assert mus == [6.0, 3.0, 2.0, 2.0] and d == [3.0, 1.5, 1.0, 1.0]


@pytest.mark.parametrize("shape,theta_q", [((30, 12), 0.5), ((25, 25), 0.3), ((40, 8), 0.8)])
def test_svt_adjoint_matches_finite_differences(shape, theta_q):
    rng = np.random.default_rng(sum(shape))
    M = rng.standard_normal(shape)
    s = np.linalg.svd(M, compute_uv=False)
    theta = float(np.quantile(s, theta_q))
    gY = rng.standard_normal(shape)
    gM, gth = U.svt_adjoint(M, theta, gY)
    f = lambda X, th: float(np.sum(gY * U._svt_full(X, th)[0]))
    h = 1e-6
    for _ in range(3):
        E = rng.standard_normal(shape)
        fd = (f(M + h * E, theta) - f(M - h * E, theta)) / (2 * h)
        assert abs(fd - np.sum(gM * E)) <= 1e-6 * (abs(fd) + 1.0)
    fd = (f(M, theta + h) - f(M, theta - h)) / (2 * h)
    assert abs(fd - gth) <= 1e-6 * (abs(fd) + 1.0)


@pytest.mark.parametrize("halvings,K,obs", [(1, 8, 0.8), (0, 6, 1.0), (2, 10, 0.7)])
def test_adjoint_matches_finite_differences(halvings, K, obs):
    p, rho = _problem(40, 28, 3, 100 + K, obs)
    D, mask, lam, mu = p["D"], p["mask"], p["lam"], p["mu"]
    rng = np.random.default_rng(K)
    L0 = rng.standard_normal(D.shape)
    gS = 0.3 * rng.standard_normal(D.shape)
    eta = 0.9

    def loss(D_, lam_, mu_):
        L, S = U.forward(D_, mask, lam_, mu_, rho, eta, halvings, K)
        return float(np.sum((L - L0) ** 2) + np.sum(gS * S))

    LK, _ = U.forward(D, mask, lam, mu, rho, eta, halvings, K)
    dD, dlam, dmu = U.adjoint(D, mask, lam, mu, rho, eta, halvings, K, 2.0 * (LK - L0), gS)
    h = 1e-6
    fd_lam = (loss(D, lam * (1 + h), mu) - loss(D, lam * (1 - h), mu)) / (2 * h * lam)
    fd_mu = (loss(D, lam, mu * (1 + h)) - loss(D, lam, mu * (1 - h))) / (2 * h * mu)
    assert abs(fd_lam - dlam) <= 1e-5 * (abs(fd_lam) + 1e-3)
    assert abs(fd_mu - dmu) <= 1e-5 * (abs(fd_mu) + 1e-3)
    for _ in range(3):
        E = rng.standard_normal(D.shape)
        E /= np.linalg.norm(E)
        fd = (loss(D + h * E, lam, mu) - loss(D - h * E, lam, mu)) / (2 * h)
        assert abs(fd - np.sum(dD * E)) <= 1e-5 * (abs(fd) + 1e-3)
    if mask is not None:
        assert np.all(dD[~mask] == 0)  # unobserved entries of D never enter


def test_one_step_diagonal_closed_form():
    # K = 1 from zero: L_1 = SVT(tau D, tau mu_0), S_1 = shrink(tau D, tau lam mu_0);
    # with D = diag(d), gL = gS = I the gradient is diagonal indicators
    d = np.array([5.0, 3.0, 2.0, 0.7, 0.2])
    D = np.diag(d)
    lam, mu, rho = 0.9, 1.0, 1.5
    mu0 = mu * rho
    dD, dlam, dmu = U.adjoint(D, None, lam, mu, rho, 0.9, 0, 1, np.eye(5), np.eye(5))
    actL = d > mu0
    actS = d > lam * mu0
    want = np.diag(0.5 * (actL.astype(float) + actS.astype(float)))
    assert np.allclose(dD, want, atol=1e-12)
    assert np.isclose(dmu, -0.5 * rho * (actL.sum() + lam * actS.sum()))
    assert np.isclose(dlam, -0.5 * mu0 * actS.sum())


def test_shrink_margins_one_step():
    # one step from zero: the shrink input is tau D, its threshold tau lam mu_0
    d = np.array([5.0, 3.0, 2.0, 0.7, 0.2])
    D = np.diag(d)
    lam, mu, rho = 0.9, 1.0, 1.5
    ent, sv = U.shrink_margins(D, None, lam, mu, rho, 0.9, 0, 1)
    th = lam * mu * rho
    assert np.allclose(np.diag(ent), np.abs(d - th) / th)
    assert np.all(ent[~np.eye(5, dtype=bool)] == 1.0)  # zero entries: | 0 - th | / th
    assert np.isclose(sv[0], np.min(np.abs(d - mu * rho)) / (mu * rho))
