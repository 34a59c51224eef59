"""fp64 oracle of the unrolled multilevel iteration and its adjoint -- TEST
INFRASTRUCTURE (same rules as the rest of ``oracle/``: only tests, the smoke
check and the benchmark's CPU leg may import it; it shares no code with the
CUDA library).

Differentiating the solver is not in the paper; this module states what the
differentiated program is and computes its gradient plainly, in numpy fp64,
with LAPACK's SVD as the (library) SVD step and the composite restriction R
of ``oracle.restriction`` (eq. (Rx), Sec. 3.1, scaled to unit norm).

The program (K iterations of the step of ``oracle.step``, at a fixed number
of halvings h, from L_0 = L_{-1} = S_0 = S_{-1} = 0):

    t_0 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, beta_k = (t_k - 1) / t_{k+1}
    mu_k = mu * max(rho eta^k, 1)                  (continuation scaled by mu)
    Lh = L_k + beta_k (L_k - L_{k-1}),  Sh = S_k + beta_k (S_k - S_{k-1})
    G  = P_Q[Lh + Sh - D]                          eq. (cpcp-grad-LS)
    S_{k+1} = shrink(Sh - tau G, tau lam mu_k)     Alg. 3 threshold
    L_{k+1} = SVT(Lh - tau G) R, tau mu_k) R^T     Alg. 4 coarse step
    tau = 1/2

Its reverse sweep uses, for the SVT of M = U diag(s) V^T (thin SVD,
f(s) = max(s - theta, 0)), the adjoint (the Jacobian of a proximal map is
self-adjoint):

    A  = U^T gY V
    B  = Gs o sym(A) + Ga o skew(A) + diag(f'(s) o diag(A))
         Gs_ij = (f_i - f_j) / (s_i - s_j), Ga_ij = (f_i + f_j) / (s_i + s_j)
    gM = [U B + (gY V - U A) diag(f / s)] V^T
    gtheta = - sum_{s_i > theta} A_ii

and for the shrink y = shrink(x, theta): gx = gy [|x| > theta],
gtheta = - sum gy sign(x) [|x| > theta].  rho is a constant of the program
(not differentiated).

Pins (tests/test_oracle_unrolled.py): the forward equals K calls of the C
oracle's ``step`` (Jacobi SVD); the gradient matches central differences of
the forward; a diagonal problem has a closed-form gradient.
"""
from __future__ import annotations

import math

import numpy as np

from . import restriction, shrink

TAU = 0.5


def momentum(K: int):
    """beta_0 .. beta_{K-1} of the FISTA weights t_k."""
    t, out = 1.0, []
    for _ in range(K):
        t1 = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        out.append((t - 1.0) / t1)
        t = t1
    return out


def weights(mu: float, rho: float, eta: float, K: int):
    """mu_0 .. mu_{K-1} = mu max(rho eta^k, 1) and d mu_k / d mu."""
    g = [max(rho * eta ** k, 1.0) for k in range(K)]
    return [mu * x for x in g], g


def _svt_full(M, theta):
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    f = np.maximum(s - theta, 0.0)
    return (U * f) @ Vt, U, s, Vt.T


def _R(n, halvings):
    if halvings == 0:
        return None
    return restriction(n, halvings, scaled=True)[0]


def forward(D, mask, lam, mu, rho, eta, halvings, K, keep=False):
    """The K-step program above; returns (L_K, S_K) or, with keep, the lists
    of states L_0..L_K, S_0..S_K."""
    D = np.asarray(D, dtype=np.float64)
    m, n = D.shape
    obs = np.ones((m, n), bool) if mask is None else np.asarray(mask, bool)
    R = _R(n, halvings)
    betas = momentum(K)
    mus, _ = weights(mu, rho, eta, K)
    L = [np.zeros((m, n)), np.zeros((m, n))]  # L_{-1}, L_0
    S = [np.zeros((m, n)), np.zeros((m, n))]
    for k in range(K):
        b = betas[k]
        Lh = L[-1] + b * (L[-1] - L[-2])
        Sh = S[-1] + b * (S[-1] - S[-2])
        G = np.where(obs, Lh + Sh - D, 0.0)
        Sn = shrink(Sh - TAU * G, TAU * lam * mus[k])
        X = Lh - TAU * G
        if R is None:
            Ln = _svt_full(X, TAU * mus[k])[0]
        else:
            Ln = _svt_full(X @ R, TAU * mus[k])[0] @ R.T
        L.append(Ln)
        S.append(Sn)
    if keep:
        return L[1:], S[1:]
    return L[-1], S[-1]


def shrink_margins(D, mask, lam, mu, rho, eta, halvings, K):
    """Per entry, the smallest relative distance ||XS| - thS| / thS of the
    shrink input to its threshold over the K steps, and per step the smallest
    relative distance |s_i - thL| / thL of a singular value to the SVT
    threshold.  Entries with a small margin sit next to a kink of the program:
    a change of the trajectory smaller than the margin moves them across it."""
    D = np.asarray(D, dtype=np.float64)
    m, n = D.shape
    obs = np.ones((m, n), bool) if mask is None else np.asarray(mask, bool)
    R = _R(n, halvings)
    betas = momentum(K)
    mus, _ = weights(mu, rho, eta, K)
    Ls, Ss = forward(D, mask, lam, mu, rho, eta, halvings, K, keep=True)
    zero = np.zeros((m, n))
    ent = np.full((m, n), np.inf)
    sv = []
    for k in range(K):
        b = betas[k]
        Lh = Ls[k] + b * (Ls[k] - (Ls[k - 1] if k else zero))
        Sh = Ss[k] + b * (Ss[k] - (Ss[k - 1] if k else zero))
        G = np.where(obs, Lh + Sh - D, 0.0)
        thS, thL = TAU * lam * mus[k], TAU * mus[k]
        ent = np.minimum(ent, np.where(obs, np.abs(np.abs(Sh - TAU * G) - thS) / thS, np.inf))
        X = Lh - TAU * G
        s = np.linalg.svd(X if R is None else X @ R, compute_uv=False)
        sv.append(float(np.min(np.abs(s - thL)) / thL))
    return ent, sv


def svt_adjoint(M, theta, gY):
    """(gM, gtheta) of Y = SVT_theta(M) for the cotangent gY (module docstring)."""
    _, U, s, V = _svt_full(M, theta)
    f = np.maximum(s - theta, 0.0)
    fp = (s > theta).astype(np.float64)
    A = U.T @ gY @ V
    q = len(s)
    si, sj = s[:, None], s[None, :]
    fi, fj = f[:, None], f[None, :]
    diff = si - sj
    with np.errstate(divide="ignore", invalid="ignore"):
        Gs = np.where(np.abs(diff) > 1e-300, (fi - fj) / np.where(diff == 0, 1.0, diff), 0.5 * (fp[:, None] + fp[None, :]))
        ssum = si + sj
        Ga = np.where(ssum > 0, (fi + fj) / np.where(ssum == 0, 1.0, ssum), 0.0)
    sym, skew = 0.5 * (A + A.T), 0.5 * (A - A.T)
    B = Gs * sym + Ga * skew
    B[np.arange(q), np.arange(q)] = fp * np.diag(A)
    with np.errstate(divide="ignore", invalid="ignore"):
        fs = np.where(s > 0, f / np.where(s > 0, s, 1.0), 0.0)
    P = gY @ V
    gM = (U @ B + (P - U @ A) * fs[None, :]) @ V.T
    gtheta = -float(np.sum(np.diag(A)[s > theta]))
    return gM, gtheta


def adjoint(D, mask, lam, mu, rho, eta, halvings, K, gL, gS=None):
    """Gradient of <gL, L_K> + <gS, S_K> with respect to D, lam and mu:
    returns (dD, dlam, dmu)."""
    D = np.asarray(D, dtype=np.float64)
    m, n = D.shape
    obs = np.ones((m, n), bool) if mask is None else np.asarray(mask, bool)
    R = _R(n, halvings)
    betas = momentum(K)
    mus, dmus = weights(mu, rho, eta, K)
    Ls, Ss = forward(D, mask, lam, mu, rho, eta, halvings, K, keep=True)  # L_0 .. L_K
    zero = np.zeros((m, n))
    gLn = np.asarray(gL, dtype=np.float64).copy()            # adjoint of L_{k+1}
    gSn = zero.copy() if gS is None else np.asarray(gS, dtype=np.float64).copy()
    gLp, gSp = zero.copy(), zero.copy()                      # partial adjoints of L_k, S_k
    dD = zero.copy()
    dlam = dmu = 0.0
    for k in range(K - 1, -1, -1):
        b = betas[k]
        Lk, Sk = Ls[k], Ss[k]
        Lkm = Ls[k - 1] if k > 0 else zero
        Skm = Ss[k - 1] if k > 0 else zero
        Lh = Lk + b * (Lk - Lkm)
        Sh = Sk + b * (Sk - Skm)
        G = np.where(obs, Lh + Sh - D, 0.0)
        XS = Sh - TAU * G
        XL = Lh - TAU * G
        thL, thS = TAU * mus[k], TAU * lam * mus[k]
        # L_{k+1} = SVT(XL R) R^T
        if R is None:
            gXL, gthL = svt_adjoint(XL, thL, gLn)
        else:
            gMH, gthL = svt_adjoint(XL @ R, thL, gLn @ R)
            gXL = gMH @ R.T
        # S_{k+1} = shrink(XS, thS)
        act = np.abs(XS) > thS
        gXS = np.where(act, gSn, 0.0)
        gthS = -float(np.sum(np.where(act, gSn * np.sign(XS), 0.0)))
        # XL = Lh - tau G, XS = Sh - tau G, G = P_Q[Lh + Sh - D]
        gG = -TAU * (gXL + gXS)
        gPQ = np.where(obs, gG, 0.0)
        gLh = gXL + gPQ
        gSh = gXS + gPQ
        dD -= gPQ
        dmu += (TAU * gthL + TAU * lam * gthS) * dmus[k]
        dlam += TAU * mus[k] * gthS
        # momentum: Lh = (1 + b) L_k - b L_{k-1}
        gLn, gLp = gLp + (1.0 + b) * gLh, -b * gLh
        gSn, gSp = gSp + (1.0 + b) * gSh, -b * gSh
    return dD, dlam, dmu
