"""fp64 CPU oracle for the multilevel CPCP proximal step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product path (the CUDA
library and its Python binding) never imports, links or calls it, and the two
share no code.

The arithmetic lives in ``cpcp_oracle.c`` (plain C99 + OpenMP, fp64); this
module compiles it with gcc on first use and exposes thin numpy wrappers.
Each wrapper cites the passage of the paper it follows:

* ``shrink``          soft thresholding, Sec. 2.1 (Alg. 1) and Alg. 3.
* ``svd`` / ``svt``   one-sided Jacobi SVD and singular value thresholding,
                      Sec. 2.1 and the coarse minimiser of Sec. 3.2.
* ``interp_level``    R_n of eq. (Rx) as fixed by its worked example, Sec. 3.1.
* ``restriction``     composite R = R_n R_{n/2} ... R_{n_H}, Sec. 3.1,
                      optionally scaled to unit spectral norm (Assumption 4).
* ``grad``/``objective``  eq. (cpcp-grad-LS) and eq. (cpcp).
* ``relkkt``          fine-level gradient-mapping residual (reading of the
                      paper's stopping rule; zero iff (L, S) solves eq. (cpcp)).
* ``fista``           accelerated proximal gradient on eq. (cpcp) whose L-prox
                      is the restrict -> SVD -> SVT -> prolong step of Alg. 4.
* ``ialm``            paper-literal IALM (Alg. 1) / ML-IALM (Alg. 4).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpcp_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Opts(C.Structure):
    _fields_ = [("tau", C.c_double), ("eta", C.c_double), ("mu0", C.c_double),
                ("check_every", C.c_int), ("max_iter", C.c_int), ("switch_ratio", C.c_double),
                ("start_level", C.c_int), ("fixed_iters", C.c_int), ("transfer", C.c_int),
                ("early_test", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("final_level", C.c_int), ("rank", C.c_int), ("checks", C.c_int),
                ("status", C.c_int), ("relkkt", C.c_double), ("objective", C.c_double),
                ("level_iters", C.c_int * 16)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            lib.or_shrink.argtypes = [C.c_size_t, _dp, C.c_double, _dp]
            lib.or_svd.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, C.c_void_p]
            lib.or_svd.restype = C.c_int
            lib.or_svt.argtypes = [C.c_int, C.c_int, _dp, C.c_double, _dp, C.POINTER(C.c_double), C.c_void_p]
            lib.or_svt.restype = C.c_int
            lib.or_coarse_size.argtypes = [C.c_int]
            lib.or_coarse_size.restype = C.c_int
            lib.or_coarse_dim.argtypes = [C.c_int, C.c_int]
            lib.or_coarse_dim.restype = C.c_int
            lib.or_interp_level.argtypes = [C.c_int, _dp]
            lib.or_restriction.argtypes = [C.c_int, C.c_int, _dp]
            lib.or_restriction.restype = C.c_int
            lib.or_restriction_scaled.argtypes = [C.c_int, C.c_int, _dp, C.POINTER(C.c_double)]
            lib.or_restriction_scaled.restype = C.c_int
            lib.or_spectral_norm.argtypes = [C.c_int, C.c_int, _dp]
            lib.or_spectral_norm.restype = C.c_double
            lib.or_grad.argtypes = [C.c_int, C.c_int, _dp, C.c_void_p, _dp, _dp, _dp]
            lib.or_nuclear_norm.argtypes = [C.c_int, C.c_int, _dp]
            lib.or_nuclear_norm.restype = C.c_double
            lib.or_objective.argtypes = [C.c_int, C.c_int, _dp, C.c_void_p, C.c_double, C.c_double, _dp, _dp]
            lib.or_objective.restype = C.c_double
            lib.or_relkkt.argtypes = [C.c_int, C.c_int, _dp, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                      _dp, _dp]
            lib.or_relkkt.restype = C.c_double
            lib.or_fista.argtypes = [C.c_int, C.c_int, _dp, C.c_void_p, C.c_double, C.c_double, C.c_int,
                                     C.c_double, C.POINTER(_Opts), _dp, _dp, C.POINTER(_Info), C.c_void_p,
                                     C.c_int]
            lib.or_fista.restype = C.c_int
            lib.or_ialm.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_int, C.c_double, C.c_double,
                                    C.c_int, C.c_double, _dp, _dp, C.c_void_p, C.POINTER(C.c_double)]
            lib.or_ialm.restype = C.c_int
            lib.or_ialm_ex.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_int, C.c_double, C.c_double,
                                       C.c_int, C.c_double, _dp, _dp, C.c_void_p, C.POINTER(C.c_double), C.c_int]
            lib.or_ialm_ex.restype = C.c_int
            lib.or_restriction_orth.argtypes = [C.c_int, C.c_int, _dp]
            lib.or_restriction_orth.restype = C.c_int
            lib.or_fw_line_search.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_double)] * 2
            lib.or_fw_line_search.restype = None
            lib.or_fwt.argtypes = [C.c_int, C.c_int, _dp, C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                                   C.c_double, _dp, _dp, C.c_void_p, C.c_void_p]
            lib.or_fwt.restype = C.c_int
            lib.or_fwt_ex.argtypes = [C.c_int, C.c_int, _dp, C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                                      C.c_double, _dp, _dp, C.c_void_p, C.c_void_p, C.c_int]
            lib.or_fwt_ex.restype = C.c_int
            lib.or_num_threads.restype = C.c_int
            lib.or_set_num_threads.argtypes = [C.c_int]
            lib.or_set_num_threads.restype = None
            lib.or_step.argtypes = [C.c_int, C.c_int, _dp, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                    C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
            lib.or_step.restype = C.c_int
            lib.or_restriction_kappa.argtypes = [C.c_int, C.c_int, _dp]
            lib.or_restriction_kappa.restype = C.c_double
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mask_ptr(mask, shape):
    if mask is None:
        return None, None
    mk = np.ascontiguousarray(np.asarray(mask, dtype=bool).astype(np.uint8))
    assert mk.shape == shape
    return mk, mk.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    """Thread count of the oracle's parallel loops; n < 1 restores the default."""
    _load().or_set_num_threads(int(n))


def shrink(X, theta: float) -> np.ndarray:
    """Soft thresholding sign(x) max(|x| - theta, 0) (Sec. 2.1, Alg. 3)."""
    X = _f64(X)
    Y = np.empty_like(X)
    _load().or_shrink(X.size, X.reshape(-1), float(theta), Y.reshape(-1))
    return Y


def svd(A, V0=None):
    """Thin SVD by one-sided Jacobi; returns (U, s, V) with A = U diag(s) V^T."""
    A = _f64(A)
    m, n = A.shape
    p = min(m, n)
    U = np.zeros((m, p))
    s = np.zeros(p)
    V = np.zeros((n, p))
    v0 = None
    if V0 is not None:
        v0 = _f64(V0)
        assert v0.shape == (n, n) and m >= n
    _load().or_svd(m, n, A, U, s, V, None if v0 is None else v0.ctypes.data_as(C.c_void_p))
    return U, s, V


def svt(M, theta: float):
    """Singular value thresholding U S_theta[Sigma] V^T; returns (L, rank, nuclear norm)."""
    M = _f64(M)
    m, n = M.shape
    L = np.zeros((m, n))
    nuc = C.c_double(0.0)
    r = _load().or_svt(m, n, M, float(theta), L, C.byref(nuc), None)
    return L, int(r), float(nuc.value)


def coarse_dim(n: int, halvings: int) -> int:
    return int(_load().or_coarse_dim(n, halvings))


def interp_level(n: int) -> np.ndarray:
    """R_n of eq. (Rx), n x ceil(n/2), following the worked example of Sec. 3.1."""
    nh = int(_load().or_coarse_size(n))
    R = np.zeros((n, nh))
    _load().or_interp_level(n, R)
    return R


def restriction(n: int, halvings: int, scaled: bool = True):
    """Composite R = R_n R_{n/2} ... (Sec. 3.1); scaled to ||R||_2 = 1 if asked.

    Returns (R, scale) where scale is the factor applied (1 if unscaled)."""
    nh = coarse_dim(n, halvings)
    R = np.zeros((n, nh))
    if scaled:
        sc = C.c_double(0.0)
        _load().or_restriction_scaled(n, halvings, R, C.byref(sc))
        return R, float(sc.value)
    _load().or_restriction(n, halvings, R)
    return R, 1.0


def restriction_orth(n: int, halvings: int):
    """R (R^T R)^{-1/2} for the composite interpolation R of Sec. 3.1."""
    nh = coarse_dim(n, halvings)
    R = np.zeros((n, nh))
    _load().or_restriction_orth(n, halvings, R)
    return R


def restriction_kappa(n: int, halvings: int) -> float:
    """Threshold of the coarse-gradient test for the unit-norm composite R."""
    R, _ = restriction(n, halvings, scaled=True)
    return float(_load().or_restriction_kappa(n, R.shape[1], R))


def spectral_norm(A) -> float:
    A = _f64(A)
    return float(_load().or_spectral_norm(A.shape[0], A.shape[1], A))


def nuclear_norm(A) -> float:
    A = _f64(A)
    return float(_load().or_nuclear_norm(A.shape[0], A.shape[1], A))


def grad(D, mask, L, S) -> np.ndarray:
    """P_Q[L + S - D], eq. (cpcp-grad-LS)."""
    D, L, S = _f64(D), _f64(L), _f64(S)
    G = np.empty_like(D)
    mk, mp = _mask_ptr(mask, D.shape)
    _load().or_grad(D.shape[0], D.shape[1], D, mp, L, S, G)
    return G


def objective(D, mask, lam, mu, L, S) -> float:
    """1/2 ||P_Q[L+S-D]||_F^2 + mu ||L||_* + lam mu ||S||_1, eq. (cpcp)."""
    D, L, S = _f64(D), _f64(L), _f64(S)
    mk, mp = _mask_ptr(mask, D.shape)
    return float(_load().or_objective(D.shape[0], D.shape[1], D, mp, float(lam), float(mu), L, S))


def relkkt(D, mask, lam, mu, L, S, tau: float = 0.5) -> float:
    """Relative gradient-mapping residual of eq. (cpcp) at (L, S) (fine level)."""
    D, L, S = _f64(D), _f64(L), _f64(S)
    mk, mp = _mask_ptr(mask, D.shape)
    return float(_load().or_relkkt(D.shape[0], D.shape[1], D, mp, float(lam), float(mu), float(tau), L, S))


def fista(D, mask, lam, mu, levels=1, tol=1e-10, *, tau=0.5, eta=0.9, mu0=0.0, check_every=10,
          max_iter=20000, switch_ratio=0.9, start_level=-1, fixed_iters=0, trace_cap=4096, transfer="unit",
          early_test=False):
    """Multilevel accelerated proximal gradient for eq. (cpcp); returns (L, S, info).

    info: iters, final_level, rank, checks, status (0 ok, 3 not converged),
    relkkt, objective, level_iters (per level), trace (rel-KKT per check)."""
    D = _f64(D)
    m, n = D.shape
    mk, mp = _mask_ptr(mask, D.shape)
    L = np.zeros((m, n))
    S = np.zeros((m, n))
    o = _Opts(tau, eta, mu0, check_every, max_iter, switch_ratio, start_level, fixed_iters,
              {"unit": 0, "orth": 1}[transfer], int(bool(early_test)))
    inf = _Info()
    tr = np.zeros(max(trace_cap, 1))
    st = _load().or_fista(m, n, D, mp, float(lam), float(mu), int(levels), float(tol), C.byref(o), L, S,
                          C.byref(inf), tr.ctypes.data_as(C.c_void_p), trace_cap)
    if st == 1:
        raise ValueError("oracle.fista: invalid argument")
    info = {"iters": inf.iters, "final_level": inf.final_level, "rank": inf.rank, "checks": inf.checks,
            "status": inf.status, "relkkt": inf.relkkt, "objective": inf.objective,
            "level_iters": list(inf.level_iters), "trace": tr[:min(inf.checks, trace_cap)].copy()}
    return L, S, info


def step(D, mask, lam, mu_k, beta, halvings, S_k, S_p, L_k, L_p):
    """One step of the multilevel proximal-gradient iteration from a dense state
    (momentum, eq. (cpcp-grad-LS), Alg. 3 shrink, Alg. 4 restrict/SVT/prolong).
    Returns (S_out, L_out, rank)."""
    D = _f64(D)
    m, n = D.shape
    mk, mp = _mask_ptr(mask, D.shape)
    S_out = np.zeros((m, n))
    L_out = np.zeros((m, n))
    r = _load().or_step(m, n, D, mp, float(lam), float(mu_k), float(beta), int(halvings), _f64(S_k), _f64(S_p),
                        _f64(L_k), _f64(L_p), S_out, L_out)
    return S_out, L_out, int(r)


def fw_line_search(A, B, C_, ga, gb):
    """Exact minimiser over [0,1]^2 of 1/2 (A a^2 + 2 C a b + B b^2) + ga a + gb b
    (the two-segment line search of Alg. 3)."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    _load().or_fw_line_search(float(A), float(B), float(C_), float(ga), float(gb), C.byref(a), C.byref(b))
    return a.value, b.value


def fwt(D, mask, lam, mu, levels=1, max_iter=1000, tol=1e-3, transfer="unit"):
    """FW-T (Alg. 3) or ML-FWT (Alg. 6, levels > 1) for eq. (cpcp) with weights
    (mu, lam mu).  Returns (L, S, iters, ftrace, (t_L, t_S)) with ftrace the
    epigraph objective after each iteration."""
    D = _f64(D)
    m, n = D.shape
    mk, mp = _mask_ptr(mask, D.shape)
    L = np.zeros((m, n))
    S = np.zeros((m, n))
    ft = np.zeros(max_iter)
    ts = np.zeros(2)
    it = _load().or_fwt_ex(m, n, D, mp, float(lam), float(mu), int(levels), int(max_iter), float(tol), L, S,
                           ft.ctypes.data_as(C.c_void_p), ts.ctypes.data_as(C.c_void_p),
                           {"unit": 0, "orth": 1}[transfer])
    return L, S, it, ft[:it].copy(), (float(ts[0]), float(ts[1]))


_TRANSFER = {"unit": 0, "orth": 1, "unscaled": 2}


def ialm(D, lam, levels=1, mu0=0.0, rho=0.0, max_iter=5000, tol=1e-7, transfer="unit"):
    """Paper-literal IALM (Alg. 1) or ML-IALM (Alg. 4, levels > 1) for eq. (rpca).

    transfer (ML-IALM only): "unit" = R scaled to unit spectral norm (the
    reading of Assumption 4), "orth" = R (R^T R)^{-1/2} (orthonormal columns,
    same range), "unscaled" = the printed R.
    Returns (L, S, iters, fg) with fg the feasibility gap per iteration."""
    D = _f64(D)
    m, n = D.shape
    L = np.zeros((m, n))
    S = np.zeros((m, n))
    fg = np.zeros(max_iter)
    last = C.c_double(0.0)
    it = _load().or_ialm_ex(m, n, D, float(lam), int(levels), float(mu0), float(rho), int(max_iter), float(tol),
                            L, S, fg.ctypes.data_as(C.c_void_p), C.byref(last), _TRANSFER[transfer])
    if it < 0:
        raise ValueError("oracle.ialm: needs n <= m")
    return L, S, it, fg[:it].copy()
