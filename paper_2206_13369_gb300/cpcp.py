"""Python binding of the C ABI in include/cpcp.h (argument marshalling only).

Every numerical step runs in the CUDA library ``_lib/libcpcp.so``; this module
only converts arrays to pointers and sizes.  If the library is missing the
import of the binding fails loudly -- there is no CPU fallback.

Arrays may be torch CUDA tensors (device pointers, the handle's stream must be
the tensor's stream) or host arrays (numpy or CPU tensors; the library stages
them through device memory inside the call).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcpcp.so")

F32, F64 = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "non-finite input", 3: "cuda error", 4: "out of memory",
          5: "not converged", 6: "timeout", 7: "numerical breakdown"}


class CPCPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("check_every", C.c_int), ("eta", C.c_double), ("mu0", C.c_double),
                ("switch_ratio", C.c_double), ("k_max", C.c_int), ("oversample", C.c_int),
                ("power_iters", C.c_int), ("check_power_iters", C.c_int), ("start_level", C.c_int),
                ("seed", C.c_uint64), ("trace", C.POINTER(C.c_double)), ("trace_cap", C.c_int),
                ("profile", C.c_int), ("precision", C.c_int), ("refine_at", C.c_double),
                ("batch_threads", C.c_int), ("batch_autotune", C.c_int), ("unroll", C.c_int),
                ("ckpt_every", C.c_int), ("rho", C.c_double), ("subspace_mode", C.c_int),
                ("pass_simt", C.c_int), ("plain_launches", C.c_int), ("transfer", C.c_int),
                ("early_test", C.c_int), ("products_tc", C.c_int), ("cholqr_fused", C.c_int),
                ("check_serial", C.c_int), ("chol_form", C.c_int), ("svd_serial", C.c_int),
                ("gram_form", C.c_int), ("jacobi_lanes", C.c_int), ("jacobi_check", C.c_int),
                ("pdl_off", C.c_int)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("level_iters", C.c_int * 8), ("final_level", C.c_int),
                ("rank", C.c_int), ("checks", C.c_int), ("relkkt", C.c_double), ("mu0", C.c_double),
                ("pqd_fro", C.c_double), ("seconds", C.c_double), ("phase_ms", C.c_double * 4),
                ("phase_count", C.c_int * 4), ("launches", C.c_longlong), ("bf16_iters", C.c_int),
                ("svt_detail_ms", C.c_double * 4), ("jacobi_calls", C.c_int), ("jacobi_sweeps", C.c_int),
                ("chol_factors", C.c_int), ("batch_threads", C.c_int), ("batch_tile", C.c_int),
                ("level_ms", C.c_double * 8)]

    PHASES = ("pass_coarse", "pass_fine", "svt", "check")

    def as_dict(self) -> dict:
        return {"status": self.status, "iters": self.iters, "level_iters": list(self.level_iters),
                "final_level": self.final_level, "rank": self.rank, "checks": self.checks,
                "relkkt": self.relkkt, "mu0": self.mu0, "pqd_fro": self.pqd_fro, "seconds": self.seconds,
                "phase_ms": dict(zip(self.PHASES, list(self.phase_ms))),
                "phase_count": dict(zip(self.PHASES, list(self.phase_count))), "launches": self.launches,
                "bf16_iters": self.bf16_iters,
                "svt_detail_ms": dict(zip(("products", "cholqr", "jacobi", "factors"), list(self.svt_detail_ms))),
                "jacobi_calls": self.jacobi_calls, "jacobi_sweeps": self.jacobi_sweeps,
                "chol_factors": self.chol_factors, "batch_threads": self.batch_threads,
                "batch_tile": self.batch_tile, "level_ms": list(self.level_ms)}


_vp, _i64, _int, _dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double


class Problem(C.Structure):
    _fields_ = [("m", C.c_int), ("n", C.c_int), ("D", _vp), ("ldd", _i64), ("Q", _vp), ("ldq", _i64),
                ("lam", C.c_double), ("mu", C.c_double), ("levels", C.c_int), ("L", _vp), ("ldl", _i64),
                ("S", _vp), ("lds", _i64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    lib.cpcp_status_string.restype = C.c_char_p
    lib.cpcp_status_string.argtypes = [_int]
    lib.cpcp_last_error.restype = C.c_char_p
    lib.cpcp_last_error.argtypes = [_vp]
    lib.cpcp_create.argtypes = [C.POINTER(_vp), _int, _vp, C.POINTER(Options)]
    lib.cpcp_destroy.argtypes = [_vp]
    lib.cpcp_destroy.restype = None
    lib.cpcp_solve.argtypes = [_vp, _int, _int, _int, _vp, _i64, _vp, _i64, _dbl, _dbl, _int, _dbl, _vp, _i64, _vp,
                               _i64, C.POINTER(Info)]
    lib.cpcp_step.argtypes = [_vp, _int, _int, _int, _vp, _i64, _vp, _i64, _dbl, _dbl, _dbl, _int, _vp, _vp, _i64,
                              _vp, _i64, _vp, _i64, _int, _vp, _i64, _vp, _i64, _int, _int, _int, _vp, _i64, _vp,
                              _i64, _vp, _i64, _vp, _i64, C.POINTER(_int), _vp]
    lib.cpcp_restrict.argtypes = [_vp, _int, _int, _int, _int, _vp, _i64, _vp, _i64]
    lib.cpcp_prolong.argtypes = [_vp, _int, _int, _int, _int, _vp, _i64, _vp, _i64]
    lib.cpcp_transfer_info.argtypes = [_int, _int, C.POINTER(_dbl), C.POINTER(_int)]
    lib.cpcp_transfer_orth.argtypes = [_int, _int, _vp, _vp, C.POINTER(_dbl)]
    lib.cpcp_svd.argtypes = [_vp, _int, _int, _int, _vp, _i64, _int, _int, _vp, _i64, _vp, _i64, _vp, _i64, _vp]
    lib.cpcp_gemm_bf16.argtypes = [_vp, _int, _int, _int, _vp, _i64, _vp, _i64, _vp, _i64]
    lib.cpcp_solve_batched.argtypes = [_vp, _int, _vp, _dbl, _vp]
    lib.cpcp_backward.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, _i64, C.POINTER(_dbl), C.POINTER(_dbl)]
    lib.cpcp_masked_norm_static.argtypes = [_vp, _int, _int, _int, _vp, _i64, _vp, _i64, C.POINTER(_dbl),
                                            C.POINTER(C.c_int64)]
    lib.cpcp_ialm.argtypes = [_vp, _int, _int, _int, _vp, _i64, _dbl, _int, _dbl, _dbl, _int, _dbl, _vp, _i64, _vp,
                              _i64, _vp, _vp]
    lib.cpcp_fwt.argtypes = [_vp, _int, _int, _int, _vp, _i64, _vp, _i64, _dbl, _dbl, _int, _int, _dbl, _vp, _i64, _vp,
                             _i64, _vp, _vp]
    return lib


_lib = _load()

EXPORTED = ["cpcp_status_string", "cpcp_last_error", "cpcp_create", "cpcp_destroy", "cpcp_solve", "cpcp_step",
            "cpcp_restrict", "cpcp_prolong", "cpcp_transfer_info", "cpcp_transfer_orth", "cpcp_svd", "cpcp_gemm_bf16",
            "cpcp_solve_batched", "cpcp_backward", "cpcp_masked_norm_static", "cpcp_ialm", "cpcp_fwt"]


def lib():
    return _lib


def pack_mask(mask) -> np.ndarray:
    """Bit-pack a boolean (m, n) mask row-major: bit j%32 of word [i, j//32]."""
    mk = np.asarray(mask, dtype=bool)
    m, n = mk.shape
    words = (n + 31) // 32
    pad = np.zeros((m, words * 32), dtype=bool)
    pad[:, :n] = mk
    bits = pad.reshape(m, words, 32).astype(np.uint64)
    vals = (bits << np.arange(32, dtype=np.uint64)).sum(axis=2)
    return np.ascontiguousarray(vals.astype(np.uint32))


def _ptr(x):
    """(pointer, leading dimension in elements, is_torch) of a 2-D row-major array or None."""
    if x is None:
        return None, 0
    if hasattr(x, "data_ptr"):
        if x.dim() == 1:
            return x.data_ptr(), x.shape[0]
        if x.stride(1) != 1:
            raise ValueError("arrays must be row-major with unit column stride")
        return x.data_ptr(), x.stride(0)
    a = x
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("numpy arrays must be C-contiguous")
    return a.ctypes.data, (a.shape[1] if a.ndim == 2 else a.shape[0])


def _dtype_code(x) -> int:
    name = str(x.dtype)
    if name.endswith("float32"):
        return F32
    if name.endswith("float64"):
        return F64
    raise TypeError(f"unsupported dtype {x.dtype}")


def _empty_like(x, shape):
    if hasattr(x, "data_ptr"):
        import torch
        return torch.empty(shape, dtype=x.dtype, device=x.device)
    return np.empty(shape, dtype=x.dtype)


def _zeros_like(x, shape):
    if hasattr(x, "data_ptr"):
        import torch
        return torch.zeros(shape, dtype=x.dtype, device=x.device)
    return np.zeros(shape, dtype=x.dtype)


class Handle:
    """Owns a cpcp_handle (device workspace, bound stream, options)."""

    def __init__(self, device: int = 0, stream=None, **opts):
        o = Options()
        self._trace = None
        tcap = int(opts.pop("trace_cap", 0))
        if tcap > 0:
            self._trace = np.zeros(tcap, dtype=np.float64)
            o.trace = self._trace.ctypes.data_as(C.POINTER(C.c_double))
            o.trace_cap = tcap
        for k, v in opts.items():
            if not hasattr(o, k) or k == "trace":
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                stream = None
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.device = device
        self.stream = stream
        h = _vp()
        st = _lib.cpcp_create(C.byref(h), device, _vp(stream) if stream else None, C.byref(o))
        if st != 0:
            raise CPCPError(st, "cpcp_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.cpcp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st: int, what: str):
        if st not in (0, 5):
            raise CPCPError(st, f"{what}: {_lib.cpcp_last_error(self._h).decode()}")
        return st

    # ------------------------------------------------------------------
    def solve(self, D, Qbits=None, lam: float = None, mu: float = None, levels: int = 1, tol: float = 1e-6,
              L_out=None, S_out=None, want_L: bool = True, want_S: bool = True):
        """Solve eq. (cpcp); returns (L, S, info).  Qbits: packed mask (see
        pack_mask) on the same side (host/device) as D, or None."""
        m, n = D.shape
        dt = _dtype_code(D)
        if L_out is None and want_L:
            L_out = _empty_like(D, (m, n))
        if S_out is None and want_S:
            S_out = _empty_like(D, (m, n))
        pD, ldd = _ptr(D)
        pQ, ldq = _ptr(Qbits)
        pL, ldl = _ptr(L_out)
        pS, lds = _ptr(S_out)
        info = Info()
        st = _lib.cpcp_solve(self._h, m, n, dt, pD, ldd, pQ, ldq, float(lam), float(mu), int(levels), float(tol),
                             pL, ldl, pS, lds, C.byref(info))
        self._check(st, "cpcp_solve")
        d = info.as_dict()
        if self._trace is not None:
            d["trace"] = self._trace[:min(info.checks, len(self._trace))].copy()
        return L_out, S_out, d

    def ialm(self, D, lam: float, levels: int = 1, mu0: float = 0.0, rho: float = 0.0, max_iter: int = 1000,
             tol: float = 1e-7, L_out=None, S_out=None):
        """IALM (Alg. 1) / ML-IALM (Alg. 4, levels > 1) for eq. (rpca) on D
        (m x n, n <= m); returns (L, S, info) with info["fg"] the feasibility
        gap after each iteration."""
        m, n = D.shape
        dt = _dtype_code(D)
        if L_out is None:
            L_out = _empty_like(D, (m, n))
        if S_out is None:
            S_out = _empty_like(D, (m, n))
        pD, ldd = _ptr(D)
        pL, ldl = _ptr(L_out)
        pS, lds = _ptr(S_out)
        fg = np.zeros(int(max_iter), dtype=np.float64)
        info = Info()
        st = _lib.cpcp_ialm(self._h, m, n, dt, pD, ldd, float(lam), int(levels), float(mu0), float(rho),
                            int(max_iter), float(tol), pL, ldl, pS, lds, fg.ctypes.data_as(_vp), C.byref(info))
        if st not in (0, 5):
            self._check(st, "cpcp_ialm")
        d = info.as_dict()
        d["fg"] = fg[:info.iters].copy()
        return L_out, S_out, d

    def fwt(self, D, Qbits, lam: float, mu: float, levels: int = 1, max_iter: int = 1000, tol: float = 1e-3,
            L_out=None, S_out=None):
        """Frank-Wolfe Thresholding (Alg. 3) / ML-FWT (Alg. 6, levels > 1) for
        eq. (cpcp) on device tensors; returns (L, S, info) with info["f"] the
        epigraph objective after each iteration."""
        m, n = D.shape
        dt = _dtype_code(D)
        if L_out is None:
            L_out = _empty_like(D, (m, n))
        if S_out is None:
            S_out = _empty_like(D, (m, n))
        pD, ldd = _ptr(D)
        pQ, ldq = _ptr(Qbits)
        pL, ldl = _ptr(L_out)
        pS, lds = _ptr(S_out)
        ft = np.zeros(int(max_iter), dtype=np.float64)
        info = Info()
        st = _lib.cpcp_fwt(self._h, m, n, dt, pD, ldd, pQ, ldq if pQ else 0, float(lam), float(mu), int(levels),
                           int(max_iter), float(tol), pL, ldl, pS, lds, ft.ctypes.data_as(_vp), C.byref(info))
        if st not in (0, 5):
            self._check(st, "cpcp_fwt")
        d = info.as_dict()
        d["f"] = ft[:info.iters].copy()
        return L_out, S_out, d

    def step(self, D, Qbits, lam, mu_k, beta, halvings, S_k, S_p, A_k, B_k, r_k, A_p, B_p, r_p, k, q=1,
             Omega0=None):
        """One accelerated proximal-gradient step of the multilevel method;
        returns (S_out, A_out, B_out, r_out, sigma)."""
        m, n = D.shape
        dt = _dtype_code(D)
        S_out = _empty_like(D, (m, n))
        A_out = _zeros_like(D, (m, k))
        B_out = _zeros_like(D, (n, k))
        pD, ldd = _ptr(D)
        pQ, ldq = _ptr(Qbits)
        pSk, ldsk = _ptr(S_k)
        pSp, _ = _ptr(S_p)
        pAk, lda = _ptr(A_k)
        pBk, ldb = _ptr(B_k)
        pAp, ldap = _ptr(A_p)
        pBp, ldbp = _ptr(B_p)
        pO, ldo = _ptr(Omega0)
        pSo, lds = _ptr(S_out)
        pAo, ldao = _ptr(A_out)
        pBo, ldbo = _ptr(B_out)
        r = _int(0)
        sig = np.zeros(k, dtype=np.float64)
        st = _lib.cpcp_step(self._h, m, n, dt, pD, ldd, pQ, ldq, float(lam), float(mu_k), float(beta),
                            int(halvings), pSk, pSp, ldsk, pAk, lda if pAk else 1, pBk, ldb if pBk else 1, int(r_k),
                            pAp, ldap if pAp else 1, pBp, ldbp if pBp else 1, int(r_p), int(k), int(q), pO, ldo,
                            pSo, lds, pAo, ldao, pBo, ldbo, C.byref(r), sig.ctypes.data)
        self._check(st, "cpcp_step")
        return S_out, A_out, B_out, int(r.value), sig

    def restrict(self, M, halvings: int):
        m, n = M.shape
        nh = transfer_info(n, halvings)[1]
        out = _empty_like(M, (m, nh))
        pM, ldm = _ptr(M)
        pO, ldo = _ptr(out)
        self._check(_lib.cpcp_restrict(self._h, m, n, int(halvings), _dtype_code(M), pM, ldm, pO, ldo),
                    "cpcp_restrict")
        return out

    def prolong(self, V, n: int, halvings: int):
        nh, r = V.shape
        out = _empty_like(V, (n, r))
        pV, ldv = _ptr(V)
        pO, ldo = _ptr(out)
        self._check(_lib.cpcp_prolong(self._h, int(n), int(halvings), int(r), _dtype_code(V), pV, ldv, pO, ldo),
                    "cpcp_prolong")
        return out

    def svd(self, M, k: int, q: int = 2, Omega0=None):
        m, n = M.shape
        U = _empty_like(M, (m, k))
        V = _empty_like(M, (n, k))
        sig = np.zeros(k, dtype=np.float64)
        pM, ldm = _ptr(M)
        pO, ldo = _ptr(Omega0)
        pU, ldu = _ptr(U)
        pV, ldv = _ptr(V)
        self._check(_lib.cpcp_svd(self._h, m, n, _dtype_code(M), pM, ldm, int(k), int(q), pO, ldo, pU, ldu, pV,
                                  ldv, sig.ctypes.data), "cpcp_svd")
        return U, sig, V

    def solve_batched(self, problems, tol: float = 1e-6, want_L: bool = True, want_S: bool = True):
        """Solve many fp32 instances in one persistent launch.  problems: list
        of dicts with D (device fp32 tensor), Q (packed device mask or None),
        lam, mu, levels.  Returns (list of L, list of S, list of info dicts,
        overall status)."""
        import torch
        arr = (Problem * len(problems))()
        Ls, Ss, keep = [], [], []
        for i, pr in enumerate(problems):
            D = pr["D"]
            m, n = D.shape
            L = torch.empty((m, n), dtype=torch.float32, device=D.device) if want_L else None
            S = torch.empty((m, n), dtype=torch.float32, device=D.device) if want_S else None
            pD, ldd = _ptr(D)
            pQ, ldq = _ptr(pr.get("Q"))
            pL, ldl = _ptr(L)
            pS, lds = _ptr(S)
            arr[i] = Problem(m, n, pD, ldd, pQ, ldq, float(pr["lam"]), float(pr["mu"]), int(pr.get("levels", 1)),
                             pL, ldl, pS, lds)
            Ls.append(L)
            Ss.append(S)
            keep.append(pr)
        infos = (Info * len(problems))()
        st = _lib.cpcp_solve_batched(self._h, len(problems), C.cast(arr, _vp), float(tol), C.cast(infos, _vp))
        if st not in (0, 2, 5):
            raise CPCPError(st, f"cpcp_solve_batched: {_lib.cpcp_last_error(self._h).decode()}")
        return Ls, Ss, [f.as_dict() for f in infos], st

    def backward(self, dL, dS=None):
        """Reverse sweep of the last unrolled run on this handle (options
        unroll = K > 0): returns (dD, dlambda, dmu) for the cotangents dL, dS
        of (L_K, S_K)."""
        import torch
        m, n = dL.shape
        dD = torch.empty((m, n), dtype=torch.float32, device=dL.device)
        pL, ldl = _ptr(dL.contiguous())
        dSc = None if dS is None else dS.contiguous()
        pS, lds = _ptr(dSc)
        pD, ldd = _ptr(dD)
        dlam, dmu = _dbl(0), _dbl(0)
        self._check(_lib.cpcp_backward(self._h, pL, ldl, pS, lds if pS else 0, pD, ldd, C.byref(dlam), C.byref(dmu)),
                    "cpcp_backward")
        return dD, float(dlam.value), float(dmu.value)

    def gemm_bf16(self, A, B):
        """C = bf16(A) bf16(B)^T with fp32 accumulation on the tensor cores;
        A (rows x K) and B (N x K) fp32 device tensors."""
        import torch
        rows, K = A.shape
        N = B.shape[0]
        Cm = torch.empty((rows, N), dtype=torch.float32, device=A.device)
        pA, lda = _ptr(A)
        pB, ldb = _ptr(B)
        pC, ldc = _ptr(Cm)
        self._check(_lib.cpcp_gemm_bf16(self._h, rows, K, N, pA, lda, pB, ldb, pC, ldc), "cpcp_gemm_bf16")
        return Cm


def unrolled_cpcp(D, lam, mu, rho: float, Qbits=None, levels: int = 3, K: int = 50, ckpt_every: int = 10,
                  eta: float = 0.9, device: int = 0):
    """Differentiable unrolled multilevel CPCP: (L_K, S_K) as torch tensors,
    differentiable with respect to D (fp32 device tensor), lam and mu (0-d
    tensors or floats).  The forward and the hand-written reverse sweep run in
    the CUDA library (cpcp_solve with options.unroll, cpcp_backward).  The
    weights are mu_k = mu max(rho eta^k, 1): rho = ||P_Q D||_2 / mu gives the
    continuation of cpcp_solve."""
    import torch

    class _Unrolled(torch.autograd.Function):
        @staticmethod
        def forward(ctx, D_, lam_, mu_):
            h = Handle(device, unroll=int(K), ckpt_every=int(ckpt_every), rho=float(rho), eta=float(eta))
            L, S, _ = h.solve(D_.contiguous(), Qbits, float(lam_), float(mu_), levels=levels, tol=1.0)
            ctx.h = h
            ctx.dtype = lam_.dtype
            return L, S

        @staticmethod
        def backward(ctx, gL, gS):
            dD, dlam, dmu = ctx.h.backward(gL.contiguous(), None if gS is None else gS.contiguous())
            ctx.h.close()
            dl = torch.tensor(dlam, dtype=ctx.dtype, device=gL.device)
            dm = torch.tensor(dmu, dtype=ctx.dtype, device=gL.device)
            return dD, dl, dm

    lam_t = lam if torch.is_tensor(lam) else torch.tensor(float(lam), dtype=torch.float64)
    mu_t = mu if torch.is_tensor(mu) else torch.tensor(float(mu), dtype=torch.float64)
    return _Unrolled.apply(D, lam_t, mu_t)


def transfer_orth(n: int, halvings: int):
    """(cd, ce, kappa) of the orthonormal-basis transfer: R^T R = C^T C with C
    upper bidiagonal (diagonal cd, super-diagonal ce), and the level-test
    threshold for R C^{-1}."""
    nh = transfer_info(n, halvings)[1]
    cd = np.zeros(nh)
    ce = np.zeros(nh)
    k = _dbl(0)
    st = _lib.cpcp_transfer_orth(int(n), int(halvings), cd.ctypes.data, ce.ctypes.data, C.byref(k))
    if st != 0:
        raise CPCPError(st, "cpcp_transfer_orth")
    return cd, ce, float(k.value)


def transfer_info(n: int, halvings: int):
    """(scale, n_H) of the composite operator: scale = 1/||R_printed||_2."""
    sc = _dbl(0)
    nh = _int(0)
    st = _lib.cpcp_transfer_info(int(n), int(halvings), C.byref(sc), C.byref(nh))
    if st != 0:
        raise CPCPError(st, "cpcp_transfer_info")
    return float(sc.value), int(nh.value)


def masked_norm_static(D, Qbits=None, stream=None):
    """||P_Q[D]||_F and the count of non-finite observed entries, through the
    entry point that allocates nothing (cpcp_masked_norm_static); D and Qbits
    are device tensors on the current device."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    m, n = D.shape
    pD, ldd = _ptr(D)
    pQ, ldq = _ptr(Qbits)
    fro = _dbl(0)
    nf = C.c_int64(0)
    st = _lib.cpcp_masked_norm_static(_vp(stream) if stream else None, m, n, _dtype_code(D), pD, ldd, pQ, ldq,
                                      C.byref(fro), C.byref(nf))
    if st != 0:
        raise CPCPError(st, "cpcp_masked_norm_static")
    return float(fro.value), int(nf.value)
