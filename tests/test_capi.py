"""C-ABI boundary checks that need no GPU: the CUDA library builds for
sm_103a, loads, exports every entry point declared in include/cpcp.h, and its
host-side logic (the composite transfer operator's scale and coarse width,
Sec. 3.1 / Assumption 4) agrees with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_13369_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cpcp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cpcp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("cpcp_create", "cpcp_destroy", "cpcp_solve", "cpcp_step", "cpcp_restrict", "cpcp_prolong",
                 "cpcp_svd", "cpcp_status_string", "cpcp_last_error", "cpcp_transfer_info"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_symbol(lib):
    from paper_2206_13369_gb300 import cpcp
    assert sorted(cpcp.EXPORTED) == declared_functions()


def test_status_strings(lib):
    lib.cpcp_status_string.restype = ctypes.c_char_p
    assert lib.cpcp_status_string(0) == b"ok"
    assert lib.cpcp_status_string(1) == b"invalid argument"
    assert lib.cpcp_status_string(99) == b"unknown status"


@pytest.mark.parametrize("n,h", [(200, 1), (96, 2), (75, 3), (301, 2), (16, 3), (1, 0), (7, 0)])
def test_transfer_scale_matches_oracle(lib, n, h):
    sc = ctypes.c_double(0)
    nh = ctypes.c_int(0)
    lib.cpcp_transfer_info.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int)]
    assert lib.cpcp_transfer_info(n, h, ctypes.byref(sc), ctypes.byref(nh)) == 0
    assert nh.value == oracle.coarse_dim(n, h)
    if h == 0:
        assert sc.value == 1.0
    else:
        _, sc_or = oracle.restriction(n, h, scaled=True)
        assert abs(sc.value - sc_or) <= 1e-13 * sc_or


@pytest.mark.parametrize("n,h", [(200, 1), (96, 2), (75, 3), (301, 2), (16, 3), (400, 2)])
def test_transfer_orth_matches_oracle(lib, n, h):
    # the host factor of the orthonormal-basis transfer: R^T R = C^T C with C upper
    # bidiagonal for the unit-norm composite R; R C^{-1} has orthonormal columns and
    # spans the oracle's R (R^T R)^{-1/2}; the level-test threshold is the oracle's
    # formula applied to that basis
    nh = oracle.coarse_dim(n, h)
    cd = np.zeros(nh)
    ce = np.zeros(nh)
    kappa = ctypes.c_double(0)
    lib.cpcp_transfer_orth.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_double)]
    assert lib.cpcp_transfer_orth(n, h, cd.ctypes.data, ce.ctypes.data, ctypes.byref(kappa)) == 0
    Cm = np.diag(cd) + np.diag(ce[:-1], 1)
    assert ce[-1] == 0.0
    R, _ = oracle.restriction(n, h, scaled=True)
    assert np.abs(Cm.T @ Cm - R.T @ R).max() <= 1e-13
    Q = R @ np.linalg.inv(Cm)
    assert np.abs(Q.T @ Q - np.eye(nh)).max() <= 1e-11
    Ro = oracle.restriction_orth(n, h)
    assert np.abs(Q @ (Q.T @ Ro) - Ro).max() <= 1e-11
    k_or = oracle._load().or_restriction_kappa(n, nh, np.ascontiguousarray(Ro))
    assert abs(kappa.value - k_or) <= 1e-12 * k_or
    assert lib.cpcp_transfer_orth(n, 0, None, None, None) == 1


@pytest.mark.parametrize("n,h", [(40, 1), (40, 2), (96, 3)])
def test_orth_lift_is_basis_independent(lib, n, h):
    # the coarse LMO of ML-FWT with transfer = 1: the top singular pair of G R C^{-1}
    # lifted by R C^{-1} (library factor) equals, up to sign, the pair of G R_o lifted
    # by R_o = R (R^T R)^{-1/2} (oracle): both bases span range(R)
    nh = oracle.coarse_dim(n, h)
    cd = np.zeros(nh)
    ce = np.zeros(nh)
    lib.cpcp_transfer_orth.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_double)]
    assert lib.cpcp_transfer_orth(n, h, cd.ctypes.data, ce.ctypes.data, None) == 0
    R, _ = oracle.restriction(n, h, scaled=True)
    B = R @ np.linalg.inv(np.diag(cd) + np.diag(ce[:-1], 1))
    Ro = oracle.restriction_orth(n, h)
    G = np.random.default_rng(n + h).normal(size=(3 * n, n))
    for basis in (B, Ro):
        U, s_, Vt = np.linalg.svd(G @ basis, full_matrices=False)
        lifted = np.outer(U[:, 0], basis @ Vt[0])
        if basis is B:
            ref, sig = lifted, s_[0]
        else:
            assert abs(s_[0] - sig) <= 1e-12 * sig
            assert np.abs(lifted - ref).max() <= 1e-10 * np.abs(ref).max()


def test_transfer_rejects_bad_sizes(lib):
    sc = ctypes.c_double(0)
    nh = ctypes.c_int(0)
    assert lib.cpcp_transfer_info(0, 1, ctypes.byref(sc), ctypes.byref(nh)) == 1
    assert lib.cpcp_transfer_info(100, 6, ctypes.byref(sc), ctypes.byref(nh)) == 1


def test_create_without_device_fails_cleanly(lib):
    # on a machine without a GPU the call returns a status instead of aborting;
    # on a GPU machine an out-of-range device index is an argument error
    h = ctypes.c_void_p()
    lib.cpcp_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    st = lib.cpcp_create(ctypes.byref(h), 9999, None, None)
    assert st in (1, 3)
    assert not h.value


def test_pack_mask_layout():
    from paper_2206_13369_gb300 import cpcp
    rng = np.random.default_rng(0)
    m = rng.random((7, 70)) < 0.5
    p = cpcp.pack_mask(m)
    assert p.shape == (7, 3) and p.dtype == np.uint32
    for i in range(7):
        for j in range(70):
            assert bool((int(p[i, j // 32]) >> (j % 32)) & 1) == bool(m[i, j])
