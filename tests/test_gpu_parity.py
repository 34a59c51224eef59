"""GPU parity: the CUDA path (through the C ABI) against the fp64 oracle on
the same seeded inputs.

Operator level (element by element): restriction / prolongation (Sec. 3.1),
the subspace SVD at full width (exact), and one full proximal step of the hot
path (momentum, masked gradient, shrink, restrict -> SVD -> SVT -> prolong).
Solver level: the optimum of eq. (cpcp) for single-level and multilevel
solves, fp64 and fp32, masked and unmasked, ragged and transposed shapes.

Tolerances: fp64 element-wise 1e-10 relative; fp32 one step 2e-5 relative
(fp32 rounding of a K-term contraction and of the SVD); solutions within
the stated relative Frobenius error of the oracle's optimum.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2206_13369_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_13369_gb300 import build
    build.build()
    from paper_2206_13369_gb300 import cpcp
    return cpcp


@pytest.fixture(scope="module")
def h(cp):
    hd = cp.Handle(0)
    yield hd
    hd.close()


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def host(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ----------------------------------------------------------------------------
# transfer operators
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n,hv", [(200, 1), (96, 2), (75, 3), (301, 2), (2000, 2)])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_restrict_prolong_match_oracle(h, n, hv, dt):
    rng = np.random.default_rng(n + hv)
    m = 37
    if n <= 400:
        R, _ = oracle.restriction(n, hv, scaled=True)
    else:  # large n: unscaled product (cheap) and the library's scale, pinned separately
        R, _ = oracle.restriction(n, hv, scaled=False)
        R = R / np.linalg.svd(R, compute_uv=False)[0]
    M = rng.normal(size=(m, n))
    MH = host(h.restrict(dev(M, dt), hv))
    tol = 1e-13 if dt == torch.float64 else 2e-6
    assert rel(MH, M @ R) <= tol
    V = rng.normal(size=(R.shape[1], 7))
    B = host(h.prolong(dev(V, dt), n, hv))
    assert rel(B, R @ V) <= tol


# ----------------------------------------------------------------------------
# subspace SVD
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dt,fused,ptc", [(torch.float64, 0, 0), (torch.float32, 0, -1), (torch.float32, 0, 1),
                                           (torch.float32, 1, 1)])
@pytest.mark.parametrize("shape", [(150, 60), (97, 33), (64, 64), (2000, 120), (3001, 17), (6000, 40)])
def test_svd_full_width_exact(cp, dt, fused, ptc, shape):
    # fused = 1: fp32 CholeskyQR2 in one thread-block cluster launch; 0: six launches.
    # ptc: the products with M on the tensor cores (1) or the SIMT cores (-1)
    rng = np.random.default_rng(5)
    m, n = shape
    if dt == torch.float64 and n > 80:
        pytest.skip("fp64 subspace width is at most 80")
    A = rng.normal(size=(m, n)) @ np.diag(np.linspace(1, 0.05, n)) @ np.linalg.qr(rng.normal(size=(n, n)))[0]
    with cp.Handle(0, cholqr_fused=fused, products_tc=ptc) as h:
        U, s, V = h.svd(dev(A, dt), k=n, q=2)
    s_ref = np.linalg.svd(A, compute_uv=False)
    # fp32: backward error of the fp32 contractions, about sqrt(m) eps ||M||
    tol = 1e-11 if dt == torch.float64 else 1e-5 * max(1.0, (m / 150) ** 0.5)
    assert np.max(np.abs(s - s_ref)) <= tol * s_ref[0]
    U, V = host(U), host(V)
    assert np.max(np.abs(U @ np.diag(s) @ V.T - A)) <= 10 * tol * s_ref[0]
    assert np.max(np.abs(V.T @ V - np.eye(n))) <= 10 * tol


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_svd_truncated_top_values(h, dt):
    rng = np.random.default_rng(6)
    m, n, r = 300, 120, 6
    A = rng.normal(size=(m, r)) @ rng.normal(size=(r, n)) * 3 + 0.01 * rng.normal(size=(m, n))
    U, s, V = h.svd(dev(A, dt), k=r + 6, q=4)
    s_ref = np.linalg.svd(A, compute_uv=False)
    tol = 1e-9 if dt == torch.float64 else 1e-5
    assert np.max(np.abs(s[:r] - s_ref[:r])) <= tol * s_ref[0]


# ----------------------------------------------------------------------------
# one hot-path step vs the oracle step
# ----------------------------------------------------------------------------

def _state(m, n, mask, rng, rk=4, rp=3):
    obs = np.ones((m, n), bool) if mask is None else mask
    Ak, Bk = rng.normal(size=(m, rk)), rng.normal(size=(n, rk))
    Ap, Bp = rng.normal(size=(m, rp)), rng.normal(size=(n, rp))
    Sk = np.where(obs & (rng.random((m, n)) < 0.2), rng.normal(size=(m, n)) * 3, 0.0)
    Sp = np.where(obs & (rng.random((m, n)) < 0.2), rng.normal(size=(m, n)) * 3, 0.0)
    return Ak, Bk, Ap, Bp, Sk, Sp


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,hv,masked,beta", [
    (150, 130, 1, True, 0.35),   # ragged tiles, odd coarse width 65
    (150, 80, 0, False, 0.0),    # fine level, no momentum
    (200, 200, 2, False, 0.5),   # config-1 shape, two halvings
    (97, 70, 2, True, 0.2),      # ragged in both dimensions, odd sizes on the way
    (300, 256, 3, True, 0.6),    # several tiles, three halvings
])
def test_step_matches_oracle(cp, h, dt, m, n, hv, masked, beta):
    rng = np.random.default_rng(m * 7 + n + hv)
    p = W.planted_cpcp(m, n, 5, 0.1, 0.8 if masked else 1.0, seed=m + n)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    Ak, Bk, Ap, Bp, Sk, Sp = _state(m, n, mask, rng)
    mu_k = 0.25 * oracle.spectral_norm(D)
    S_ref, L_ref, r_ref = oracle.step(D, mask, lam, mu_k, beta, hv, Sk, Sp, Ak @ Bk.T, Ap @ Bp.T)
    k = oracle.coarse_dim(n, hv)  # full coarse width: the subspace SVD is exact
    Qb = None if mask is None else torch.as_tensor(cp.pack_mask(mask)).cuda()
    S1, A1, B1, r, sig = h.step(dev(D, dt), Qb, lam, mu_k, beta, hv, dev(Sk, dt), dev(Sp, dt), dev(Ak, dt),
                                dev(Bk, dt), Ak.shape[1], dev(Ap, dt), dev(Bp, dt), Ap.shape[1], k=k, q=2)
    S1 = host(S1)
    L1 = host(A1) @ host(B1).T
    assert r == r_ref
    if dt == torch.float64:
        assert rel(S1, S_ref) <= 1e-11 and rel(L1, L_ref) <= 1e-10
    else:
        assert rel(S1, S_ref) <= 2e-6 and rel(L1, L_ref) <= 2e-5
        # support of S bit-exact where the shrink margin exceeds 1e-3
        Lh, Sh = Ak @ Bk.T + beta * (Ak @ Bk.T - Ap @ Bp.T), Sk + beta * (Sk - Sp)
        obs = np.ones((m, n), bool) if mask is None else mask
        X = Sh - 0.5 * np.where(obs, Lh + Sh - D, 0.0)
        th = 0.5 * lam * mu_k
        safe = np.abs(np.abs(X) - th) > 1e-3 * th
        assert np.array_equal((S1 != 0)[safe], (S_ref != 0)[safe])
    if mask is not None:
        assert np.all(S1[~mask] == 0)


# ----------------------------------------------------------------------------
# solver: optimum parity
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg1():
    p = W.config(1)
    ref = {lv: oracle.fista(p["D"], None, p["lam"], p["mu"], levels=lv, tol=1e-11)[:2] for lv in (1,)}
    return p, ref


@pytest.mark.parametrize("levels", [1, 2])
def test_solve_cfg1_fp64_matches_oracle(h, cfg1, levels):
    p, ref = cfg1
    Lr, Sr = ref[1]
    L, S, info = h.solve(dev(p["D"]), None, p["lam"], p["mu"], levels=levels, tol=1e-11)
    assert info["status"] == 0, info
    assert info["final_level"] == 0
    L, S = host(L), host(S)
    assert rel(L, Lr) <= 1e-8 and rel(S, Sr) <= 1e-8, (rel(L, Lr), rel(S, Sr))
    assert oracle.relkkt(p["D"], None, p["lam"], p["mu"], L, S) <= 1e-10


@pytest.mark.parametrize("levels", [1, 2])
def test_solve_cfg1_bench_tolerance(h, cfg1, levels):
    p, ref = cfg1
    L, S, info = h.solve(dev(p["D"]), None, p["lam"], p["mu"], levels=levels, tol=1e-6)
    assert info["status"] == 0 and info["relkkt"] <= 1e-6
    # the library's residual agrees with the oracle's definition
    r_or = oracle.relkkt(p["D"], None, p["lam"], p["mu"], host(L), host(S))
    assert abs(r_or - info["relkkt"]) <= 0.05 * r_or + 1e-9


@pytest.fixture(scope="module")
def small_cpcp():
    p = W.planted_cpcp(300, 260, 8, 0.1, 0.8, seed=2024, levels=2)
    L, S, info = oracle.fista(p["D"], p["mask"], p["lam"], p["mu"], levels=1, tol=1e-11)
    return p, L, S


@pytest.mark.parametrize("levels", [1, 2])
def test_solve_fp32_cpcp_matches_oracle(cp, small_cpcp, levels):
    # the fp32 path has a residual floor near 3.5e-7 on this problem; solve to
    # (or up to 600 iterations at) 4e-7 and compare with the fp64 optimum
    p, Lr, Sr = small_cpcp
    Qb = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0, max_iter=600) as hh:
        L, S, info = hh.solve(dev(p["D"], torch.float32), Qb, p["lam"], p["mu"], levels=levels, tol=4e-7)
    assert info["status"] in (0, 5) and info["relkkt"] <= 5e-7, info
    L, S = host(L), host(S)
    eL, eS = rel(L, Lr), rel(S, Sr)
    print(f"fp32 levels={levels}: rel err L {eL:.3e} S {eS:.3e} relkkt {info['relkkt']:.3e} iters {info['iters']}")
    assert eL <= 1e-6 and eS <= 1e-6
    assert np.all(S[~p["mask"]] == 0)


@pytest.mark.parametrize("levels", [1, 2])
def test_solve_fp64_cpcp_masked_nan_offmask(cp, h, small_cpcp, levels):
    p, Lr, Sr = small_cpcp
    D = p["D"].copy()
    D[~p["mask"]] = np.nan  # unobserved entries are never used
    Qb = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    L, S, info = h.solve(dev(D), Qb, p["lam"], p["mu"], levels=levels, tol=1e-10)
    assert info["status"] == 0, info
    L, S = host(L), host(S)
    assert rel(L, Lr) <= 1e-7 and rel(S, Sr) <= 1e-7


def test_solve_wide_transposed(cp, h):
    p = W.planted_cpcp(90, 150, 3, 0.08, 0.85, seed=77, levels=2)
    Lr, Sr, _ = oracle.fista(p["D"], p["mask"], p["lam"], p["mu"], levels=1, tol=1e-11)
    Qb = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    L, S, info = h.solve(dev(p["D"]), Qb, p["lam"], p["mu"], levels=2, tol=1e-10)
    assert info["status"] == 0, info
    assert rel(host(L), Lr) <= 1e-7 and rel(host(S), Sr) <= 1e-7


def test_solve_host_buffers_equal_device(cp, h):
    p = W.planted_cpcp(120, 100, 4, 0.1, 0.9, seed=78, levels=2)
    Qh = cp.pack_mask(p["mask"])
    Dh = np.ascontiguousarray(p["D"].astype(np.float32))
    L1, S1, i1 = h.solve(Dh, Qh, p["lam"], p["mu"], levels=2, tol=1e-6)
    L2, S2, i2 = h.solve(dev(p["D"], torch.float32), torch.as_tensor(Qh).cuda(), p["lam"], p["mu"], levels=2,
                         tol=1e-6)
    assert i1["iters"] == i2["iters"]
    assert np.array_equal(L1, host(L2).astype(np.float32)) and np.array_equal(S1, host(S2).astype(np.float32))


def test_solve_is_deterministic(cp, h, small_cpcp):
    p, _, _ = small_cpcp
    Qb = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    D = dev(p["D"], torch.float32)
    L1, S1, _ = h.solve(D, Qb, p["lam"], p["mu"], levels=2, tol=1e-6)
    L2, S2, _ = h.solve(D, Qb, p["lam"], p["mu"], levels=2, tol=1e-6)
    assert torch.equal(L1, L2) and torch.equal(S1, S2)


# ----------------------------------------------------------------------------
# error handling
# ----------------------------------------------------------------------------

def test_invalid_arguments_and_nonfinite(cp, h):
    D = dev(np.random.default_rng(1).normal(size=(40, 30)))
    with pytest.raises(cp.CPCPError) as e:
        h.solve(D, None, -1.0, 1.0)
    assert e.value.status == 1
    with pytest.raises(cp.CPCPError) as e:
        h.solve(D, None, 0.1, 1.0, levels=7)
    assert e.value.status == 1
    with pytest.raises(cp.CPCPError) as e:  # zero tolerance
        h.solve(D, None, 0.1, 1.0, tol=0.0)
    assert e.value.status == 1
    Dn = D.clone()
    Dn[3, 4] = float("nan")
    with pytest.raises(cp.CPCPError) as e:
        h.solve(Dn, None, 0.1, 1.0)
    assert e.value.status == 2
    # the handle stays usable
    L, S, info = h.solve(D, None, 0.2, 0.05, tol=1e-6)
    assert info["status"] == 0


def test_iteration_cap_returns_not_converged(cp):
    with cp.Handle(0, max_iter=15) as hh:
        p = W.config(1)
        L, S, info = hh.solve(dev(p["D"]), None, p["lam"], p["mu"], tol=1e-12)
        assert info["status"] == 5 and info["iters"] == 15
        assert torch.isfinite(L).all() and torch.isfinite(S).all()


def test_graph_replay_equals_plain_launches(cp, small_cpcp):
    # the iterations replayed from a captured CUDA graph run the same kernels
    # on the same data as direct launches: bit-identical results, and the
    # same launch count with the residual checks in order (overlapped checks
    # also launch the iterations they drop: tests/test_gpu_check_overlap.py)
    p, _, _ = small_cpcp
    Qb = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    D = dev(p["D"], torch.float32)
    out = []
    for plain in (0, 1):
        with cp.Handle(0, plain_launches=plain, check_serial=1) as hh:
            L, S, info = hh.solve(D, Qb, p["lam"], p["mu"], levels=2, tol=1e-6)
        out.append((L, S, info))
    (L0, S0, i0), (L1, S1, i1) = out
    assert i0["iters"] == i1["iters"] and i0["launches"] == i1["launches"]
    assert torch.equal(L0, L1) and torch.equal(S0, S1)
