"""Frank-Wolfe Thresholding (Alg. 3) and ML-FWT (Alg. 6) for eq. (cpcp): the
CUDA path (cpcp_fwt) against the oracle's implementation.

With the subspace block as wide as the matrix (option oversample), the
subspace SVD behind the nuclear-ball LMO is exact, and the CUDA iterates must
follow the oracle's (its own Jacobi SVD) step by step in fp64: the same LMO
decisions, line-search steps and thresholding, so the same objective trace."""
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


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_fwt_fp64_matches_oracle(cp, levels):
    p = W.planted_cpcp(60, 40, 3, 0.1, 0.8, seed=5, levels=levels)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    mu = 0.05 * np.linalg.svd(np.where(mask, D, 0.0), compute_uv=False)[0]
    Lr, Sr, it_r, fr, _ = oracle.fwt(D, mask, lam, mu, levels=levels, max_iter=60, tol=0.0)
    Dt = torch.as_tensor(D).cuda()
    Qt = torch.as_tensor(cp.pack_mask(mask)).cuda()
    with cp.Handle(0, oversample=64, power_iters=2) as h:
        L, S, info = h.fwt(Dt, Qt, lam, mu, levels=levels, max_iter=60, tol=0.0)
    assert info["status"] == 5 and info["iters"] == it_r == 60
    assert np.allclose(info["f"], fr, rtol=1e-10, atol=0), np.abs(info["f"] / fr - 1).max()
    assert _rel(L.cpu().numpy(), Lr) <= 1e-8 and _rel(S.cpu().numpy(), Sr) <= 1e-8


def test_fwt_fp32_default_width(cp):
    # fp32 with the default block width (10 columns, one power pass per
    # iteration, warm started): an approximate LMO, so a trajectory of its own;
    # it descends, and after 300 iterations its objective gap to the optimum of
    # eq. (cpcp) is of the size of the exact-LMO fp64 oracle's
    p = W.planted_cpcp(200, 150, 3, 0.1, 0.8, seed=9, levels=1)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    mu = 0.05 * np.linalg.svd(np.where(mask, D, 0.0), compute_uv=False)[0]
    Lf, Sf, _ = oracle.fista(D, mask, lam, mu, levels=1, tol=1e-11)
    fstar = oracle.objective(D, mask, lam, mu, Lf, Sf)
    Lo, So, _, _, _ = oracle.fwt(D, mask, lam, mu, max_iter=300, tol=0.0)
    go = oracle.objective(D, mask, lam, mu, Lo, So) / fstar - 1.0
    Qt = torch.as_tensor(cp.pack_mask(mask)).cuda()
    with cp.Handle(0) as h:
        L, S, info = h.fwt(torch.as_tensor(D, dtype=torch.float32).cuda(), Qt, lam, mu, max_iter=300, tol=0.0)
    f = info["f"]
    assert info["status"] == 5 and len(f) == 300
    assert np.all(np.diff(f) <= 1e-5 * f[:-1])
    F = oracle.objective(D, mask, lam, mu, L.double().cpu().numpy(), S.double().cpu().numpy())
    assert F >= fstar * (1 - 1e-6) and F <= f[-1] * (1 + 1e-5)
    assert F / fstar - 1.0 <= 2.0 * go + 2e-3, (F / fstar - 1.0, go)


def test_fwt_stopping_rule(cp):
    p = W.planted_cpcp(60, 40, 3, 0.1, 0.8, seed=5, levels=1)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    mu = 0.05 * np.linalg.svd(np.where(mask, D, 0.0), compute_uv=False)[0]
    _, _, it_r, fr, _ = oracle.fwt(D, mask, lam, mu, max_iter=1000, tol=1e-3)
    with cp.Handle(0, oversample=64, power_iters=2) as h:
        _, _, info = h.fwt(torch.as_tensor(D).cuda(), torch.as_tensor(cp.pack_mask(mask)).cuda(), lam, mu,
                           max_iter=1000, tol=1e-3)
    assert info["status"] == 0 and info["iters"] == it_r < 1000
    assert abs(info["f"][-2] - info["f"][-1]) <= 1e-3 * info["f"][-2]


def test_fwt_rejects_host_buffers(cp):
    with cp.Handle(0) as h:
        with pytest.raises(cp.CPCPError) as e:
            h.fwt(np.ones((8, 6)), None, 0.1, 1.0)
        assert e.value.status == 1


@pytest.mark.parametrize("levels", [2, 3])
def test_ml_fwt_orthonormal_transfer_matches_oracle(cp, levels):
    # ML-FWT with an orthonormal basis of the range of R (option transfer = 1): the
    # library lifts by R C^{-1}, the oracle by R (R^T R)^{-1/2}; both bases span the
    # same range, so the lifted top singular vector, and with it every iterate, agree
    p = W.planted_cpcp(60, 40, 3, 0.1, 0.8, seed=5, levels=levels)
    D, mask, lam = p["D"], p["mask"], p["lam"]
    mu = 0.05 * np.linalg.svd(np.where(mask, D, 0.0), compute_uv=False)[0]
    Lr, Sr, it_r, fr, _ = oracle.fwt(D, mask, lam, mu, levels=levels, max_iter=60, tol=0.0, transfer="orth")
    Qt = torch.as_tensor(cp.pack_mask(mask)).cuda()
    with cp.Handle(0, oversample=64, power_iters=2, transfer=1) as h:
        L, S, info = h.fwt(torch.as_tensor(D).cuda(), Qt, lam, mu, levels=levels, max_iter=60, tol=0.0)
    assert info["status"] == 5 and info["iters"] == it_r == 60
    assert np.allclose(info["f"], fr, rtol=1e-9, atol=0), np.abs(info["f"] / fr - 1).max()
    assert _rel(L.cpu().numpy(), Lr) <= 1e-7 and _rel(S.cpu().numpy(), Sr) <= 1e-7
