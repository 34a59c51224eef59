"""The hyperspectral-shaped workload (pixels x bands, smooth spectra): the
fp32 CUDA solve against the fp64 oracle, single-level and multilevel."""
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


def _solve(cp, p, levels, tol=1e-6):
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0, max_iter=800) as h:
        L, S, info = h.solve(D, Q, p["lam"], p["mu"], levels=levels, tol=tol)
    return L.double().cpu().numpy(), S.double().cpu().numpy(), info


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_small_hyperspectral_matches_oracle_optimum(cp, levels):
    p = W.hyperspectral_cpcp(7, h=32, w=32, bands=64, rank=5, levels=levels)
    Lr, Sr, _ = oracle.fista(p["D"], p["mask"], p["lam"], p["mu"], levels=1, tol=1e-9)
    L, S, info = _solve(cp, p, levels)
    assert info["status"] == 0, info
    assert oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], L, S) <= 2e-6
    assert _rel(L, Lr) <= 1e-4 and _rel(S, Sr) <= 1e-3
    assert np.all(S[~p["mask"]] == 0)


def test_full_hyperspectral_multilevel_and_single(cp):
    # 65536 pixels x 128 bands, rank 8: both solves reach the tolerance, the
    # oracle's fp64 residual confirms it, and the ranks agree with the plant
    p = W.config(6)
    out = {}
    for lv in (3, 1):
        L, S, info = _solve(cp, p, lv)
        assert info["status"] == 0, info
        assert info["rank"] == 8
        assert oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], L, S) <= 2e-6
        out[lv] = (L, S)
    assert _rel(out[3][0], out[1][0]) <= 1e-4
