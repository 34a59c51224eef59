"""GPU parity of the alternative forms of the iteration's subspace SVD (fp32):
the Cholesky of CholeskyQR by 16-column block rows (chol_form 0; the
compact unblocked form for widths up to 32) or one elimination step per
barrier (1: registers, 2: shared memory); the core Jacobi rounds with 16 or 8
lanes per column pair; the iteration's SVD on two streams with
Z = (M^T Y) R_Y^{-1} (svd_serial 0 and 2) or in order with Z = M^T Q_Y (1);
Gram matrices of tall blocks by row ranges (gram_form 0) or by 64 x 64 tiles
(1).  Every form solves eq. (cpcp) to the fp64 oracle's optimum (FISTA with
Alg. 4's coarse step), and the forms agree with each other at the fp32 level.
"""
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def solve(cp, p, levels, tol, **opts):
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0, max_iter=600, **opts) as h:
        L, S, info = h.solve(D, Q, p["lam"], p["mu"], levels=levels, tol=tol)
    torch.cuda.synchronize()
    return L.double().cpu().numpy(), S.double().cpu().numpy(), info


@pytest.fixture(scope="module", params=[(8, 0.1, 0.8), (24, 0.05, 0.9)])
def small(request):
    # 300 x 260 (SIMT products, tiled Gram matrices): ragged tiles, masked;
    # rank 8 gives a subspace width k = 18 (the compact Cholesky of form 0),
    # rank 24 k = 34 (its blocked form)
    rank, corr, obs = request.param
    p = W.planted_cpcp(300, 260, rank, corr, obs, seed=2024, levels=2)
    L, S, _ = oracle.fista(p["D"], p["mask"], p["lam"], p["mu"], levels=1, tol=1e-10 if rank > 8 else 1e-11)
    return p, L, S


@pytest.fixture(scope="module")
def tall():
    # 4096 x 96: tensor-core products, Gram matrices of Y by row ranges, and
    # M^T Y small enough (64 CTAs) for the two-stream form.  (The oracle needs
    # about a minute to solve it, so its optimality is checked through the
    # oracle's fp64 residual of each result over the whole matrix instead.)
    return W.planted_cpcp(4096, 96, 4, 0.1, 0.8, seed=77, levels=2)


@pytest.mark.parametrize("svd_serial", [0, 1, 2])
@pytest.mark.parametrize("chol_form", [0, 1, 2])
@pytest.mark.parametrize("levels", [1, 2])
def test_forms_match_oracle_small(cp, small, svd_serial, chol_form, levels):
    p, Lr, Sr = small
    L, S, info = solve(cp, p, levels, 4e-7, svd_serial=svd_serial, chol_form=chol_form)
    assert info["status"] in (0, 5) and info["relkkt"] <= 5e-7, info
    eL, eS = rel(L, Lr), rel(S, Sr)
    print(f"svd_serial={svd_serial} chol_form={chol_form} levels={levels}: L {eL:.2e} S {eS:.2e} "
          f"iters {info['iters']} chol {info['chol_factors']}")
    assert eL <= 1e-6 and eS <= 1e-6
    assert np.all(S[~p["mask"]] == 0)


@pytest.mark.parametrize("levels", [1, 2])
def test_forms_tall_oracle_residual_and_agreement(cp, tall, levels):
    p = tall
    ref = None
    for opts in ({"svd_serial": 1, "chol_form": 1, "gram_form": 1}, {}, {"svd_serial": 2},
                 {"chol_form": 1, "gram_form": 1}, {"chol_form": 2, "jacobi_lanes": 8}):
        L, S, info = solve(cp, p, levels, 1e-6, **opts)
        assert info["status"] == 0, (opts, info)
        r = oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], L, S)
        print(f"{opts} levels={levels}: iters {info['iters']} relkkt {info['relkkt']:.2e} oracle {r:.2e}")
        assert r <= 1.5e-6
        assert np.all(S[~p["mask"]] == 0)
        if ref is None:
            ref = (L, S)
        else:
            assert rel(L, ref[0]) <= 1e-5 and rel(S, ref[1]) <= 1e-5, opts


def test_forms_reject_bad_values(cp):
    p = W.planted_cpcp(64, 48, 2, 0.1, 0.8, seed=1, levels=1)
    for opts in ({"svd_serial": 3}, {"chol_form": 3}, {"gram_form": -1}, {"jacobi_lanes": 4}, {"pdl_off": 2},
                 {"jacobi_check": 2}):
        with pytest.raises(cp.CPCPError):
            solve(cp, p, 1, 1e-6, **opts)


@pytest.mark.parametrize("svd_serial", [0, 1])
def test_pdl_results_bit_identical(cp, tall, svd_serial):
    # programmatic dependent launch changes only when kernels start, never
    # what they compute: the results match the in-order launches bit for bit
    p = tall
    L0, S0, i0 = solve(cp, p, 2, 1e-6, svd_serial=svd_serial, pdl_off=1)
    L1, S1, i1 = solve(cp, p, 2, 1e-6, svd_serial=svd_serial)
    assert i0["status"] == 0 and i1["status"] == 0
    assert i0["iters"] == i1["iters"]
    assert np.array_equal(L0, L1) and np.array_equal(S0, S1)
