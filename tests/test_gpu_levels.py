"""GPU parity of the level rule: the coarse-gradient test (move one level finer
when ||G R||_F < kappa ||G||_F) run after the first iteration on each coarse
level as well as every check_every iterations (option early_test, default on),
against the fp64 oracle's same rule (oracle.fista(early_test=True)).

Gaussian factors (no coarse structure, Assumption 3 fails): both hand over
after one iteration on each coarse level.  Smooth video-shaped data with the
orthonormal transfer: both keep the coarsest level for at least one decision
period.  Either way the solve ends on the fine level at the single-level
optimum of eq. (cpcp).
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


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_gaussian_factors_hand_over_at_once(cp):
    p = W.planted_cpcp(240, 200, 5, 0.1, 0.8, seed=3, levels=3)
    D, mask, lam, mu = p["D"], p["mask"], p["lam"], p["mu"]
    L1, S1, _ = oracle.fista(D, mask, lam, mu, levels=1, tol=1e-10)
    _, _, ie = oracle.fista(D, mask, lam, mu, levels=3, tol=1e-8, early_test=True)
    Qb = torch.as_tensor(cp.pack_mask(mask)).cuda()
    with cp.Handle(0) as h:
        L, S, info = h.solve(dev(D), Qb, lam, mu, levels=3, tol=1e-10)
    assert info["status"] == 0 and info["final_level"] == 0, info
    assert list(info["level_iters"][1:3]) == list(ie["level_iters"][1:3]) == [1, 1]
    L, S = L.cpu().numpy(), S.cpu().numpy()
    assert rel(L, L1) <= 1e-7 and rel(S, S1) <= 1e-7
    # the rule of the periodic test alone keeps each coarse level for a decision period
    with cp.Handle(0, early_test=-1) as h:
        _, _, late = h.solve(dev(D), Qb, lam, mu, levels=3, tol=1e-10)
    assert late["level_iters"][2] >= 10 and late["level_iters"][1] >= 10


def test_gaussian_factors_fp32_bench_shape_hands_over_at_once(cp):
    # the 2000 x 2000 rank-50 workload: the first decision on each coarse level hands over
    p = W.planted_cpcp(2000, 2000, 50, 0.10, 0.8, 2000, levels=3)
    Qb = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0) as h:
        _, _, info = h.solve(dev(p["D"], torch.float32), Qb, p["lam"], p["mu"], levels=3, tol=1e-6)
    assert info["status"] == 0 and list(info["level_iters"][1:3]) == [1, 1], info


def test_smooth_data_keep_the_coarse_levels(cp):
    v = W.video_cpcp(7, h=16, w=24, frames=64, rank=2, blocks=3, block=4, obs=0.8, levels=3)
    D, mask, lam, mu = v["D"], v["mask"], v["lam"], v["mu"]
    L1, S1, _ = oracle.fista(D, mask, lam, mu, levels=1, tol=1e-10)
    _, _, iv = oracle.fista(D, mask, lam, mu, levels=3, tol=1e-8, transfer="orth", early_test=True)
    Qb = torch.as_tensor(cp.pack_mask(mask)).cuda()
    with cp.Handle(0, transfer=1) as h:
        L, S, info = h.solve(dev(D), Qb, lam, mu, levels=3, tol=1e-10)
    assert info["status"] == 0 and info["final_level"] == 0, info
    assert iv["level_iters"][2] >= 10 and info["level_iters"][2] >= 10
    L, S = L.cpu().numpy(), S.cpu().numpy()
    assert rel(L, L1) <= 1e-7 and rel(S, S1) <= 1e-7


def test_early_test_option_is_validated(cp):
    D = dev(np.random.default_rng(1).normal(size=(40, 30)))
    with cp.Handle(0, early_test=2) as h:
        with pytest.raises(cp.CPCPError) as e:
            h.solve(D, None, 0.1, 1.0)
    assert e.value.status == 1


@pytest.mark.parametrize("profile", [1, 2])
def test_level_times_add_up(cp, profile):
    # the per-level device times of a profiled solve: positive exactly on the
    # levels that ran iterations, and together the iterations' pass and SVT
    # phase times (residual checks are not counted at any level)
    v = W.video_cpcp(7, h=16, w=24, frames=64, rank=2, blocks=3, block=4, obs=0.8, levels=3)
    Qb = torch.as_tensor(cp.pack_mask(v["mask"])).cuda()
    with cp.Handle(0, transfer=1, profile=profile) as h:
        _, _, info = h.solve(dev(v["D"], torch.float32), Qb, v["lam"], v["mu"], levels=3, tol=1e-6)
    assert info["status"] == 0, info
    lm, li = info["level_ms"], info["level_iters"]
    for lv in range(8):
        assert (lm[lv] > 0) == (li[lv] > 0), (lm, li)
    ph = info["phase_ms"]
    tot = ph["pass_coarse"] + ph["pass_fine"] + ph["svt"]
    assert abs(sum(lm) - tot) <= 1e-9 * max(tot, 1.0) + 1e-6, (lm, ph)
