"""The fine residual check run on a second stream, from a copy of the checked
iterate, while the solve stream computes the next iterations (option
check_serial = 0, the default with graph replay) against the same solve with
every check run in order (check_serial = 1): the iterates, the decisions and
the result must not change.  Bit-identical L and S, and the same iteration,
check and level counts and residual, on solves that stop at a check, that run
out of iterations between checks, on the mixed-precision path (checks in
order until the fp32 refinement, overlapped after it), in fp64, and with the
phase profile on.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2206_13369_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_13369_gb300 import build
    build.build()
    from paper_2206_13369_gb300 import cpcp
    return cpcp


def solve_pair(cp, D, Q, lam, mu, levels, tol, **opts):
    out = []
    for serial in (1, 0):
        with cp.Handle(0, check_serial=serial, **opts) as h:
            L, S, info = h.solve(D, Q, lam, mu, levels=levels, tol=tol)
            torch.cuda.synchronize()
        out.append((L.cpu(), S.cpu(), info))
    return out


def assert_same(a, b):
    (L1, S1, i1), (L2, S2, i2) = a, b
    for key in ("status", "iters", "level_iters", "final_level", "rank", "checks", "relkkt", "bf16_iters"):
        assert i1[key] == i2[key], (key, i1[key], i2[key])
    assert torch.equal(L1, L2) and torch.equal(S1, S2)


@pytest.mark.parametrize("levels", [1, 3])
def test_overlap_same_result_bench_workload(cp, levels):
    p = W.config(2)
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    a, b = solve_pair(cp, D, Q, p["lam"], p["mu"], levels, 1e-6)
    assert a[2]["status"] == 0 and a[2]["checks"] >= 2
    assert_same(a, b)


def test_overlap_same_result_when_iterations_run_out(cp):
    # max_iter two and one iterations after a check (the weight is final from
    # iteration 66, checks every 10): the iterations computed beside the last
    # check are the solve's last ones
    p = W.config(2)
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    for max_iter in (72, 81):
        a, b = solve_pair(cp, D, Q, p["lam"], p["mu"], 1, 1e-9, max_iter=max_iter)
        assert a[2]["iters"] == max_iter and a[2]["status"] != 0
        assert_same(a, b)


def test_overlap_same_result_mixed_precision(cp):
    v = W.config(3)
    D = torch.as_tensor(v["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(v["mask"])).cuda()
    a, b = solve_pair(cp, D, Q, v["lam"], v["mu"], 1, 1e-6, precision=1)
    assert a[2]["status"] == 0 and a[2]["bf16_iters"] > 0
    assert_same(a, b)


def test_overlap_same_result_fp64_and_profiled(cp):
    p = W.planted_cpcp(300, 260, 6, 0.1, 0.8, 11, levels=2)
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    D = torch.as_tensor(p["D"], dtype=torch.float64).cuda()
    a, b = solve_pair(cp, D, Q, p["lam"], p["mu"], 2, 1e-9)
    assert a[2]["status"] == 0
    assert_same(a, b)
    Df = D.float()
    a, b = solve_pair(cp, Df, Q, p["lam"], p["mu"], 2, 1e-6, profile=1)
    assert_same(a, b)
    # the profiled times count only the iterations that count
    for _, _, info in (a, b):
        assert info["phase_count"]["pass_fine"] == info["level_iters"][0]
