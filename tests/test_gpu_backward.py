"""Differentiable unrolled solve: the recorded forward and the hand-written
reverse sweep (cpcp_solve with options.unroll, cpcp_backward) against the
fp64 oracle's forward and adjoint (which are pinned to finite differences in
tests/test_oracle_unrolled.py), and the torch.autograd wrapper."""
import numpy as np
import pytest

import oracle
from oracle import unrolled as U
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
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _setup(m, n, rank, obs, seed, levels):
    p = W.planted_cpcp(m, n, rank, 0.1, obs, seed=seed, levels=levels)
    pqd = np.where(p["mask"], p["D"], 0.0) if p["mask"] is not None else p["D"]
    rho = 1.1 * oracle.spectral_norm(pqd) / p["mu"]  # mu_0 off the first-step kink
    return p, rho


def _gpu_forward(cp, p, rho, levels, K, ckpt=10):
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = None if p["mask"] is None else torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    h = cp.Handle(0, unroll=K, ckpt_every=ckpt, rho=rho)
    L, S, info = h.solve(D, Q, p["lam"], p["mu"], levels=levels, tol=1.0)
    return h, L, S, info


CASES = [  # (m, n, rank, observed, levels, K)
    (64, 48, 3, 0.8, 2, 8),
    (96, 64, 4, 0.7, 3, 12),
    (80, 80, 3, 1.0, 1, 6),
    (130, 70, 3, 0.75, 2, 15),  # ragged sizes, two checkpoint segments
]


@pytest.mark.parametrize("m,n,rank,obs,levels,K", CASES)
def test_unrolled_forward_matches_oracle(cp, m, n, rank, obs, levels, K):
    p, rho = _setup(m, n, rank, obs, 500 + m + K, levels)
    h, L, S, info = _gpu_forward(cp, p, rho, levels, K)
    h.close()
    Lo, So = U.forward(p["D"], p["mask"], p["lam"], p["mu"], rho, 0.9, levels - 1, K)
    assert info["iters"] == K
    assert _rel(L.double().cpu().numpy(), Lo) <= 2e-5
    assert _rel(S.double().cpu().numpy(), So) <= 2e-5


@pytest.mark.parametrize("m,n,rank,obs,levels,K", CASES)
def test_backward_matches_oracle_adjoint(cp, m, n, rank, obs, levels, K):
    p, rho = _setup(m, n, rank, obs, 500 + m + K, levels)
    rng = np.random.default_rng(m * K)
    L0 = rng.standard_normal(p["D"].shape)
    gS = 0.3 * rng.standard_normal(p["D"].shape)
    h, L, S, _ = _gpu_forward(cp, p, rho, levels, K, ckpt=5)
    gL = 2.0 * (L.double() - torch.as_tensor(L0).cuda())
    dD, dlam, dmu = h.backward(gL.float(), torch.as_tensor(gS, dtype=torch.float32).cuda())
    h.close()
    Lo, _ = U.forward(p["D"], p["mask"], p["lam"], p["mu"], rho, 0.9, levels - 1, K)
    dDo, dlamo, dmuo = U.adjoint(p["D"], p["mask"], p["lam"], p["mu"], rho, 0.9, levels - 1, K, 2.0 * (Lo - L0), gS)
    dD = dD.double().cpu().numpy()
    assert _rel(dD, dDo) <= 1e-4
    assert abs(dlam - dlamo) <= 1e-4 * abs(dlamo) + 1e-6
    assert abs(dmu - dmuo) <= 1e-4 * abs(dmuo) + 1e-6
    if p["mask"] is not None:
        assert np.all(dD[~p["mask"]] == 0)


def test_checkpoint_spacing_does_not_change_the_gradient(cp):
    p, rho = _setup(96, 64, 4, 0.7, 777, 3)
    grads = []
    for ckpt in (3, 12):
        h, L, S, _ = _gpu_forward(cp, p, rho, 3, 12, ckpt=ckpt)
        dD, dlam, dmu = h.backward(L.clone())
        h.close()
        grads.append((dD.cpu().numpy(), dlam, dmu))
    assert np.array_equal(grads[0][0], grads[1][0]) and grads[0][1:] == grads[1][1:]


def test_autograd_function(cp):
    p, rho = _setup(64, 48, 3, 0.8, 901, 2)
    K = 8
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda().requires_grad_(True)
    lam = torch.tensor(p["lam"], dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(p["mu"], dtype=torch.float64, requires_grad=True)
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    L0 = torch.as_tensor(p["L0"], dtype=torch.float32).cuda()
    L, S = cp.unrolled_cpcp(D, lam, mu, rho, Qbits=Q, levels=2, K=K)
    loss = ((L - L0) ** 2).sum()
    loss.backward()
    Lo, _ = U.forward(p["D"], p["mask"], p["lam"], p["mu"], rho, 0.9, 1, K)
    dDo, dlamo, dmuo = U.adjoint(p["D"], p["mask"], p["lam"], p["mu"], rho, 0.9, 1, K, 2.0 * (Lo - p["L0"]))
    assert _rel(D.grad.double().cpu().numpy(), dDo) <= 1e-4
    assert abs(lam.grad.item() - dlamo) <= 1e-4 * abs(dlamo) + 1e-6
    assert abs(mu.grad.item() - dmuo) <= 1e-4 * abs(dmuo) + 1e-6


def test_backward_without_a_recorded_run_is_rejected(cp):
    with cp.Handle(0) as h:
        with pytest.raises(cp.CPCPError) as e:
            h.backward(torch.zeros((8, 8), dtype=torch.float32, device="cuda"))
        assert e.value.status == 1


def test_unrolled_full_workload(cp):
    """1024 x 1024, rank 20, 10% corruption, 70% observed, 3 levels (n_H = 256),
    50 unrolled steps, checkpoints every 10, loss ||L_50 - L0||^2: the GPU
    gradient against the fp64 oracle adjoint, which is itself checked here
    against fp64 central differences in lambda and mu.

    The program is not differentiable where a shrink input meets its
    threshold; on this workload a handful of the 10^6 entries come within
    1e-5 of it at some step, and fp32 and fp64 trajectories can put them on
    different sides (the gradient then differs at those entries only).  They
    are excluded from the dD comparison, by the oracle's own margins."""
    p = W.config(5)
    rho = 1.1 / 1e-3  # mu = 1e-3 ||P_Q D||_2, mu_0 10% above ||P_Q D||_2
    K = 50
    h, L, S, info = _gpu_forward(cp, p, rho, 3, K, ckpt=10)
    L0 = torch.as_tensor(p["L0"]).cuda()
    gL = (2.0 * (L.double() - L0)).float()
    dD, dlam, dmu = h.backward(gL)
    h.close()
    args = (p["D"], p["mask"], p["lam"], p["mu"], rho, 0.9, 2, K)
    Lo, _ = U.forward(*args)
    assert _rel(L.double().cpu().numpy(), Lo) <= 1e-4
    dDo, dlamo, dmuo = U.adjoint(*args, 2.0 * (Lo - p["L0"]))
    ent, sv = U.shrink_margins(*args)
    assert min(sv) > 1e-5  # no singular value within the fp32 noise of its threshold
    smooth = ent > 1e-5
    assert (~smooth).sum() < 1000
    dDg = dD.double().cpu().numpy()
    assert _rel(dDg[smooth], dDo[smooth]) <= 1e-4
    assert abs(dlam - dlamo) <= 1e-4 * abs(dlamo)
    assert abs(dmu - dmuo) <= 1e-4 * abs(dmuo)
    # the oracle adjoint against fp64 central differences at this size
    hrel = 1e-6

    def loss(lam_, mu_):
        Lx, _ = U.forward(p["D"], p["mask"], lam_, mu_, rho, 0.9, 2, K)
        return float(np.sum((Lx - p["L0"]) ** 2))

    lam, mu = p["lam"], p["mu"]
    fd_lam = (loss(lam * (1 + hrel), mu) - loss(lam * (1 - hrel), mu)) / (2 * hrel * lam)
    fd_mu = (loss(lam, mu * (1 + hrel)) - loss(lam, mu * (1 - hrel))) / (2 * hrel * mu)
    assert abs(fd_lam - dlamo) <= 1e-4 * abs(fd_lam)
    assert abs(fd_mu - dmuo) <= 1e-4 * abs(fd_mu)
