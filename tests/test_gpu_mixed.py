"""Mixed-precision path: tensor-core BF16 contractions of the subspace
iteration, the SVD built on them, and mixed-precision solves against the
oracle (video-shaped workloads, relative Frobenius tolerance 1e-4)."""
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


def bf16_round(x):
    """Round fp32 values to the nearest BF16 (ties to even), kept as fp32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def test_bf16_round_helper():
    # 1 + 2^-8 lies halfway between two BF16 values: ties to even keeps 1
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e-3], dtype=np.float32)
    r = bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -6 and r[3] == -2.5
    assert abs(r[4] - 3.0e-3) <= 3.0e-3 * 2.0 ** -8


@pytest.mark.parametrize("rows,K,N", [
    (300, 130, 15),     # ragged in rows, K and N
    (2000, 500, 60),    # coarse Y = M_H Omega of the 2000 x 2000 workload
    (50, 19200, 16),    # Z = M_H^T Q of the video workload: long K, split-K
    (1, 1, 1),          # smallest
    (129, 65, 17),      # one past each tile edge
    (1000, 64, 128),
    (257, 1000, 256),   # widest N
])
def test_gemm_bf16_matches_exact_product(cp, rows, K, N):
    rng = np.random.default_rng(rows * 7 + K * 3 + N)
    A = rng.standard_normal((rows, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    with cp.Handle(0) as h:
        Cd = h.gemm_bf16(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy().astype(np.float64)
        Cd2 = h.gemm_bf16(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy().astype(np.float64)
    Ar, Br = bf16_round(A).astype(np.float64), bf16_round(B).astype(np.float64)
    exact = Ar @ Br.T
    scale = np.abs(Ar) @ np.abs(Br).T
    u = 2.0 ** -24
    # products of BF16 values are exact in fp32; only the fp32 sums round
    assert np.all(np.abs(Cd - exact) <= 4 * u * np.sqrt(K) * scale + 1e-30)
    assert np.array_equal(Cd, Cd2)  # fixed-order split-K reduction
    # and it is far from the unrounded product, so BF16 really was used
    if K >= 64:
        assert np.abs(Cd - A.astype(np.float64) @ B.astype(np.float64).T).max() > 1e3 * u * np.sqrt(K) * scale.max() / K


def test_gemm_bf16_rejects_bad_arguments(cp):
    A = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    B = torch.zeros((300, 4), dtype=torch.float32, device="cuda")
    with cp.Handle(0) as h:
        with pytest.raises(cp.CPCPError) as e:
            h.gemm_bf16(A, B)  # N = 300 > 256
        assert e.value.status == 1


def test_svd_mixed_spectrum(cp):
    rng = np.random.default_rng(11)
    m, n, k = 1200, 300, 24
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.concatenate([np.geomspace(1.0, 0.1, 10), np.geomspace(1e-3, 1e-5, n - 10)])
    M = ((U * s) @ V.T).astype(np.float32)
    Md = torch.from_numpy(M).cuda()
    with cp.Handle(0, precision=1) as h:
        Ub, sb, Vb = h.svd(Md, k, q=3)
    with cp.Handle(0) as h:
        Uf, sf, Vf = h.svd(Md, k, q=3)
    # BF16 rounding of M moves singular values by at most ||M_bf16 - M||_2
    pert = np.linalg.norm(bf16_round(M).astype(np.float64) - M.astype(np.float64), 2)
    assert np.all(np.abs(sb[:10] - s[:10]) <= 4 * pert + 2e-3 * s[:10])
    assert np.all(np.abs(sf[:10] - s[:10]) <= 1e-4 * s[0])
    # the leading vectors agree with the fp32 ones
    Ub, Uf = Ub.cpu().numpy(), Uf.cpu().numpy()
    assert np.all(np.abs(np.abs(np.sum(Ub[:, :5] * Uf[:, :5], 0)) - 1) < 1e-3)


def _solve(cp, p, levels, tol=1e-6, **opts):
    D = torch.as_tensor(p["D"], dtype=torch.float32).cuda()
    Q = torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    with cp.Handle(0, max_iter=3000, **opts) as h:
        L, S, info = h.solve(D, Q, p["lam"], p["mu"], levels=levels, tol=tol)
    return L.double().cpu().numpy(), S.double().cpu().numpy(), info


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def small_video():
    p = W.video_cpcp(3000, h=24, w=32, frames=64, rank=3, blocks=3, block=4, levels=3)
    Lo, So, io = oracle.fista(p["D"], p["mask"], p["lam"], p["mu"], levels=1, tol=1e-9)
    assert io["status"] == 0
    return p, Lo, So


@pytest.mark.parametrize("levels", [3, 1])
def test_mixed_solve_matches_oracle_small_video(cp, small_video, levels):
    p, Lo, So = small_video
    # rel-KKT 1e-6 leaves about 1.2e-4 of L error on this problem (its
    # conditioning, not the precision); parity is checked at 2e-7, near the
    # fp32 floor of the residual (status 5 only if the floor stops it)
    L, S, info = _solve(cp, p, levels, tol=2e-7, precision=1)
    assert info["status"] in (0, 5) and info["relkkt"] <= 5e-7
    assert 0 < info["bf16_iters"] < info["iters"]
    assert _rel(L, Lo) <= 1e-4 and _rel(S, So) <= 1e-4
    # S vanishes off the mask exactly; its support agrees wherever the
    # optimum's shrink margin is clear of the solve tolerance
    assert np.all(S[~p["mask"]] == 0)
    th = 0.5 * p["lam"] * p["mu"]
    X = So - 0.5 * oracle.grad(p["D"], p["mask"], Lo, So)
    clear = np.abs(np.abs(X) - th) > 0.1 * th
    assert np.array_equal((S != 0)[clear], (So != 0)[clear])


def test_mixed_solve_video_full_size(cp):
    """19200 x 400 video-shaped CPCP, 4 levels: the mixed solve reaches the
    tolerance, agrees with the fp32 solve to 1e-4, and its residual
    recomputed in fp64 by the oracle is at the tolerance."""
    p = W.config(3)
    Lm, Sm, im = _solve(cp, p, 4, precision=1)
    Lf, Sf, inf = _solve(cp, p, 4)
    assert im["status"] == 0 and inf["status"] == 0
    assert im["bf16_iters"] > 0
    # two solutions at rel-KKT 1e-6 of a problem with condition ~1e2
    assert _rel(Lm, Lf) <= 1e-3 and _rel(Sm, Sf) <= 1e-3
    # optimality of the mixed solution, recomputed in fp64 by the oracle
    r = oracle.relkkt(p["D"], p["mask"], p["lam"], p["mu"], Lm, Sm)
    assert r <= 2e-6
