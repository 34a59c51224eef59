"""The entry point that allocates nothing (cpcp_masked_norm_static).

Some callers cannot allocate device memory while they run: code whose device
memory is all handed out up front by its own pool or arena, and latency-critical
loops that cannot pay for cudaMalloc's device-wide synchronisation.  For them the library computes ||P_Q[D]||_F with its scratch in
a fixed static device array.  This test calls it through the C ABI, twice in a
row on each input (the scratch keeps the previous call's contents), and checks
it against the same quantity reported by the handle-based cpcp_solve.

The file is named so that pytest collects it last; it also runs on its own in
a fresh process (it builds and loads the library itself).
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


def _reference_norm(cp, D, Qb, lam, mu):
    # the existing entry point: cpcp_solve reports ||P_Q D||_F in its info
    with cp.Handle(0, max_iter=1) as h:
        _, _, info = h.solve(D, Qb, lam, mu, levels=1, tol=1e-6)
    return info["pqd_fro"]


@pytest.mark.parametrize("dt,m,n,obs", [
    (torch.float32, 300, 260, 0.8),   # several tiles and ragged edges, masked
    (torch.float64, 200, 200, 1.0),   # unmasked
    (torch.float32, 97, 70, 0.6),     # ragged in both dimensions
    (torch.float64, 1000, 130, 0.9),  # tall
])
def test_static_norm_matches_solver(cp, dt, m, n, obs):
    p = W.planted_cpcp(m, n, 4, 0.1, obs, seed=m + n)
    D = torch.as_tensor(p["D"], dtype=dt).cuda()
    Qb = None if p["mask"] is None else torch.as_tensor(cp.pack_mask(p["mask"])).cuda()
    ref = _reference_norm(cp, D, Qb, p["lam"], p["mu"])
    tol = 1e-6 if dt == torch.float32 else 1e-12
    first = cp.masked_norm_static(D, Qb)
    second = cp.masked_norm_static(D, Qb)
    assert first == second  # the shared scratch carries nothing over
    fro, nf = first
    assert nf == 0
    assert abs(fro - ref) <= tol * ref
    # exact value of the definition (fp64 on the host)
    x = np.where(p["mask"], D.double().cpu().numpy(), 0.0) if p["mask"] is not None else D.double().cpu().numpy()
    assert abs(fro - np.linalg.norm(x)) <= 1e-12 * np.linalg.norm(x)


def test_static_norm_smaller_after_larger_and_nonfinite(cp):
    big = W.planted_cpcp(400, 380, 3, 0.1, 0.7, seed=5)
    small = W.planted_cpcp(40, 33, 2, 0.1, 0.7, seed=6)
    Db = torch.as_tensor(big["D"], dtype=torch.float32).cuda()
    Qbb = torch.as_tensor(cp.pack_mask(big["mask"])).cuda()
    Ds = torch.as_tensor(small["D"], dtype=torch.float32).cuda()
    Qbs = torch.as_tensor(cp.pack_mask(small["mask"])).cuda()
    cp.masked_norm_static(Db, Qbb)
    fro_s, _ = cp.masked_norm_static(Ds, Qbs)
    ref = _reference_norm(cp, Ds, Qbs, small["lam"], small["mu"])
    assert abs(fro_s - ref) <= 1e-6 * ref
    # non-finite values count only where observed
    Dn = Ds.clone()
    obs = np.argwhere(small["mask"])[0]
    hid = np.argwhere(~small["mask"])[0]
    Dn[obs[0], obs[1]] = float("nan")
    Dn[hid[0], hid[1]] = float("inf")
    _, nf = cp.masked_norm_static(Dn, Qbs)
    assert nf == 1


def test_static_norm_tall_single_column_tile(cp):
    # one column tile and 65536 row tiles: the largest tile count the scratch takes,
    # with more row tiles than a grid's y dimension could hold (the tiles run on a
    # one-dimensional grid)
    m, n = 64 * 65535 + 1, 64
    g = torch.Generator(device="cuda").manual_seed(11)
    D = torch.randn((m, n), generator=g, device="cuda", dtype=torch.float32)
    ref = float(torch.linalg.vector_norm(D.double()))
    first = cp.masked_norm_static(D, None)
    second = cp.masked_norm_static(D, None)
    assert first == second
    fro, nf = first
    assert nf == 0
    assert abs(fro - ref) <= 1e-12 * ref
    del D


def test_static_norm_rejects_sizes_beyond_the_scratch(cp):
    D = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    # 65537 tiles of 64 x 64 do not fit the static scratch; rejected before any device work
    with pytest.raises(cp.CPCPError) as e:
        import ctypes
        fro = ctypes.c_double(0)
        st = cp.lib().cpcp_masked_norm_static(None, 64 * 65537, 64, cp.F32, D.data_ptr(), 64, None, 0,
                                              ctypes.byref(fro), None)
        if st != 0:
            raise cp.CPCPError(st, "rejected")
    assert e.value.status == 1
