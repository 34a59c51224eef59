"""Host-side checks of the seeded workload generators (no GPU): shapes,
determinism, mask fractions and the structure each recipe promises."""
import numpy as np

from paper_2206_13369_gb300 import workloads as W


def test_hyperspectral_recipe():
    p = W.hyperspectral_cpcp(7, h=32, w=32, bands=64, rank=5, levels=2)
    m, n = p["D"].shape
    assert (m, n) == (1024, 64)
    # rank of the planted part and smoothness of its right singular vectors
    # in the band index (the setting of Assumption 3)
    U, s, Vt = np.linalg.svd(p["L0"], full_matrices=False)
    assert s[4] > 1e-6 * s[0] and s[5] < 1e-12 * s[0]
    V = Vt[:5].T
    rough = np.linalg.norm(np.diff(V, 2, axis=0)) / np.linalg.norm(V)
    assert rough < 0.1
    # abundances of the linear mixing model are non-negative and sum to one
    assert np.all(p["L0"] >= 0)
    # mask and outlier fractions, observed entries only in D
    assert abs(p["mask"].mean() - 0.8) < 0.02
    assert abs((p["S0"] != 0).mean() - 0.05) < 0.01
    assert np.all(p["D"][~p["mask"]] == 0)
    assert p["lam"] == 1.0 / np.sqrt(max(m, n)) and p["levels"] == 2
    # seeded: the same bytes every time
    q = W.hyperspectral_cpcp(7, h=32, w=32, bands=64, rank=5, levels=2)
    assert np.array_equal(p["D"], q["D"]) and np.array_equal(p["mask"], q["mask"])


def test_config_names_cover_configs():
    assert set(W.CONFIG_NAMES) == {1, 2, 3, 4, 5, 6}


def test_batched_instance_matches_the_batch():
    # one instance built alone equals the same instance of the whole batch
    batch = W.batched_cpcp(6, 4000)
    for i in (0, 5):
        q = W.batched_instance(4000, i)
        assert q["D"].shape == batch[i]["D"].shape and q["levels"] == batch[i]["levels"]
        assert np.array_equal(q["D"], batch[i]["D"]) and np.array_equal(q["mask"], batch[i]["mask"])
        assert q["lam"] == batch[i]["lam"] and q["mu"] == batch[i]["mu"]
