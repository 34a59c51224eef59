"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and assembles test matrices.  It holds
none of the solver's arithmetic, so the CUDA path, the fp64 oracle, the tests
and the benchmark can all consume the same bytes without sharing any code of
the method itself.

Every generator uses ``numpy.random.default_rng(seed)`` (PCG64) in float64
and returns a plain dict:

    D      (m, n) float64   observed data; entries off the mask are 0
    mask   (m, n) bool or None (None = everything observed, i.e. PCP)
    L0, S0 (m, n) float64   planted low-rank and sparse parts
    lam    float            weight of the l1 term (lambda of eq. (rpca))
    mu     float            nuclear-norm weight mu_bar of the solved program
    levels int              number of levels (1 = single level)

The solved program is the CPCP objective of Sec. 2, eq. (cpcp), with
lambda_L = mu and lambda_S = lam * mu.  mu defaults to 1e-3 * ||P_Q[D]||_2.

Workload recipes (the paper's data sets are not available; these stand in
for their shapes and structure):

* planted PCP, Sec. 4.1 style: D = L0 + S0, L0 = U V^T with U, V iid
  N(0, 1/max(m, n)), S0 with Bernoulli(rho) support and +-1 values.
* planted CPCP: L0 = U V^T / sqrt(r) with U, V iid N(0, 1) (unit-variance
  entries), S0 Bernoulli(rho) support with values U[-5, 5], mask
  Bernoulli(obs), D = P_Q[L0 + S0].
* video-shaped CPCP (Sec. 4.2 shapes): 120x160 frames stacked as columns,
  rank-5 background of smooth random fields with smooth temporal
  coefficients, 10x10 moving foreground blocks, mask Bernoulli(0.6).
* batched CPCP: many uneven planted CPCP instances.
* hyperspectral-shaped CPCP (the hyperspectral motivation of Sec. 1):
  pixels x bands under a linear mixing model, smooth endmember spectra
  (so the right singular subspace is smooth in the band index, the setting
  of Assumption 3), sparse outliers, mask Bernoulli(obs).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "spectral_norm",
    "planted_pcp",
    "planted_cpcp",
    "video_cpcp",
    "batched_cpcp",
    "hyperspectral_cpcp",
    "planted_cpcp_fw",
    "config",
    "CONFIG_NAMES",
]


def spectral_norm(A: np.ndarray) -> float:
    """Largest singular value of A via LAPACK (workload parameter only)."""
    return float(np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)[0])


def _finish(D, mask, L0, S0, lam, levels, mu_rel=1e-3):
    PQD = D if mask is None else np.where(mask, D, 0.0)
    mu = mu_rel * spectral_norm(PQD)
    return {
        "D": np.ascontiguousarray(PQD, dtype=np.float64),
        "mask": None if mask is None else np.ascontiguousarray(mask, dtype=bool),
        "L0": L0,
        "S0": S0,
        "lam": float(lam),
        "mu": float(mu),
        "levels": int(levels),
    }


def planted_pcp(m: int, n: int, rank: int, rho: float, seed: int, levels: int = 1,
                factor_var: float | None = None) -> dict:
    """Fully observed planted problem (Candes et al. convention).

    U, V ~ N(0, factor_var) with factor_var = 1/max(m, n) by default;
    S0 has Bernoulli(rho) support and equiprobable +-1 values.
    """
    rng = np.random.default_rng(seed)
    var = 1.0 / max(m, n) if factor_var is None else factor_var
    U = rng.normal(0.0, math.sqrt(var), size=(m, rank))
    V = rng.normal(0.0, math.sqrt(var), size=(n, rank))
    L0 = U @ V.T
    supp = rng.random((m, n)) < rho
    signs = np.where(rng.random((m, n)) < 0.5, -1.0, 1.0)
    S0 = np.where(supp, signs, 0.0)
    D = L0 + S0
    return _finish(D, None, L0, S0, 1.0 / math.sqrt(max(m, n)), levels)


def planted_cpcp(m: int, n: int, rank: int, rho: float, obs: float, seed: int,
                 levels: int = 1, amp: float = 5.0) -> dict:
    """Partially observed planted problem with unit-variance low-rank entries.

    L0 = U V^T / sqrt(rank), U, V iid N(0, 1); S0 support Bernoulli(rho) with
    values U[-amp, amp]; mask Bernoulli(obs) (obs >= 1 means no mask).
    """
    rng = np.random.default_rng(seed)
    U = rng.normal(size=(m, rank))
    V = rng.normal(size=(n, rank))
    L0 = (U @ V.T) / math.sqrt(rank)
    supp = rng.random((m, n)) < rho
    vals = rng.uniform(-amp, amp, size=(m, n))
    S0 = np.where(supp, vals, 0.0)
    mask = None if obs >= 1.0 else (rng.random((m, n)) < obs)
    D = L0 + S0
    return _finish(D, mask, L0, S0, 1.0 / math.sqrt(max(m, n)), levels)


def _gauss_blur(field: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian blur with reflected borders (numpy only)."""
    rad = int(math.ceil(4 * sigma))
    x = np.arange(-rad, rad + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    k /= k.sum()
    out = field
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (rad, rad)
        p = np.pad(out, pad, mode="reflect")
        acc = np.zeros_like(out)
        for i, w in enumerate(k):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(i, i + out.shape[axis])
            acc += w * p[tuple(sl)]
        out = acc
    return out


def video_cpcp(seed: int, h: int = 120, w: int = 160, frames: int = 400, rank: int = 5,
               blocks: int = 15, block: int = 10, obs: float = 0.6, levels: int = 4) -> dict:
    """Video-shaped CPCP: pixels x frames, smooth background, moving blocks.

    Background L0 = sum_i f_i c_i^T with f_i a white-noise field blurred with a
    Gaussian of 8 px, rescaled to [0, 1] / rank; c_1 = 1 (static component) and
    c_i(t) = 0.2 sin(2 pi (omega_i t / frames + phi_i)), omega_i in {1..4}.
    Foreground: `blocks` squares of `block` px moving at a constant velocity of
    1..3 px/frame, reflected at the borders, additive values U[0, 1].
    """
    rng = np.random.default_rng(seed)
    m = h * w
    F = np.empty((m, rank))
    for i in range(rank):
        f = _gauss_blur(rng.normal(size=(h, w)), 8.0)
        f = (f - f.min()) / max(f.max() - f.min(), 1e-30)
        F[:, i] = f.reshape(-1) / rank
    t = np.arange(frames, dtype=np.float64)
    C = np.empty((frames, rank))
    C[:, 0] = 1.0
    for i in range(1, rank):
        omega = rng.integers(1, 5)
        phi = rng.random()
        C[:, i] = 0.2 * np.sin(2 * math.pi * (omega * t / frames + phi))
    L0 = F @ C.T
    S0 = np.zeros((m, frames))
    pos = np.stack([rng.uniform(0, h - block, blocks), rng.uniform(0, w - block, blocks)], 1)
    speed = rng.uniform(1.0, 3.0, blocks)
    ang = rng.uniform(0, 2 * math.pi, blocks)
    vel = np.stack([speed * np.sin(ang), speed * np.cos(ang)], 1)
    lim = np.array([h - block, w - block], dtype=np.float64)
    for fr in range(frames):
        img = np.zeros((h, w))
        for b in range(blocks):
            y, x = int(round(pos[b, 0])), int(round(pos[b, 1]))
            img[y:y + block, x:x + block] += rng.random((block, block))
        S0[:, fr] = img.reshape(-1)
        pos += vel
        for ax in range(2):
            lo = pos[:, ax] < 0
            hi = pos[:, ax] > lim[ax]
            pos[lo, ax] = -pos[lo, ax]
            pos[hi, ax] = 2 * lim[ax] - pos[hi, ax]
            vel[lo | hi, ax] *= -1
    mask = rng.random((m, frames)) < obs
    D = L0 + S0
    return _finish(D, mask, L0, S0, 1.0 / math.sqrt(max(m, frames)), levels)


def hyperspectral_cpcp(seed: int, h: int = 256, w: int = 256, bands: int = 128, rank: int = 8,
                       rho: float = 0.05, obs: float = 0.8, levels: int = 3) -> dict:
    """Hyperspectral-shaped CPCP: pixels x bands, linear mixing of smooth spectra.

    Endmember spectra V (bands x rank): each a sum of three Gaussian bumps in
    the band index (centres U[0, bands), widths U[6, 20] bands, heights
    U[0.5, 1]).  Abundances U (pixels x rank): white-noise fields blurred with a
    Gaussian of 6 px, shifted to be non-negative and normalised to sum to 1 per
    pixel.  L0 = U V^T.  Outliers S0: Bernoulli(rho) support with values
    U[-1, 1] * max|L0|.  Mask Bernoulli(obs).
    """
    rng = np.random.default_rng(seed)
    m = h * w
    b = np.arange(bands, dtype=np.float64)
    V = np.zeros((bands, rank))
    for i in range(rank):
        for _ in range(3):
            c, wd, ht = rng.uniform(0, bands), rng.uniform(6, 20), rng.uniform(0.5, 1.0)
            V[:, i] += ht * np.exp(-0.5 * ((b - c) / wd) ** 2)
    U = np.empty((m, rank))
    for i in range(rank):
        f = _gauss_blur(rng.normal(size=(h, w)), 6.0)
        U[:, i] = (f - f.min()).reshape(-1)
    U /= np.maximum(U.sum(axis=1, keepdims=True), 1e-30)
    L0 = U @ V.T
    support = rng.random((m, bands)) < rho
    S0 = np.where(support, rng.uniform(-1.0, 1.0, (m, bands)) * np.abs(L0).max(), 0.0)
    mask = rng.random((m, bands)) < obs
    return _finish(L0 + S0, mask, L0, S0, 1.0 / math.sqrt(max(m, bands)), levels)


def planted_cpcp_fw(m: int, n: int, rank: int, rho: float, obs: float, seed: int, mu_rel: float = 0.05,
                    levels: int = 1) -> dict:
    """The planted CPCP recipe at the shapes of the Frank-Wolfe comparisons
    (m x n up to 10000 x 5000), in float32 storage (fp64 generation).  The
    weight mu = mu_rel ||P_Q D||_2 takes the spectral norm from 50 seeded power
    steps instead of a full SVD (a workload parameter, not the method)."""
    rng = np.random.default_rng(seed)
    U = rng.normal(size=(m, rank))
    V = rng.normal(size=(n, rank))
    L0 = (U @ V.T) / math.sqrt(rank)
    supp = rng.random((m, n)) < rho
    S0 = np.where(supp, rng.uniform(-5.0, 5.0, size=(m, n)), 0.0)
    mask = None if obs >= 1.0 else (rng.random((m, n)) < obs)
    D = L0 + S0
    PQD = D if mask is None else np.where(mask, D, 0.0)
    x = rng.normal(size=n)
    for _ in range(50):
        x = PQD.T @ (PQD @ x)
        x /= np.linalg.norm(x)
    snorm = float(np.linalg.norm(PQD @ x))
    return {"D": np.ascontiguousarray(PQD, dtype=np.float32), "mask": mask, "L0": L0, "S0": S0,
            "lam": 1.0 / math.sqrt(max(m, n)), "mu": mu_rel * snorm, "levels": int(levels)}


def _batched_levels(m: int, n: int, rank: int, max_levels: int = 3) -> int:
    """Deepest level count <= max_levels with n_H >= 2 (rank + 10) and
    n_H <= (m + 1) / 2 (Assumption 2), halving n with ceil per level."""
    best = 1
    nh = n
    for lv in range(2, max_levels + 1):
        nh = (nh + 1) // 2
        if nh >= 2 * (rank + 10) and nh <= (m + 1) / 2:
            best = lv
    return best


def batched_cpcp(count: int, seed: int, m_range=(64, 1024), n_range=(64, 512),
                 rank_range=(2, 20), rho_range=(0.05, 0.20), obs_range=(0.5, 1.0)) -> list:
    """Independent uneven planted CPCP instances (instance i uses seed + i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        r = int(rng.integers(rank_range[0], rank_range[1] + 1))
        rho = float(rng.uniform(*rho_range))
        obs = float(rng.uniform(*obs_range))
        lv = _batched_levels(m, n, r)
        p = planted_cpcp(m, n, r, rho, obs, seed + 1 + i, levels=lv)
        out.append(p)
    return out


def batched_instance(seed: int, index: int, **ranges) -> dict:
    """Instance `index` of batched_cpcp(count, seed, **ranges) (count > index),
    built alone: the size draws of the instances before it are replayed, their
    matrices are not."""
    keys = ("m_range", "n_range", "rank_range", "rho_range", "obs_range")
    defaults = dict(zip(keys, ((64, 1024), (64, 512), (2, 20), (0.05, 0.20), (0.5, 1.0))))
    rg = {k: ranges.get(k, defaults[k]) for k in keys}
    rng = np.random.default_rng(seed)
    for i in range(index + 1):
        m = int(rng.integers(rg["m_range"][0], rg["m_range"][1] + 1))
        n = int(rng.integers(rg["n_range"][0], rg["n_range"][1] + 1))
        r = int(rng.integers(rg["rank_range"][0], rg["rank_range"][1] + 1))
        rho = float(rng.uniform(*rg["rho_range"]))
        obs = float(rng.uniform(*rg["obs_range"]))
    return planted_cpcp(m, n, r, rho, obs, seed + 1 + index, levels=_batched_levels(m, n, r))


CONFIG_NAMES = {
    1: "pcp-200x200-r10-fp64",
    2: "cpcp-2000x2000-r50-fp32-3lv",
    3: "video-19200x400-r5-mixed-4lv",
    4: "batched-256-cpcp-fp32",
    5: "unrolled-1024x1024-r20-fp32-3lv",
    6: "hyperspectral-65536x128-r8-fp32-3lv",
}


def config(idx: int):
    """The workload configurations (seed 1000 * idx); 6 is the hyperspectral
    shape of the next-steps list."""
    seed = 1000 * idx
    if idx == 1:
        return planted_pcp(200, 200, 10, 0.05, seed, levels=2, factor_var=1.0 / 200)
    if idx == 2:
        return planted_cpcp(2000, 2000, 50, 0.10, 0.8, seed, levels=3)
    if idx == 3:
        return video_cpcp(seed)
    if idx == 4:
        return batched_cpcp(256, seed)
    if idx == 5:
        return planted_cpcp(1024, 1024, 20, 0.10, 0.7, seed, levels=3)
    if idx == 6:
        return hyperspectral_cpcp(seed)
    raise ValueError(f"unknown config {idx}")
