"""Seeded synthetic point clouds shaped like the paper's workloads.

This module only draws random numbers (numpy PCG64) and lays out arrays; it
holds none of the method's arithmetic, so both the oracle-based tests and the
CUDA path can take their inputs from it.  The paper uses no dataset: its
inputs are points sampled from a support in Z^2 (Sec. 1, Fig. 1) and Gaussian
samples N(0, I_m) / N(0, Sigma) (Sec. 4.3).  The sizes here are the five
workloads the benchmark and the parity tests use.
"""
from __future__ import annotations

import math

import numpy as np

SEEDS = {"grid": 1005, "mixture": 1002, "cube": 1003, "normal": 1004, "batch": 1006, "runtime": 1007}


def grid_support_cloud(seed: int = SEEDS["grid"], samples: int = 1000, grid: int = 64):
    """Integer points in a 64x64 grid of Z^2: the union of 3 random discs and 2
    random axis-aligned rectangles; `samples` cells drawn uniformly with
    replacement from that support, then de-duplicated (Fig. 1's recipe; the
    paper does not specify its support, so discs/rectangles stand in).
    Radii ~ U[4, 16], rectangle sides ~ U[4, 24]."""
    rng = np.random.default_rng(seed)
    ii, jj = np.meshgrid(np.arange(grid), np.arange(grid), indexing="ij")
    mask = np.zeros((grid, grid), dtype=bool)
    for _ in range(3):
        cx, cy = rng.uniform(0, grid, size=2)
        rad = rng.uniform(4, 16)
        mask |= (ii - cx) ** 2 + (jj - cy) ** 2 <= rad * rad
    for _ in range(2):
        x0, y0 = rng.uniform(0, grid, size=2)
        wx, wy = rng.uniform(4, 24, size=2)
        mask |= (ii >= x0) & (ii <= x0 + wx) & (jj >= y0) & (jj <= y0 + wy)
    cells = np.argwhere(mask)
    pick = rng.integers(0, len(cells), size=samples)
    pts = np.unique(cells[pick], axis=0)
    return np.ascontiguousarray(pts, dtype=np.float64)


def gaussian_mixture_cloud(n: int = 16384, m: int = 3, components: int = 8, sigma: float = 0.5,
                           seed: int = SEEDS["mixture"]):
    """n points from an isotropic Gaussian mixture: means ~ U[0, 10]^m, each
    point assigned to a component uniformly, N(mean, sigma^2 I)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(0.0, 10.0, size=(components, m))
    comp = rng.integers(0, components, size=n)
    X = means[comp] + sigma * rng.standard_normal((n, m))
    return np.ascontiguousarray(X, dtype=np.float64)


def unit_cube_cloud(n: int = 100_000, m: int = 8, seed: int = SEEDS["cube"]):
    """n points uniform in [0, 1]^m."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.random((n, m)), dtype=np.float64)


def normal_cloud(n: int = 8192, m: int = 16, scale: float | None = None, seed: int = SEEDS["normal"]):
    """n points ~ N(0, I_m) times `scale` (default 1/sqrt(m))."""
    rng = np.random.default_rng(seed)
    s = 1.0 / math.sqrt(m) if scale is None else scale
    return np.ascontiguousarray(s * rng.standard_normal((n, m)), dtype=np.float64)


def anisotropic_normal_cloud(n: int, m: int, seed: int = 7):
    """N(0, Sigma) with Sigma_jj = 2^-(j-1) (Sec. 4.3's second distribution)."""
    rng = np.random.default_rng(seed)
    sd = np.sqrt(2.0 ** -np.arange(m))
    return np.ascontiguousarray(rng.standard_normal((n, m)) * sd, dtype=np.float64)


def batch_clouds(count: int = 512, m: int = 32, n_min: int = 64, n_max: int = 2048, n_t: int = 8,
                 t_min: float = 0.1, t_max: float = 10.0, seed: int = SEEDS["batch"]):
    """`count` clouds in R^m with sizes round(exp(U[ln n_min, ln n_max])), points
    ~ N(0, I_m) per cloud, each to be solved at n_t values of t log-spaced in
    [t_min, t_max].  Returns (list of arrays, t values)."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=count))).astype(int)
    clouds = [np.ascontiguousarray(rng.standard_normal((int(s), m)), dtype=np.float64) for s in sizes]
    ts = np.geomspace(t_min, t_max, n_t)
    return clouds, ts


PAPER_RUNTIME_NS = (1000, 3000, 10000, 30000)
PAPER_RUNTIME_MS = (3, 10, 30, 100)
PAPER_RUNTIME_COVS = ("identity", "halving")


def paper_runtime_cloud(n: int, m: int, cov: str = "identity", run: int = 0, seed: int = SEEDS["runtime"]):
    """The paper's runtime workload (Sec. 4, experimental results): n points
    from N(0, I_m) ("identity") or from N(0, Sigma) with Sigma_jj = 2^-(j-1)
    ("halving"), for n in PAPER_RUNTIME_NS and m in PAPER_RUNTIME_MS, three
    runs per configuration; the task is t_+ and the weighting at t_+.  Each
    (n, m, cov, run) has its own seeded stream."""
    ci = PAPER_RUNTIME_COVS.index(cov)
    rng = np.random.default_rng([seed, n, m, ci, run])
    sd = np.ones(m) if cov == "identity" else np.sqrt(2.0 ** -np.arange(m))
    return np.ascontiguousarray(rng.standard_normal((n, m)) * sd, dtype=np.float64)


def subsample(X, n: int, seed: int = 0):
    """A seeded subset of n rows (used for bounded CPU samples of a workload)."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(X.shape[0], size=n, replace=False))
    return np.ascontiguousarray(X[idx])
