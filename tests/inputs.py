"""Seeded synthetic inputs shared by the oracle side and the CUDA side of tests.

Holds no arithmetic of the method: only states drawn from numpy's seeded
generator, with the shapes and value ranges of the workloads (particle clouds
with X_0 ~ N(0, I_d), optionally widened to reach the heavy tails that the
implicit cubic drift produces).
"""
import numpy as np


def gaussian_cloud(N, d, seed, scale=1.0, mean=0.0):
    rng = np.random.default_rng(seed)
    return mean + scale * rng.standard_normal((N, d))


def heavy_cloud(N, d, seed):
    """A cloud mixing N(0, I) with a few far particles (|x| up to ~4.5)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((N, d))
    k = max(1, N // 64)
    idx = rng.choice(N, size=k, replace=False)
    x[idx] *= 2.0
    return x


def uniform_points(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n)
