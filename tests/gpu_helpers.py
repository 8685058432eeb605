"""Shared helpers for the GPU parity tests (seeded inputs, tolerances)."""
import numpy as np

from paper_2101_11751_gb300 import synth


def problem(d, M, n, seed=0, dtype=np.float32, clustered=False):
    """Seeded points on [0,1]^d with a smooth target plus noise, on a grid padded around the box."""
    rng = np.random.default_rng(seed)
    if clustered:
        c = rng.uniform(0.2, 0.8, size=(4, d))
        X = c[rng.integers(0, 4, n)] + rng.normal(0, 0.08, size=(n, d))
        X = np.clip(X, 0, 1).T
    else:
        X = rng.uniform(0, 1, size=(d, n))
    y = np.sin(3 * X[0]) + (np.cos(2 * X[1]) if d > 1 else 0) + (X[2] ** 2 if d > 2 else 0)
    y = y + 0.1 * rng.normal(size=n)
    grid = synth.grid_for_box([0.0] * d, [1.0] * d, M)
    return grid, np.ascontiguousarray(X.astype(dtype)), y.astype(dtype)


def rel_fro(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def max_rel(a, b):
    return float(np.max(np.abs(np.ravel(a) - np.ravel(b))) / max(np.max(np.abs(b)), 1e-300))
