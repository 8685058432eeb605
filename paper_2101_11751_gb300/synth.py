"""Seeded synthetic workloads shaped like the paper's experiments.

This module only draws inputs (points, targets, grids, hyperparameters). It holds none of the
method's arithmetic and is shared by the CUDA path's tests/bench and by the CPU oracle's tests.

The paper's datasets (sine, Sound, Radar, Precipitation; Sec. 5, Table 1) are not available, so
each generator stands in for one workload shape:

* ``sine_1d``      -- the synthetic sine experiment of Sec. 5 (Fig. 2), d=1, FP64.
* ``gmm_2d``       -- clustered 2-D spatial data (d=2, Matern-5/2 kernel), FP32.
* ``grf_3d``       -- precipitation-like 3-D field (d=3, RBF ARD, gradient workload), FP32.
* ``radar_3d``     -- the 120M-point weather-radar run of Sec. 5: conical sweeps to Cartesian.
* ``batch_2d``     -- many independent uneven 2-D problems (serving-style batch).

All randomness comes from ``numpy.random.default_rng(seed)``; the heavier deterministic
evaluations (blob sums, trilinear sampling) use torch CPU ops only for speed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache
from typing import List, Optional, Tuple

import numpy as np

RBF = 0
MATERN52 = 1


@dataclass
class Grid:
    """Regular grid: node j on axis k sits at lo[k] + j*h[k], j = 0..M[k]-1 (C order)."""
    d: int
    M: Tuple[int, ...]
    lo: Tuple[float, ...]
    h: Tuple[float, ...]

    @property
    def m(self) -> int:
        return int(np.prod(self.M))

    @property
    def ncells(self) -> int:
        return int(np.prod([mk - 3 for mk in self.M]))


@dataclass
class Kernel:
    type: int
    lengthscale: Tuple[float, ...]
    outputscale: float
    noise_var: float


@dataclass
class Problem:
    name: str
    X: np.ndarray          # d x n, float32 or float64 (SoA)
    y: np.ndarray          # n, same dtype as X
    grid: Grid
    kernel: Kernel
    rtol: float
    n_probes: int = 0
    probe_seed: int = 0
    Xstar: Optional[np.ndarray] = None   # d x n* test points
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.X.shape[1])

    @property
    def d(self) -> int:
        return int(self.X.shape[0])


def grid_for_box(lo_data, hi_data, M) -> Grid:
    """Grid whose interior [g_1, g_{M-2}] covers the data box with a relative margin of 1e-5.

    Cubic convolution needs nodes c-1..c+2 around each point, so the data must sit in
    [g_1, g_{M-2}]; one spacing of padding on each side provides that.
    """
    lo_data = np.asarray(lo_data, dtype=np.float64)
    hi_data = np.asarray(hi_data, dtype=np.float64)
    M = tuple(int(v) for v in M)
    span = hi_data - lo_data
    a = lo_data - 1e-5 * span
    b = hi_data + 1e-5 * span
    h = (b - a) / (np.asarray(M, dtype=np.float64) - 3.0)
    lo = a - h
    return Grid(d=len(M), M=M, lo=tuple(float(v) for v in lo), h=tuple(float(v) for v in h))


# ---------------------------------------------------------------- sine (d = 1)

def sine_1d(n: int = 10_000, seed: int = 0, M: int = 1000) -> Problem:
    """d=1, x ~ U[0,1] FP64, y = sin(6 pi x) + 0.3 cos(20 pi x) + N(0, 0.1^2).

    Grid of M=1000 nodes uniform on [-0.01, 1.01]; RBF l=0.05, s=1, sigma^2=0.01, rtol 1e-10.
    """
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, n)
    y = np.sin(6 * np.pi * x) + 0.3 * np.cos(20 * np.pi * x) + rng.normal(0.0, 0.1, n)
    grid = Grid(d=1, M=(M,), lo=(-0.01,), h=(1.02 / (M - 1),))
    kern = Kernel(RBF, (0.05,), 1.0, 0.01)
    xs = np.linspace(0.0, 1.0, 1001)[None, :]
    return Problem("sine_1d", x[None, :].astype(np.float64), y.astype(np.float64), grid, kern,
                   rtol=1e-10, Xstar=xs)


def sine_sweep(n: int, m: int, seed: int = 0) -> Problem:
    """Sec. 5's per-iteration benchmark data: a sine with two periods on [0, 1],
    y = sin(4 pi x) + N(0, 0.25), x ~ U[0,1] FP32, m grid nodes spanning [0, 1]; RBF l = 0.1,
    s = 1, sigma^2 = 0.25."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, n)
    y = np.sin(4 * np.pi * x) + rng.normal(0.0, 0.5, n)
    grid = grid_for_box([0.0], [1.0], (m,))
    return Problem(f"sine_sweep_{n}_{m}", x[None, :].astype(np.float32), y.astype(np.float32), grid,
                   Kernel(RBF, (0.1,), 1.0, 0.25), rtol=1e-2, Xstar=None)


# ---------------------------------------------------------------- Gaussian mixture (d = 2)

def gmm_2d(n: int = 1_000_000, seed: int = 0, M=(128, 128)) -> Problem:
    """d=2 FP32: 8-component isotropic Gaussian mixture (sigma 0.08, means ~ U[0.15,0.85]^2,
    equal weights), clipped to [0,1]^2; y = sin(4 pi x1) cos(3 pi x2) + N(0, 0.05^2).
    Matern-5/2, l = (0.04, 0.06), s = 1, sigma^2 = 2.5e-3, rtol 1e-6."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(0.15, 0.85, size=(8, 2))
    comp = rng.integers(0, 8, size=n)
    x = means[comp] + rng.normal(0.0, 0.08, size=(n, 2))
    x = np.clip(x, 0.0, 1.0)
    y = np.sin(4 * np.pi * x[:, 0]) * np.cos(3 * np.pi * x[:, 1]) + rng.normal(0.0, 0.05, n)
    grid = grid_for_box([0.0, 0.0], [1.0, 1.0], M)
    kern = Kernel(MATERN52, (0.04, 0.06), 1.0, 2.5e-3)
    xs = rng.uniform(0.0, 1.0, size=(2, 4096))
    return Problem("gmm_2d", np.ascontiguousarray(x.T.astype(np.float32)), y.astype(np.float32),
                   grid, kern, rtol=1e-6, Xstar=xs.astype(np.float32))


# ---------------------------------------------------------------- Gaussian random field (d = 3)

@lru_cache(maxsize=2)
def _grf_lattice(L: int, ell: float, seed: int) -> np.ndarray:
    """GRF sample on an L^3 lattice over [0,1]^3 with RBF covariance (lengthscale ell, scale 1).

    Drawn as (A1 (x) A2 (x) A3) xi with A = V Lambda^(1/2) from the per-axis eigendecomposition
    of the 1-D lattice kernel matrix (negative eigenvalues clipped to zero)."""
    g = np.linspace(0.0, 1.0, L)
    K1 = np.exp(-0.5 * ((g[:, None] - g[None, :]) / ell) ** 2)
    lam, V = np.linalg.eigh(K1)
    A = V * np.sqrt(np.clip(lam, 0.0, None))[None, :]
    rng = np.random.default_rng(seed + 7919)
    xi = rng.standard_normal((L, L, L))
    f = np.einsum("ai,ijk->ajk", A, xi, optimize=True)
    f = np.einsum("bj,ajk->abk", A, f, optimize=True)
    f = np.einsum("ck,abk->abc", A, f, optimize=True)
    return np.ascontiguousarray(f.astype(np.float32))


def _trilinear(field: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Trilinear sample of an L^3 lattice over [0,1]^3 at points x (3 x n)."""
    import torch
    L = field.shape[0]
    f = torch.from_numpy(field)
    p = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)) * (L - 1)
    i0 = torch.clamp(torch.floor(p).long(), 0, L - 2)
    w = p - i0.to(p.dtype)
    out = torch.zeros(p.shape[1], dtype=torch.float32)
    for dx in (0, 1):
        wx = w[0] if dx else 1 - w[0]
        for dy in (0, 1):
            wy = w[1] if dy else 1 - w[1]
            for dz in (0, 1):
                wz = w[2] if dz else 1 - w[2]
                out += wx * wy * wz * f[i0[0] + dx, i0[1] + dy, i0[2] + dz]
    return out.numpy()


def grf_3d(n: int = 10_000_000, seed: int = 0, M=(64, 64, 64), lattice: int = 256,
           n_probes: int = 16) -> Problem:
    """d=3 FP32: x ~ U[0,1]^3; y = GRF sample (RBF l=0.1) on a lattice^3 grid sampled trilinearly
    plus N(0, 0.1^2). RBF ARD initial theta: l = (0.1, 0.1, 0.1), s = 1, sigma^2 = 0.01; 16 probes."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, size=(3, n)).astype(np.float32)
    f = _grf_lattice(lattice, 0.1, seed)
    y = _trilinear(f, x) + rng.normal(0.0, 0.1, n).astype(np.float32)
    grid = grid_for_box([0.0] * 3, [1.0] * 3, M)
    kern = Kernel(RBF, (0.1, 0.1, 0.1), 1.0, 0.01)
    xs = rng.uniform(0.0, 1.0, size=(3, 4096)).astype(np.float32)
    return Problem("grf_3d", x, y.astype(np.float32), grid, kern, rtol=1e-4, n_probes=n_probes,
                   probe_seed=0, Xstar=xs)


# ---------------------------------------------------------------- radar volumes (d = 3)

RADAR_ELEV_DEG = np.linspace(0.5, 19.5, 14)
RADAR_AZ_DEG = np.arange(720) * 0.5
RADAR_RANGE_KM = 2.0 + 0.25 * np.arange(593)


def radar_geometry(n_sweeps: int = 14, n_az: int = 720, n_gates: int = 593) -> np.ndarray:
    """Flat-earth Cartesian coordinates (km) of one volume scan: 3 x (sweeps*az*gates)."""
    e = np.deg2rad(RADAR_ELEV_DEG[:n_sweeps])[:, None, None]
    a = np.deg2rad(RADAR_AZ_DEG[:n_az])[None, :, None]
    r = RADAR_RANGE_KM[:n_gates][None, None, :]
    x = r * np.cos(e) * np.sin(a)
    y = r * np.cos(e) * np.cos(a)
    z = r * np.sin(e) * np.ones_like(a)
    return np.stack([x.ravel(), y.ravel(), z.ravel()]).astype(np.float32)


def radar_3d(n_volumes: int = 20, seed: int = 0, M=(128, 128, 32), n_sweeps: int = 14,
             n_az: int = 720, n_gates: int = 593, device: str = "cpu") -> Problem:
    """Radar-shaped d=3 FP32 workload (default n = 20*14*720*593 = 119,548,800 points).

    Each volume scan has the same sweep geometry (one site observed at 20 times). Reflectivity
    in dBZ is a sum of 32 Gaussian blobs per volume (amplitude exp(N(3, 0.5)), horizontal width
    U[5,30] km, vertical width U[1,4] km, advected 5 km per volume) plus N(0,1) noise.
    Grid 128 x 128 x 32 over the full sweep box; RBF ARD l = (8, 8, 1.5) km, s = 100, sigma^2 = 1.
    The blob sums are evaluated with torch on `device` (the random draws are numpy's either way)."""
    import torch
    rng = np.random.default_rng(seed)
    geo = radar_geometry(n_sweeps, n_az, n_gates)
    npv = geo.shape[1]
    n = n_volumes * npv
    X = np.empty((3, n), dtype=np.float32)
    y = np.empty(n, dtype=np.float32)
    gt = torch.from_numpy(geo).to(device)
    nb = 32
    amp = np.exp(rng.normal(3.0, 0.5, nb))
    cxy = rng.uniform(-120.0, 120.0, size=(nb, 2))
    cz = rng.uniform(0.5, 8.0, nb)
    wxy = rng.uniform(5.0, 30.0, nb)
    wz = rng.uniform(1.0, 4.0, nb)
    ang = rng.uniform(0.0, 2 * np.pi, nb)
    vel = 5.0 * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    for v in range(n_volumes):
        sl = slice(v * npv, (v + 1) * npv)
        X[:, sl] = geo
        acc = torch.zeros(npv, dtype=torch.float32, device=device)
        for b in range(nb):
            c = cxy[b] + v * vel[b]
            q = ((gt[0] - float(c[0])) ** 2 + (gt[1] - float(c[1])) ** 2) / float(wxy[b] ** 2)
            q = q + (gt[2] - float(cz[b])) ** 2 / float(wz[b] ** 2)
            acc += float(amp[b]) * torch.exp(-0.5 * q)
        y[sl] = acc.cpu().numpy() + rng.normal(0.0, 1.0, npv).astype(np.float32)
    lo = X.min(axis=1).astype(np.float64)
    hi = X.max(axis=1).astype(np.float64)
    grid = grid_for_box(lo, hi, M)
    kern = Kernel(RBF, (8.0, 8.0, 1.5), 100.0, 1.0)
    xs = np.stack([rng.uniform(lo[k], hi[k], 65536) for k in range(3)]).astype(np.float32)
    return Problem("radar_3d", X, y, grid, kern, rtol=1e-5, Xstar=xs,
                   meta={"n_volumes": n_volumes, "points_per_volume": npv})


# ---------------------------------------------------------------- serving batch (d = 2)

def batch_2d(n_problems: int = 64, seed: int = 1000, n_lo: float = 1e4, n_hi: float = 2e6,
             n_test: int = 100_000, sides=(32, 64, 128, 256)) -> List[Problem]:
    """Independent uneven d=2 FP32 problems: n ~ log-U[n_lo, n_hi], grid side uniform in
    `sides`, x ~ U[0,1]^2, y = sin(2 pi f1 x1) cos(2 pi f2 x2) + N(0, sigma^2) with f ~ U[1,4],
    isotropic RBF l ~ U[0.02, 0.2], sigma^2 ~ U[1e-3, 1e-1]."""
    out = []
    for p in range(n_problems):
        rng = np.random.default_rng(seed + p)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        side = int(rng.choice(np.asarray(sides)))
        ell = float(rng.uniform(0.02, 0.2))
        s2 = float(rng.uniform(1e-3, 1e-1))
        f1, f2 = rng.uniform(1.0, 4.0, 2)
        x = rng.uniform(0.0, 1.0, size=(2, n))
        y = np.sin(2 * np.pi * f1 * x[0]) * np.cos(2 * np.pi * f2 * x[1]) \
            + rng.normal(0.0, math.sqrt(s2), n)
        xs = rng.uniform(0.0, 1.0, size=(2, n_test))
        grid = grid_for_box([0.0, 0.0], [1.0, 1.0], (side, side))
        out.append(Problem(f"batch_{p}", x.astype(np.float32), y.astype(np.float32), grid,
                           Kernel(RBF, (ell, ell), 1.0, s2), rtol=1e-4,
                           Xstar=xs.astype(np.float32)))
    return out
