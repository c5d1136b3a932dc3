"""Seeded synthetic densities for the dynamical optimal-transport solver.

This module is shared by the CPU oracle and the CUDA path.  It only builds
*inputs*: the boundary densities rho_in and rho_f as cell averages on the
coarse (density) mesh.  It holds none of the solver's arithmetic.

Mesh convention (the public cell ordering of the C ABI):
  the unit square is cut into n x n squares of side h = 1/n; square (i, j)
  spans [i h, (i+1) h] x [j h, (j+1) h] and is split by its diagonal from
  (i h, j h) to ((i+1) h, (j+1) h) into
    t = 0 (lower-right): vertices (i, j), (i+1, j), (i+1, j+1)
    t = 1 (upper-left):  vertices (i, j), (i+1, j+1), (i, j+1)
  and triangle (t, i, j) has index t*n*n + j*n + i.

The densities follow the test cases of Section 4.1 (Gaussian bumps bounded
below by a floor) and the seeded mixtures used for the larger workloads:
  value = max(cell average of sum_g w_g N(c_g, sigma_g^2 I), floor),
  then scaled so that sum_cells |cell| * value = 1.
Cell averages use the three-edge-midpoint rule (exact for quadratics) on the
16 triangles of a twice-repeated midpoint split of each cell.

The 3D Cartesian variant (test 4 of Section 4.1) uses n^3 cubes of side 1/n,
cube (i, j, k) at index (k n + j) n + i, with cell averages by the tensor
3-point Gauss-Legendre rule in each direction.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "coarse_triangles",
    "gaussian_mixture_cell_average",
    "make_density",
    "mixture_params",
    "config_densities",
    "batched_problem_specs",
    "mass_preserving_directions",
    "make_cube_density",
    "cube_config_densities",
]


def coarse_triangles(n: int) -> np.ndarray:
    """Vertex coordinates of the 2 n^2 triangles, shape (2 n^2, 3, 2), canonical order."""
    h = 1.0 / n
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i = i.ravel().astype(np.float64)
    j = j.ravel().astype(np.float64)
    p00 = np.stack([i * h, j * h], -1)
    p10 = np.stack([(i + 1) * h, j * h], -1)
    p11 = np.stack([(i + 1) * h, (j + 1) * h], -1)
    p01 = np.stack([i * h, (j + 1) * h], -1)
    lower = np.stack([p00, p10, p11], 1)
    upper = np.stack([p00, p11, p01], 1)
    return np.concatenate([lower, upper], 0)


def _split4(tri: np.ndarray) -> np.ndarray:
    a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
    ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
    kids = [
        np.stack([a, ab, ca], 1),
        np.stack([ab, b, bc], 1),
        np.stack([ca, bc, c], 1),
        np.stack([ab, bc, ca], 1),
    ]
    return np.stack(kids, 1).reshape(-1, 3, 2)


def gaussian_mixture_cell_average(tri: np.ndarray, centres, sigmas, weights) -> np.ndarray:
    """Average over each triangle of sum_g w_g * N(c_g, sigma_g^2 I)(x)."""
    sub = _split4(_split4(tri))  # 16 sub-triangles per cell, equal areas
    mids = np.stack(
        [(sub[:, 0] + sub[:, 1]) / 2, (sub[:, 1] + sub[:, 2]) / 2, (sub[:, 2] + sub[:, 0]) / 2], 1
    )  # (16 T, 3, 2)
    val = np.zeros(mids.shape[:2])
    for c, s, w in zip(centres, sigmas, weights):
        d2 = ((mids - np.asarray(c, dtype=np.float64)) ** 2).sum(-1)
        val += w * np.exp(-d2 / (2.0 * s * s)) / (2.0 * np.pi * s * s)
    per_sub = val.mean(1)  # midpoint rule: equal weights 1/3
    return per_sub.reshape(tri.shape[0], 16).mean(1)


def make_density(n: int, centres, sigmas, weights, floor: float) -> np.ndarray:
    """Floored, unit-mass cell averages on the n x n coarse mesh (float64, canonical order)."""
    tri = coarse_triangles(n)
    v = gaussian_mixture_cell_average(tri, centres, sigmas, weights)
    v = np.maximum(v, floor)
    area = 0.5 / (n * n)
    return v / (area * v.sum())


def mixture_params(seed: int, n_gauss: int, sigma_range=(0.05, 0.15)):
    """Centres U[0.15,0.85]^2, sigma U[sigma_range], weights U[0.5,1.5] from numpy's PCG64."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.15, 0.85, size=(n_gauss, 2))
    sigmas = rng.uniform(sigma_range[0], sigma_range[1], size=n_gauss)
    weights = rng.uniform(0.5, 1.5, size=n_gauss)
    return centres, sigmas, weights


def config_densities(name: str, n: int | None = None):
    """(n, K, rho_in, rho_f) for the named synthetic workloads.

    'gauss8'   : 8x8 squares, K=8, Gaussians sigma=0.1 at (0.3,0.3) -> (0.7,0.7), floor 1e-3.
    'mix64'    : 64x64 squares, K=32, 3-Gaussian mixtures (seeds 2, 3), floor 1e-4.
    'mix128'   : 128x128 squares, K=32, 3-Gaussian mixtures (seeds 4, 5), floor 1e-4.
    'fd32'     : 32x32 squares, K=16, 3-Gaussian mixtures (seeds 6, 7), floor 1e-4.
    'stress256': 256x256 squares, K=64, 5-Gaussian mixtures sigma in [0.02,0.15] (seeds 9, 10), floor 1e-6.
    'mixN'     : n x n (argument), K=max(4, n/2), 3-Gaussian mixtures (seeds 2, 3), floor 1e-4.
    """
    if name == "gauss8":
        n, K = 8, 8
        r0 = make_density(n, [(0.3, 0.3)], [0.1], [1.0], 1e-3)
        r1 = make_density(n, [(0.7, 0.7)], [0.1], [1.0], 1e-3)
        return n, K, r0, r1
    table = {
        "mix64": (64, 32, 2, 3, 3, (0.05, 0.15), 1e-4),
        "mix128": (128, 32, 4, 5, 3, (0.05, 0.15), 1e-4),
        "fd32": (32, 16, 6, 7, 3, (0.05, 0.15), 1e-4),
        "stress256": (256, 64, 9, 10, 5, (0.02, 0.15), 1e-6),
    }
    if name == "mixN":
        nn, K, s0, s1, g, sr, fl = n, max(4, n // 2), 2, 3, 3, (0.05, 0.15), 1e-4
    else:
        nn, K, s0, s1, g, sr, fl = table[name]
    r0 = make_density(nn, *mixture_params(s0, g, sr), fl)
    r1 = make_density(nn, *mixture_params(s1, g, sr), fl)
    return nn, K, r0, r1


def batched_problem_specs(count: int = 64, base_seed: int = 1000):
    """Uneven batch: side from {16,24,32,48,64}, K from {8,16,24,32}, 1-4 Gaussians, floor 1e-4."""
    specs = []
    for p in range(count):
        rng = np.random.default_rng(base_seed + p)
        n = int(rng.choice([16, 24, 32, 48, 64]))
        K = int(rng.choice([8, 16, 24, 32]))
        g0 = int(rng.integers(1, 5))
        g1 = int(rng.integers(1, 5))
        s0, s1 = (int(x) for x in rng.integers(0, 2**31 - 1, size=2))
        r0 = make_density(n, *mixture_params(s0, g0), 1e-4)
        r1 = make_density(n, *mixture_params(s1, g1), 1e-4)
        specs.append((n, K, r0, r1))
    return specs


def mass_preserving_directions(n: int, count: int, seed: int) -> np.ndarray:
    """Random directions v with sum_cells |cell| v = 0 and max|v| <= 1, shape (count, 2 n^2)."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1.0, 1.0, size=(count, 2 * n * n))
    v -= v.mean(1, keepdims=True)
    v /= np.abs(v).max(1, keepdims=True)
    return v


def make_cube_density(n: int, centres, sigmas, weights, floor: float) -> np.ndarray:
    """Floored, unit-mass cell averages of sum_g w_g N(c_g, sigma_g^2 I) on n^3 cubes."""
    h = 1.0 / n
    nodes = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
    wts = np.array([5.0, 8.0, 5.0]) / 18.0          # Gauss-Legendre on [0, 1] after the map below
    g = np.arange(n) * h
    pts = (g[:, None] + h * (0.5 + 0.5 * nodes)[None, :]).ravel()   # (3n,) quadrature abscissae
    w1 = np.tile(wts, n)
    val = np.zeros((n, n, n))
    for c, s, w in zip(centres, sigmas, weights):
        f = [np.exp(-((pts - c[a]) ** 2) / (2.0 * s * s)) * w1 for a in range(3)]
        fx, fy, fz = (fa.reshape(n, 3).sum(1) for fa in f)   # per-cell 1D averages
        val += w * np.einsum("k,j,i->kji", fz, fy, fx) / (2.0 * np.pi * s * s) ** 1.5
    v = np.maximum(val.ravel(), floor)
    return v / (h ** 3 * v.sum())


def cube_config_densities(name: str, n: int | None = None):
    """(n, K, rho_in, rho_f) for the 3D test: Gaussians sigma = 0.1 at
    (0.3,0.3,0.3) -> (0.7,0.7,0.7), floor 1e-3 (test 4 of Section 4.1).
    'gauss_cube8': 8^3 cubes, K + 1 = 8 time intervals; 'gauss_cubeN': n^3 (argument), K + 1 = n."""
    if name == "gauss_cube8":
        n = 8
    elif name != "gauss_cubeN":
        raise KeyError(name)
    K = n - 1
    r0 = make_cube_density(n, [(0.3, 0.3, 0.3)], [0.1], [1.0], 1e-3)
    r1 = make_cube_density(n, [(0.7, 0.7, 0.7)], [0.1], [1.0], 1e-3)
    return n, K, r0, r1
