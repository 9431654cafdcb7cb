"""Seeded synthetic inputs for the G-prox PDHG solvers.

This module holds only input generators: no step of the method's arithmetic
lives here.  Both the CUDA path and the FP64 oracle are fed from these arrays,
so the two never share any computation beyond the inputs themselves.

Conventions (shared by every generator):
  * the domain is the unit square [0,1]^2 with an N x N cell-centred grid,
    h = 1/N, cell (i, j) has centre (x_j, y_i) = ((j + 1/2) h, (i + 1/2) h);
    row index i is y (slow axis), column index j is x (fast axis);
  * every random parameter is drawn with ``numpy.random.default_rng(seed)``
    (PCG64) in the order documented per generator;
  * fields are evaluated in float64 and returned as C-contiguous float32.

Workloads follow the paper's experiments (section 4: a disc image for ROF,
translated discs and delta measures for EMD) and the noisy multi-shape /
Gaussian-mixture inputs of the benchmark configurations.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "cell_centres",
    "rof_image",
    "gaussian_mixture_pair",
    "disc_image",
    "translated_discs",
    "delta_pair",
    "random_state",
    "cell_centres3",
    "ball_image3",
    "translated_balls3",
    "gaussian_mixture_pair3",
]


def cell_centres(N: int):
    """Return (x, y) float64 arrays of shape (N, N) holding cell centres."""
    c = (np.arange(N, dtype=np.float64) + 0.5) / N
    return np.meshgrid(c, c, indexing="xy")


def rof_image(N: int, seed: int, noise: float = 0.1, n_disks: int = 3) -> np.ndarray:
    """Noisy piecewise-constant test image for the ROF model.

    Draw order: for each of ``n_disks`` disks, radius r ~ U(0.10, 0.25), centre
    ~ U(r, 1-r)^2 (x then y), intensity ~ U(0, 1); then one axis-aligned
    rectangle with width, height ~ U(0.1, 0.5), lower-left corner ~
    U(0, 1-w) x U(0, 1-h), intensity ~ U(0, 1); then i.i.d. N(0, noise^2) per
    cell in row-major order.  Background 0, shapes painted in draw order (each
    overwrites), no clipping after the noise.
    """
    rng = np.random.default_rng(seed)
    x, y = cell_centres(N)
    img = np.zeros((N, N), dtype=np.float64)
    for _ in range(n_disks):
        r = rng.uniform(0.10, 0.25)
        cx = rng.uniform(r, 1.0 - r)
        cy = rng.uniform(r, 1.0 - r)
        val = rng.uniform(0.0, 1.0)
        img[(x - cx) ** 2 + (y - cy) ** 2 <= r * r] = val
    w = rng.uniform(0.1, 0.5)
    hh = rng.uniform(0.1, 0.5)
    x0 = rng.uniform(0.0, 1.0 - w)
    y0 = rng.uniform(0.0, 1.0 - hh)
    val = rng.uniform(0.0, 1.0)
    img[(x >= x0) & (x <= x0 + w) & (y >= y0) & (y <= y0 + hh)] = val
    if noise > 0:
        img = img + rng.normal(0.0, noise, size=(N, N))
    return np.ascontiguousarray(img, dtype=np.float32)


def _mixture(N: int, rng, n_comp: int, floor: float) -> np.ndarray:
    x, y = cell_centres(N)
    f = np.zeros((N, N), dtype=np.float64)
    params = []
    for _ in range(n_comp):
        cx = rng.uniform(0.1, 0.9)
        cy = rng.uniform(0.1, 0.9)
        s = rng.uniform(0.02, 0.08)
        w = rng.uniform(0.0, 1.0)
        params.append((cx, cy, s, w))
    for cx, cy, s, w in params:
        f += w * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s)) / (2 * np.pi * s * s)
    f += floor
    f /= f.sum() / (N * N)  # unit mass: h^2 * sum f = 1
    return f


def gaussian_mixture_pair(N: int, seed: int, n_comp: int = 8, floor: float = 1e-3):
    """Two probability densities for the L1 EMD problem.

    Each density is a mixture of ``n_comp`` isotropic Gaussians with centre ~
    U(0.1, 0.9)^2, width sigma ~ U(0.02, 0.08) and weight ~ U(0, 1) (drawn per
    component in that order, all of f0's components before f1's), plus an
    additive floor, then normalised in float64 to unit mass h^2 * sum f = 1
    before the cast to float32.
    """
    rng = np.random.default_rng(seed)
    f0 = _mixture(N, rng, n_comp, floor)
    f1 = _mixture(N, rng, n_comp, floor)
    return (np.ascontiguousarray(f0, dtype=np.float32),
            np.ascontiguousarray(f1, dtype=np.float32))


def disc_image(N: int, radius: float = 0.25, centre=(0.5, 0.5)) -> np.ndarray:
    """Indicator of a disc (section 4.1 ROF experiment: r = 1/4 at the centre)."""
    x, y = cell_centres(N)
    img = ((x - centre[0]) ** 2 + (y - centre[1]) ** 2 <= radius * radius).astype(np.float64)
    return np.ascontiguousarray(img, dtype=np.float32)


def translated_discs(N: int, radius: float = 0.25, c0=(0.375, 0.375), c1=(0.625, 0.625)):
    """Uniform unit-mass discs translated by (1/4, 1/4) (section 4.2 EMD experiment).

    Returns (f0, f1) with f0 centred at c0 and f1 at c1, each normalised to
    h^2 * sum f = 1 on the grid.
    """
    x, y = cell_centres(N)
    out = []
    for c in (c0, c1):
        f = ((x - c[0]) ** 2 + (y - c[1]) ** 2 <= radius * radius).astype(np.float64)
        f /= f.sum() / (N * N)
        out.append(np.ascontiguousarray(f, dtype=np.float32))
    return out[0], out[1]


def delta_pair(N: int, p0=(0.375, 0.375), p1=(0.625, 0.625)):
    """Delta measures at p0 and p1 (section 4.2): one cell of value 1/h^2 each."""
    out = []
    for p in (p0, p1):
        f = np.zeros((N, N), dtype=np.float64)
        j = min(int(p[0] * N), N - 1)
        i = min(int(p[1] * N), N - 1)
        f[i, j] = float(N * N)
        out.append(np.ascontiguousarray(f, dtype=np.float32))
    return out[0], out[1]


def random_state(N: int, seed: int, n_fields: int, scale: float = 1.0):
    """``n_fields`` i.i.d. U(-scale, scale) float32 planes (random solver states)."""
    rng = np.random.default_rng(seed)
    return [np.ascontiguousarray(rng.uniform(-scale, scale, size=(N, N)), dtype=np.float32)
            for _ in range(n_fields)]


# ------------------------------------------------------------- 3-D grids
# N x N x N cell-centred grid on [0,1]^3, arrays indexed (z, y, x), x fastest.

def cell_centres3(N: int):
    """Return (x, y, z) float64 arrays of shape (N, N, N) holding cell centres."""
    c = (np.arange(N, dtype=np.float64) + 0.5) / N
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z


def ball_image3(N: int, radius: float = 0.25, centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Indicator of a ball (the 3-D counterpart of the section-4.1 disc)."""
    x, y, z = cell_centres3(N)
    img = ((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2 <= radius * radius)
    return np.ascontiguousarray(img, dtype=np.float32)


def translated_balls3(N: int, radius: float = 0.25, c0=(0.375, 0.375, 0.375), c1=(0.625, 0.625, 0.625)):
    """Uniform unit-mass balls translated by (1/4, 1/4, 1/4), each normalised to h^3 sum f = 1."""
    x, y, z = cell_centres3(N)
    out = []
    for c in (c0, c1):
        f = ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= radius * radius).astype(np.float64)
        f /= f.sum() / N ** 3
        out.append(np.ascontiguousarray(f, dtype=np.float32))
    return out[0], out[1]


def gaussian_mixture_pair3(N: int, seed: int, n_comp: int = 8, floor: float = 1e-3):
    """The 3-D form of gaussian_mixture_pair: per component centre ~ U(0.1, 0.9)^3,
    width ~ U(0.04, 0.12), weight ~ U(0, 1) (drawn in that order, f0's
    components first), plus the floor, normalised to h^3 sum f = 1."""
    rng = np.random.default_rng(seed)
    x, y, z = cell_centres3(N)
    out = []
    for _ in range(2):
        params = [(rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9),
                   rng.uniform(0.04, 0.12), rng.uniform(0.0, 1.0)) for _ in range(n_comp)]
        f = np.zeros((N, N, N), dtype=np.float64)
        for cx, cy, cz, sd, w in params:
            f += w * np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2 * sd * sd)) / (2 * np.pi * sd * sd) ** 1.5
        f += floor
        f /= f.sum() / N ** 3
        out.append(np.ascontiguousarray(f, dtype=np.float32))
    return out[0], out[1]
