"""FP64 CPU oracle of G-prox PDHG on three-dimensional grids (ROF and L1-EMD).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module; the
product path never imports, links or calls anything here, and this module
imports nothing from the product.

The method of Algorithm 2 (section 3) is stated for general dimension d
(the ROF and EMD analyses of sections 3.1 / 3.2 carry d through their
constants); this is its d = 3 instance, in plain float64, written out the
same way as the two-dimensional oracle:
  * cell-centred N x N x N grid on [0,1]^3, h = 1/N, arrays indexed
    (z, y, x) (x fastest);
  * grad = forward differences with a zero last slot along each axis, div =
    -grad^T (backward differences), Laplacian = div grad (7-point Neumann
    stencil): K^T K = -Laplacian exactly and the cosine basis of Appendix A
    diagonalises it with mu_i + mu_j + mu_k, mu_k = (4/h^2) sin^2(pi k / 2N)
    (scipy.fft's orthonormal DCT-II over the three axes as a library
    primitive);
  * inner products h^3-weighted; the pointwise norm is the isotropic
    |(px, py, pz)|_2;
  * ROF: u_{n+1} = (lambda tau - Lap)^{-1}(lambda tau I + tau div pbar_n -
    Lap u_n), p_{n+1} = proj(p_n + sigma grad u_{n+1}), pbar = 2 p_{n+1} - p_n;
    step rule tau = min(sqrt(lambda) T / sqrt(eps), ||grad I||_L2),
    T = min(||I||_TV, lambda/2 ||I - mean I||^2), sigma = 1/tau;
  * EMD (div m = f0 - f1): m_{n+1} = m_n - tau Leray(pbar_n) with
    Leray(q) = q - grad Lap^{-1} div q, p_{n+1} = proj(p_n + sigma m_{n+1});
    m_0 = grad psi, Lap psi = f0 - f1; gap with phi = Lap^{-1} div p,
    D = (phi, f1 - f0) / max(1, max |grad phi|).
Every function is pinned by ``tests/test_oracle_3d.py`` (adjointness, the
cosine eigenvectors, a dense solve, invariants, the ball's two-valued ROF
solution, the one-dimensional EMD identity).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

__all__ = [
    "grad3", "div3", "laplacian3", "helmholtz_solve3", "project3",
    "rof_step_rule3", "rof_solve3", "rof_primal3", "rof_dual3",
    "emd_init3", "emd_iterate3", "emd_primal3", "emd_dual3", "emd_solve3",
]


def grad3(u: np.ndarray, h: float):
    """Forward differences along x, y, z, zero in each axis's last slot."""
    g = []
    for ax in (2, 1, 0):  # x, y, z
        d = np.zeros_like(u)
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[ax] = slice(0, -1)
        sl_hi[ax] = slice(1, None)
        d[tuple(sl_lo)] = (u[tuple(sl_hi)] - u[tuple(sl_lo)]) / h
        g.append(d)
    return g[0], g[1], g[2]


def div3(px: np.ndarray, py: np.ndarray, pz: np.ndarray, h: float) -> np.ndarray:
    """-grad^T: backward differences, each component's last slot ignored."""
    out = np.zeros_like(px)
    for p, ax in ((px, 2), (py, 1), (pz, 0)):
        q = p.copy()
        sl_last = [slice(None)] * 3
        sl_last[ax] = -1
        q[tuple(sl_last)] = 0.0  # structural zero slot
        prev = np.zeros_like(q)
        sl_dst = [slice(None)] * 3
        sl_src = [slice(None)] * 3
        sl_dst[ax] = slice(1, None)
        sl_src[ax] = slice(0, -1)
        prev[tuple(sl_dst)] = q[tuple(sl_src)]
        out += (q - prev) / h
    return out


def laplacian3(u: np.ndarray, h: float) -> np.ndarray:
    return div3(*grad3(u, h), h)


def _mu(N: int, h: float) -> np.ndarray:
    k = np.arange(N, dtype=np.float64)
    return (4.0 / (h * h)) * np.sin(np.pi * k / (2.0 * N)) ** 2


def helmholtz_solve3(b: np.ndarray, alpha: float, h: float) -> np.ndarray:
    """(alpha - Lap) x = b, zero Neumann conditions; alpha = 0: zero-mean solution."""
    N = b.shape[0]
    mu = _mu(N, h)
    den = alpha + mu[:, None, None] + mu[None, :, None] + mu[None, None, :]
    bh = sfft.dctn(b, type=2, norm="ortho")
    if alpha == 0.0:
        den[0, 0, 0] = 1.0
        bh[0, 0, 0] = 0.0
    return sfft.idctn(bh / den, type=2, norm="ortho")


def project3(qx, qy, qz):
    n = np.maximum(1.0, np.sqrt(qx * qx + qy * qy + qz * qz))
    return qx / n, qy / n, qz / n


# ------------------------------------------------------------------- ROF
def rof_step_rule3(I: np.ndarray, lam: float, eps: float = 1e-3):
    I = np.asarray(I, dtype=np.float64)
    h = 1.0 / I.shape[0]
    gx, gy, gz = grad3(I, h)
    mag = np.sqrt(gx * gx + gy * gy + gz * gz)
    h3 = h ** 3
    tv = h3 * mag.sum()
    grad_l2 = math.sqrt(h3 * (mag * mag).sum())
    fid = 0.5 * lam * h3 * ((I - I.mean()) ** 2).sum()
    tau = min(math.sqrt(lam) * min(tv, fid) / math.sqrt(eps), grad_l2)
    if not tau > 0:
        tau = 1.0
    return tau, 1.0 / tau


def rof_primal3(u, I, lam):
    h = 1.0 / u.shape[0]
    gx, gy, gz = grad3(u, h)
    return h ** 3 * (np.sqrt(gx * gx + gy * gy + gz * gz).sum() + 0.5 * lam * ((u - I) ** 2).sum())


def rof_dual3(px, py, pz, I, lam):
    h = 1.0 / I.shape[0]
    d = div3(px, py, pz, h)
    return h ** 3 * (-(I * d).sum() - (d * d).sum() / (2.0 * lam))


def rof_solve3(I, lam, n_iters, tau=None, sigma=None, callback=None):
    """n_iters iterations from the zero state; returns the final iterate and P, D."""
    I = np.asarray(I, dtype=np.float64)
    h = 1.0 / I.shape[0]
    if tau is None:
        tau, sigma = rof_step_rule3(I, lam)
    u = np.zeros_like(I)
    px, py, pz = np.zeros_like(I), np.zeros_like(I), np.zeros_like(I)
    bx, by, bz = px, py, pz
    for n in range(n_iters):
        rhs = lam * tau * I + tau * div3(bx, by, bz, h) - laplacian3(u, h)
        u = helmholtz_solve3(rhs, lam * tau, h)
        gx, gy, gz = grad3(u, h)
        nx, ny, nz = project3(px + sigma * gx, py + sigma * gy, pz + sigma * gz)
        bx, by, bz = 2 * nx - px, 2 * ny - py, 2 * nz - pz
        px, py, pz = nx, ny, nz
        if callback is not None:
            callback(n + 1, u, px, py, pz)
    return {"u": u, "p": (px, py, pz), "tau": tau, "sigma": sigma,
            "primal": rof_primal3(u, I, lam), "dual": rof_dual3(px, py, pz, I, lam)}


# ------------------------------------------------------------------- EMD
def emd_init3(f0, f1):
    f0 = np.asarray(f0, dtype=np.float64)
    f1 = np.asarray(f1, dtype=np.float64)
    h = 1.0 / f0.shape[0]
    psi = -helmholtz_solve3(f0 - f1, 0.0, h)  # Lap psi = f0 - f1
    return {"m": grad3(psi, h), "p": (np.zeros_like(f0),) * 3, "pbar": (np.zeros_like(f0),) * 3, "n": 0}


def _leray3(qx, qy, qz, h):
    c = -helmholtz_solve3(div3(qx, qy, qz, h), 0.0, h)  # Lap c = div q
    gx, gy, gz = grad3(c, h)
    return qx - gx, qy - gy, qz - gz


def emd_iterate3(st, tau, sigma, n_iters, callback=None):
    h = 1.0 / st["m"][0].shape[0]
    (mx, my, mz), (px, py, pz), (bx, by, bz) = st["m"], st["p"], st["pbar"]
    for _ in range(n_iters):
        lx, ly, lz = _leray3(bx, by, bz, h)
        mx, my, mz = mx - tau * lx, my - tau * ly, mz - tau * lz
        nx, ny, nz = project3(px + sigma * mx, py + sigma * my, pz + sigma * mz)
        bx, by, bz = 2 * nx - px, 2 * ny - py, 2 * nz - pz
        px, py, pz = nx, ny, nz
        st["n"] += 1
        if callback is not None:
            callback(st["n"], mx, my, mz, px, py, pz)
    st.update(m=(mx, my, mz), p=(px, py, pz), pbar=(bx, by, bz))
    return st


def emd_primal3(mx, my, mz):
    h = 1.0 / mx.shape[0]
    return h ** 3 * np.sqrt(mx * mx + my * my + mz * mz).sum()


def emd_dual3(px, py, pz, f0, f1):
    h = 1.0 / px.shape[0]
    phi = -helmholtz_solve3(div3(px, py, pz, h), 0.0, h)  # Lap phi = div p
    gx, gy, gz = grad3(phi, h)
    s = max(1.0, float(np.sqrt(gx * gx + gy * gy + gz * gz).max()))
    return h ** 3 * (phi * (np.asarray(f1, np.float64) - np.asarray(f0, np.float64))).sum() / s


def emd_solve3(f0, f1, n_iters, tau=1.0, sigma=1.0):
    st = emd_init3(f0, f1)
    emd_iterate3(st, tau, sigma, n_iters)
    mx, my, mz = st["m"]
    px, py, pz = st["p"]
    return {**st, "primal": emd_primal3(mx, my, mz), "dual": emd_dual3(px, py, pz, f0, f1)}
