"""FP64 CPU oracle of G-prox PDHG for the ROF and L1-EMD (Beckmann) problems.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this module.  The product path (the CUDA library and its Python binding) never
imports, links or calls anything here, and this module imports nothing from
the product.

It is a plain, slow, obviously-correct restatement of the method in float64:
  * Algorithm 2 (G-prox PDHG) of Jacobs, Leger, Li, Osher, arXiv 1805.09453,
    section 3, instantiated for ROF (section 3.1) and EMD (section 3.2);
  * the Neumann Laplacian inverted in the cosine basis, which is what the
    even-reflection argument of Appendix A gives (scipy.fft's orthonormal
    DCT-II is used as a library primitive for that step);
  * the step-size rules of sections 3.1 / 4.1 (ROF) and 4.2 (EMD).

Readings of points the paper leaves open:
  R1  cell-centred N x N grid on [0,1]^2, h = 1/N;
  R2  forward differences for grad with a zero last slot (zero Neumann flux),
      div = -grad^T (backward differences), Laplacian = div grad (5-point
      Neumann stencil).  With this choice K^T K = -Laplacian exactly, so the
      G-prox metric is exact and the cosine basis diagonalises it;
  R3  inner products are h^2-weighted (L2 on the unit square);
  R4  the pointwise norm is the isotropic |(px, py)|_2 at one cell;
  R5  the "+1/(2 sigma)" inside the argmax of Algorithms 1-2 is read as "-";
      the closed-form projections printed in sections 3.1 and 3.2 are used;
  R6  EMD sign convention div m = f0 - f1 (the paper writes rho1 - rho0; the
      two are the same problem under m -> -m);
  R7  zero initial state (u0 = 0, p0 = pbar0 = 0; EMD m0 = grad psi);
  R8  sigma = 1/tau (sections 3.1, 3.2 and 4), times an optional multiplier;
  R9  ROF tau = min(sqrt(lambda) T / sqrt(eps), ||grad I||_L2) with
      T = min(||I||_TV, lambda/2 ||I - mean(I)||^2): the section-4.1 rule with
      the a-priori bound of section 3.1 on ||u*||_TV (dimension constants
      dropped, as section 4.1 does); a constant image (tau = 0) uses tau = 1;
  R10 EMD tau = sigma = 1 for bounded densities (section 4.2, discs);
  R11 ROF gap = P(u) - D(p) with D(p) = -(I, div p) - ||div p||^2/(2 lambda);
      EMD gap = P(m) - D(phi) with phi = Lap^{-1} div p and
      D(phi) = (phi, f1 - f0) / max(1, max|grad phi|) (a valid lower bound by
      weak duality for any feasible m; the paper prints no EMD gap formula);
      relative gap = (P - D) / max(|P|, |D|).

Every function here is pinned by tests under ``tests/`` against closed forms,
invariants, textbook matrices or brute-force solvers on tiny grids.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

__all__ = [
    "grad", "div", "laplacian", "eigenvalues", "helmholtz_solve", "project",
    "rof_step_rule", "rof_init", "rof_iterate", "rof_primal", "rof_dual", "rof_gap",
    "emd_init", "emd_iterate", "emd_primal", "emd_dual", "emd_gap", "emd_mass_residual",
    "rel_gap", "rof_solve", "emd_solve",
]

_WORKERS = -1  # scipy.fft threads: all host cores


# ---------------------------------------------------------------------------
# Discrete operators (reading R2)
# ---------------------------------------------------------------------------

def grad(u: np.ndarray, h: float):
    """Forward-difference gradient with zero last slots (Neumann flux = 0)."""
    gx = np.zeros_like(u)
    gy = np.zeros_like(u)
    gx[:, :-1] = (u[:, 1:] - u[:, :-1]) / h
    gy[:-1, :] = (u[1:, :] - u[:-1, :]) / h
    return gx, gy


def div(px: np.ndarray, py: np.ndarray, h: float) -> np.ndarray:
    """Divergence = -grad^T; the last slot of each component is ignored."""
    d = np.zeros_like(px)
    d[:, :-1] += px[:, :-1]
    d[:, 1:] -= px[:, :-1]
    d[:-1, :] += py[:-1, :]
    d[1:, :] -= py[:-1, :]
    return d / h


def laplacian(u: np.ndarray, h: float) -> np.ndarray:
    """5-point Neumann Laplacian, div(grad u)."""
    gx, gy = grad(u, h)
    return div(gx, gy, h)


def eigenvalues(N: int, h: float) -> np.ndarray:
    """Eigenvalues of the 1-D Neumann -d^2/dx^2 in the cosine basis (Appendix A):
    mu_k = (4/h^2) sin^2(pi k / (2N))."""
    k = np.arange(N, dtype=np.float64)
    return (4.0 / (h * h)) * np.sin(np.pi * k / (2.0 * N)) ** 2


def helmholtz_solve(b: np.ndarray, alpha: float, h: float) -> np.ndarray:
    """Solve (alpha - Laplacian) x = b with zero Neumann conditions.

    The even reflection of Appendix A turns the problem into a cosine series,
    in which -Laplacian is diagonal with entries mu_k + mu_l.  For alpha = 0
    the constant mode is set to zero (the solution with zero mean; b's own
    mean is dropped).
    """
    N = b.shape[0]
    assert b.shape == (N, N)
    mu = eigenvalues(N, h)
    denom = alpha + mu[:, None] + mu[None, :]
    bh = sfft.dctn(b, type=2, norm="ortho", workers=_WORKERS)
    if alpha == 0.0:
        denom[0, 0] = 1.0
        bh[0, 0] = 0.0
    return sfft.idctn(bh / denom, type=2, norm="ortho", workers=_WORKERS)


def project(qx: np.ndarray, qy: np.ndarray, norm: str = "l2"):
    """Projection onto the pointwise unit ball (prox of the L-infinity indicator).

    ``l2``: q / max(1, |q|_2) (sections 3.1, 3.2).  ``l1``: componentwise clip
    to [-1, 1], the projection for the anisotropic |mx| + |my| norm (used only
    to pin the iteration against an exact LP on tiny grids).
    """
    if norm == "l2":
        nrm = np.maximum(1.0, np.hypot(qx, qy))
        return qx / nrm, qy / nrm
    if norm == "l1":
        return np.clip(qx, -1.0, 1.0), np.clip(qy, -1.0, 1.0)
    raise ValueError(norm)


def _pointwise_norm(x, y, norm):
    return np.hypot(x, y) if norm == "l2" else np.abs(x) + np.abs(y)


def _dual_norm_max(x, y, norm):
    return float(np.max(np.hypot(x, y))) if norm == "l2" else float(max(np.max(np.abs(x)), np.max(np.abs(y))))


def rel_gap(P: float, D: float) -> float:
    """Relative duality gap (P - D) / max(|P|, |D|) (0 when both vanish)."""
    s = max(abs(P), abs(D))
    return 0.0 if s == 0.0 else (P - D) / s


# ---------------------------------------------------------------------------
# ROF (section 3.1)
# ---------------------------------------------------------------------------

def rof_step_rule(I: np.ndarray, lam: float, eps: float = 1e-3, tau_scale: float = 1.0):
    """Step sizes for ROF (reading R9): returns (tau, sigma, stats)."""
    I = np.asarray(I, dtype=np.float64)
    N = I.shape[0]
    h = 1.0 / N
    gx, gy = grad(I, h)
    tv = h * h * float(np.sum(np.hypot(gx, gy)))
    grad_l2 = math.sqrt(h * h * float(np.sum(gx * gx + gy * gy)))
    fid = 0.5 * lam * h * h * float(np.sum((I - I.mean()) ** 2))
    T = min(tv, fid)
    tau = min(math.sqrt(lam) * T / math.sqrt(eps), grad_l2)
    if not tau > 0.0:
        tau = 1.0
    tau *= tau_scale
    return tau, 1.0 / tau, {"tv": tv, "grad_l2": grad_l2, "fid": fid}


def rof_init(I, u0=None, p0=None, pbar0=None):
    N = I.shape[0]
    z = np.zeros((N, N))
    u = z.copy() if u0 is None else np.array(u0, dtype=np.float64)
    px, py = (z.copy(), z.copy()) if p0 is None else (np.array(p0[0], np.float64), np.array(p0[1], np.float64))
    if pbar0 is None:
        pbx, pby = px.copy(), py.copy()
    else:
        pbx, pby = np.array(pbar0[0], np.float64), np.array(pbar0[1], np.float64)
    return {"u": u, "px": px, "py": py, "pbx": pbx, "pby": pby, "n": 0}


def rof_iterate(state: dict, I: np.ndarray, lam: float, tau: float, sigma: float,
                n_iters: int, callback=None) -> dict:
    """Run ``n_iters`` G-prox PDHG iterations for ROF (section 3.1 updates).

    u_{n+1} = (lam tau - Lap)^{-1} (lam tau I + tau div pbar_n - Lap u_n)
    p_{n+1} = (p_n + sigma grad u_{n+1}) / max(1, |p_n + sigma grad u_{n+1}|)
    pbar_{n+1} = 2 p_{n+1} - p_n
    """
    I = np.asarray(I, dtype=np.float64)
    h = 1.0 / I.shape[0]
    u, px, py, pbx, pby = state["u"], state["px"], state["py"], state["pbx"], state["pby"]
    for _ in range(n_iters):
        rhs = lam * tau * I + tau * div(pbx, pby, h) - laplacian(u, h)
        u = helmholtz_solve(rhs, lam * tau, h)
        gx, gy = grad(u, h)
        nx, ny = project(px + sigma * gx, py + sigma * gy)
        pbx, pby = 2.0 * nx - px, 2.0 * ny - py
        px, py = nx, ny
        state["n"] += 1
        if callback is not None:
            callback(state["n"], u, px, py)
    state.update(u=u, px=px, py=py, pbx=pbx, pby=pby)
    return state


def rof_primal(u, I, lam):
    """ROF energy ||u||_TV + lam/2 ||u - I||^2 (isotropic, h^2-weighted)."""
    u = np.asarray(u, np.float64)
    I = np.asarray(I, np.float64)
    h = 1.0 / u.shape[0]
    gx, gy = grad(u, h)
    return h * h * float(np.sum(np.hypot(gx, gy))) + 0.5 * lam * h * h * float(np.sum((u - I) ** 2))


def rof_dual(px, py, I, lam):
    """Dual value min_u L(u, p) = -(I, div p) - ||div p||^2 / (2 lam), for |p| <= 1."""
    I = np.asarray(I, np.float64)
    h = 1.0 / I.shape[0]
    d = div(np.asarray(px, np.float64), np.asarray(py, np.float64), h)
    return -h * h * float(np.sum(I * d)) - h * h * float(np.sum(d * d)) / (2.0 * lam)


def rof_gap(u, px, py, I, lam):
    P = rof_primal(u, I, lam)
    D = rof_dual(px, py, I, lam)
    return P, D, rel_gap(P, D)


def rof_solve(I, lam, n_iters=None, tol=None, gap_every=10, max_iters=100000,
              eps=1e-3, tau=None, sigma=None, tau_scale=1.0):
    """Convenience driver: fixed iteration count, or run until rel gap <= tol."""
    I = np.asarray(I, np.float64)
    if tau is None:
        tau, sigma, _ = rof_step_rule(I, lam, eps, tau_scale)
    elif sigma is None:
        sigma = 1.0 / tau
    st = rof_init(I)
    if n_iters is not None:
        rof_iterate(st, I, lam, tau, sigma, n_iters)
    else:
        while st["n"] < max_iters:
            rof_iterate(st, I, lam, tau, sigma, gap_every)
            if rof_gap(st["u"], st["px"], st["py"], I, lam)[2] <= tol:
                break
    P, D, g = rof_gap(st["u"], st["px"], st["py"], I, lam)
    st.update(primal=P, dual=D, rel_gap=g, tau=tau, sigma=sigma)
    return st


# ---------------------------------------------------------------------------
# CP2: the accelerated PDHG the paper compares against (section 4.1, Tables 4-5)
# ---------------------------------------------------------------------------

def rof_cp2_steps(N: int):
    """Initial step sizes of section 4.1: tau0 = sigma0 = 1 / sqrt(||Lap||), with
    ||Lap|| = 2 mu_{N-1} the largest eigenvalue of the 5-point Neumann -Lap
    (so tau0 sigma0 ||grad^T grad|| = 1)."""
    h = 1.0 / N
    t0 = 1.0 / np.sqrt(2.0 * eigenvalues(N, h)[-1])
    return t0, t0


def rof_cp2_init(I, u0=None, p0=None):
    I = np.asarray(I, np.float64)
    N = I.shape[0]
    u = np.zeros_like(I) if u0 is None else np.array(u0, np.float64)
    z = np.zeros((N, N))
    px, py = (z.copy(), z.copy()) if p0 is None else (np.array(p0[0], np.float64), np.array(p0[1], np.float64))
    tau, sigma = rof_cp2_steps(N)
    return {"u": u, "ubar": u.copy(), "px": px, "py": py, "tau": tau, "sigma": sigma, "n": 0}


def rof_cp2_iterate(state: dict, I: np.ndarray, lam: float, n_iters: int, gamma: float = None,
                    callback=None) -> dict:
    """``n_iters`` iterations of the accelerated primal-dual method for the ROF
    saddle problem L(u, p) = (grad u, p) + lam/2 ||u - I||^2 - chi(|p| <= 1):
    the primal term is strongly convex with modulus gamma = lam (h^2-weighted
    L2), which the method exploits by shrinking tau and growing sigma:

    p_{n+1}  = proj(p_n + sigma_n grad ubar_n)
    u_{n+1}  = (u_n + tau_n div p_{n+1} + tau_n lam I) / (1 + tau_n lam)
    theta_n  = 1 / sqrt(1 + 2 gamma tau_n)
    tau_{n+1} = theta_n tau_n,  sigma_{n+1} = sigma_n / theta_n
    ubar_{n+1} = u_{n+1} + theta_n (u_{n+1} - u_n)
    """
    I = np.asarray(I, np.float64)
    h = 1.0 / I.shape[0]
    g = lam if gamma is None else gamma
    u, ubar, px, py = state["u"], state["ubar"], state["px"], state["py"]
    tau, sigma = state["tau"], state["sigma"]
    for _ in range(n_iters):
        gx, gy = grad(ubar, h)
        px, py = project(px + sigma * gx, py + sigma * gy)
        un = (u + tau * div(px, py, h) + tau * lam * I) / (1.0 + tau * lam)
        theta = 1.0 / np.sqrt(1.0 + 2.0 * g * tau)
        ubar = un + theta * (un - u)
        u = un
        tau, sigma = theta * tau, sigma / theta
        state["n"] += 1
        if callback is not None:
            callback(state["n"], u, px, py)
    state.update(u=u, ubar=ubar, px=px, py=py, tau=tau, sigma=sigma)
    return state


def rof_cp2_solve(I, lam, n_iters=None, tol=None, gap_every=10, max_iters=200000):
    """CP2 driver: fixed iteration count, or run until the ROF rel gap <= tol."""
    I = np.asarray(I, np.float64)
    st = rof_cp2_init(I)
    if n_iters is not None:
        rof_cp2_iterate(st, I, lam, n_iters)
    else:
        while st["n"] < max_iters:
            rof_cp2_iterate(st, I, lam, gap_every)
            if rof_gap(st["u"], st["px"], st["py"], I, lam)[2] <= tol:
                break
    P, D, g = rof_gap(st["u"], st["px"], st["py"], I, lam)
    st.update(primal=P, dual=D, rel_gap=g)
    return st


# ---------------------------------------------------------------------------
# EMD / Beckmann (section 3.2)
# ---------------------------------------------------------------------------

def emd_init(f0, f1, m0=None, p0=None, pbar0=None):
    """Hodge split: psi solves Lap psi = f0 - f1 (Neumann), m0 = grad psi (u0 = 0)."""
    f0 = np.asarray(f0, np.float64)
    f1 = np.asarray(f1, np.float64)
    N = f0.shape[0]
    h = 1.0 / N
    psi = -helmholtz_solve(f0 - f1, 0.0, h)
    if m0 is None:
        mx, my = grad(psi, h)
    else:
        mx, my = np.array(m0[0], np.float64), np.array(m0[1], np.float64)
    z = np.zeros((N, N))
    px, py = (z.copy(), z.copy()) if p0 is None else (np.array(p0[0], np.float64), np.array(p0[1], np.float64))
    if pbar0 is None:
        pbx, pby = px.copy(), py.copy()
    else:
        pbx, pby = np.array(pbar0[0], np.float64), np.array(pbar0[1], np.float64)
    return {"psi": psi, "mx": mx, "my": my, "px": px, "py": py, "pbx": pbx, "pby": pby, "n": 0}


def leray(px, py, h):
    """Leray projection onto discretely divergence-free fields: p - grad Lap^{-1} div p."""
    q = -helmholtz_solve(div(px, py, h), 0.0, h)  # Lap q = div p
    gx, gy = grad(q, h)
    return px - gx, py - gy


def emd_iterate(state: dict, tau: float, sigma: float, n_iters: int, norm: str = "l2",
                callback=None) -> dict:
    """Run ``n_iters`` G-prox PDHG iterations for EMD (section 3.2 updates),
    written for m = u + grad psi:

    m_{n+1} = m_n - tau * Leray(pbar_n)
    p_{n+1} = proj(p_n + sigma m_{n+1})
    pbar_{n+1} = 2 p_{n+1} - p_n
    """
    h = 1.0 / state["mx"].shape[0]
    mx, my, px, py, pbx, pby = (state[k] for k in ("mx", "my", "px", "py", "pbx", "pby"))
    for _ in range(n_iters):
        lx, ly = leray(pbx, pby, h)
        mx = mx - tau * lx
        my = my - tau * ly
        nx, ny = project(px + sigma * mx, py + sigma * my, norm)
        pbx, pby = 2.0 * nx - px, 2.0 * ny - py
        px, py = nx, ny
        state["n"] += 1
        if callback is not None:
            callback(state["n"], mx, my, px, py)
    state.update(mx=mx, my=my, px=px, py=py, pbx=pbx, pby=pby)
    return state


def emd_primal(mx, my, norm: str = "l2"):
    h = 1.0 / mx.shape[0]
    return h * h * float(np.sum(_pointwise_norm(np.asarray(mx, np.float64), np.asarray(my, np.float64), norm)))


def emd_dual(px, py, f0, f1, norm: str = "l2"):
    """Lower bound (phi, f1 - f0) / max(1, max|grad phi|*) with phi = Lap^{-1} div p.

    Returns (D, phi, s).  |.|* is the dual of the pointwise norm (l2 -> l2,
    l1 -> l-infinity).
    """
    f0 = np.asarray(f0, np.float64)
    f1 = np.asarray(f1, np.float64)
    h = 1.0 / f0.shape[0]
    phi = -helmholtz_solve(div(np.asarray(px, np.float64), np.asarray(py, np.float64), h), 0.0, h)
    gx, gy = grad(phi, h)
    s = max(1.0, _dual_norm_max(gx, gy, norm))
    D = h * h * float(np.sum(phi * (f1 - f0))) / s
    return D, phi, s


def emd_mass_residual(mx, my, f0, f1):
    """h^2 sum |div m - (f0 - f1)| / h^2 sum |f0 - f1| (0/0 -> 0)."""
    f0 = np.asarray(f0, np.float64)
    f1 = np.asarray(f1, np.float64)
    h = 1.0 / f0.shape[0]
    r = np.abs(div(np.asarray(mx, np.float64), np.asarray(my, np.float64), h) - (f0 - f1))
    den = float(np.sum(np.abs(f0 - f1)))
    return float(np.sum(r)) / den if den > 0 else float(np.sum(r))


def emd_gap(state, f0, f1, norm: str = "l2"):
    P = emd_primal(state["mx"], state["my"], norm)
    D, phi, s = emd_dual(state["px"], state["py"], f0, f1, norm)
    return P, D, rel_gap(P, D)


def emd_solve(f0, f1, n_iters=None, tol=None, gap_every=10, max_iters=100000,
              tau=1.0, sigma=None, norm: str = "l2"):
    """Convenience driver: fixed iteration count, or run until rel gap <= tol."""
    if sigma is None:
        sigma = 1.0 / tau
    st = emd_init(f0, f1)
    if n_iters is not None:
        emd_iterate(st, tau, sigma, n_iters, norm)
    else:
        while st["n"] < max_iters:
            emd_iterate(st, tau, sigma, gap_every, norm)
            if emd_gap(st, f0, f1, norm)[2] <= tol:
                break
    P, D, g = emd_gap(st, f0, f1, norm)
    st.update(primal=P, dual=D, rel_gap=g, tau=tau, sigma=sigma,
              mass_residual=emd_mass_residual(st["mx"], st["my"], f0, f1))
    return st
