"""Pins of the oracle's EMD iteration (section 3.2) against facts the paper and
the mathematics fix:

* mass balance: the Leray projection maps into discretely divergence-free
  fields, so div m_n = f0 - f1 at every iterate (the Hodge split of
  section 3.2);
* EMD(f, f) = 0 and symmetry EMD(f0, f1) = EMD(f1, f0);
* exact 1-D identity: for densities varying along x only the discrete optimum
  is sum_j h |F0_j - F1_j| with F_j = h sum_{k<=j} f_k (the forced flux plus a
  tight dual certificate);
* brute force on 8 x 8 grids: the anisotropic (l1) variant against an exact
  LP (HiGHS), the isotropic problem against its dual solved by SLSQP;
* the duality gap is non-negative and falls (section 2.1), and the paper's
  translated-disc value 1/sqrt(8) (section 4.2) is approached on a grid.
"""
import math

import numpy as np
import pytest
from scipy.optimize import linprog, minimize

from oracle import gprox_oracle as O
from paper_1805_09453_gb300 import synth


def _rand_pair(N, seed):
    rng = np.random.default_rng(seed)
    h = 1.0 / N
    f0 = rng.uniform(0.1, 1, (N, N))
    f1 = rng.uniform(0.1, 1, (N, N))
    return f0 / (f0.sum() * h * h), f1 / (f1.sum() * h * h)


def test_mass_balance_every_iterate():
    f0, f1 = synth.gaussian_mixture_pair(32, 7)
    f0, f1 = f0.astype(np.float64), f1.astype(np.float64)
    f1 *= f0.sum() / f1.sum()  # exactly equal masses in float64
    h = 1.0 / 32
    st = O.emd_init(f0, f1)
    worst = []
    O.emd_iterate(st, 1.0, 1.0, 50, callback=lambda n, mx, my, px, py: worst.append(
        np.abs(O.div(mx, my, h) - (f0 - f1)).max()))
    assert max(worst) < 1e-10 * np.abs(f0 - f1).max()


def test_identical_densities_zero():
    f0, _ = synth.gaussian_mixture_pair(16, 2)
    st = O.emd_solve(f0, f0, n_iters=20)
    assert st["primal"] == 0.0 and abs(st["dual"]) == 0.0


def test_symmetry():
    f0, f1 = _rand_pair(8, 11)
    a = O.emd_solve(f0, f1, tol=1e-10, max_iters=200000)
    b = O.emd_solve(f1, f0, tol=1e-10, max_iters=200000)
    assert abs(a["primal"] - b["primal"]) < 1e-8 * a["primal"]


@pytest.mark.parametrize("seed", [0, 1])
def test_exact_1d_identity(seed):
    N = 32
    h = 1.0 / N
    rng = np.random.default_rng(seed)
    g0 = rng.uniform(0.2, 1, N)
    g1 = rng.uniform(0.2, 1, N)
    g0 /= g0.sum() * h
    g1 /= g1.sum() * h
    F0 = h * np.cumsum(g0)
    F1 = h * np.cumsum(g1)
    exact = h * np.sum(np.abs(F0 - F1))
    f0, f1 = np.tile(g0, (N, 1)), np.tile(g1, (N, 1))
    st = O.emd_solve(f0, f1, tol=1e-10, max_iters=400000)
    assert st["rel_gap"] <= 1e-10
    assert abs(st["primal"] - exact) < 1e-8 * exact


def _div_matrix(N):
    h = 1.0 / N
    nv = 2 * N * (N - 1)
    A = np.zeros((N * N, nv))
    for k in range(nv):
        e = np.zeros(nv)
        e[k] = 1.0
        px = np.zeros((N, N))
        py = np.zeros((N, N))
        px[:, :-1] = e[: N * (N - 1)].reshape(N, N - 1)
        py[:-1, :] = e[N * (N - 1):].reshape(N - 1, N)
        A[:, k] = O.div(px, py, h).ravel()
    return A


def test_brute_force_8x8_l1_lp():
    N = 8
    h = 1.0 / N
    f0, f1 = _rand_pair(N, 5)
    A = _div_matrix(N)
    nv = A.shape[1]
    res = linprog(h * h * np.ones(2 * nv), A_eq=np.hstack([A, -A]), b_eq=(f0 - f1).ravel(),
                  bounds=(0, None), method="highs")
    assert res.status == 0
    st = O.emd_solve(f0, f1, tol=1e-11, max_iters=400000, norm="l1")
    assert abs(st["primal"] - res.fun) < 1e-9 * res.fun
    assert st["mass_residual"] < 1e-9


def test_brute_force_8x8_isotropic_dual():
    N = 8
    h = 1.0 / N
    f0, f1 = _rand_pair(N, 5)

    def phi_of(x):
        return np.concatenate([[0.0], x]).reshape(N, N)

    res = minimize(lambda x: -h * h * np.sum(phi_of(x) * (f1 - f0)), np.zeros(N * N - 1),
                   jac=lambda x: -h * h * (f1 - f0).ravel()[1:], method="SLSQP",
                   constraints=[{"type": "ineq", "fun": lambda x: (1 - sum(g ** 2 for g in O.grad(phi_of(x), h))).ravel()}],
                   options={"ftol": 1e-15, "maxiter": 2000})
    assert res.success
    st = O.emd_solve(f0, f1, tol=1e-11, max_iters=400000)
    assert abs(st["primal"] - (-res.fun)) < 1e-8 * st["primal"]


def test_gap_nonneg_and_falls():
    f0, f1 = synth.gaussian_mixture_pair(32, 4)
    st = O.emd_init(f0, f1)
    gaps = []
    for _ in range(40):
        O.emd_iterate(st, 1.0, 1.0, 25)
        P, D, g = O.emd_gap(st, f0, f1)
        assert P - D >= -1e-12
        gaps.append(g)
    assert gaps[-1] < 0.05 * gaps[0]


def test_translated_discs_near_the_translation_length():
    """Section 4.2: translated measures are |v| = 1/sqrt(8) apart (cited
    fixture tests/golden/section42_translation.json); at 48^2 the grid's
    anisotropy leaves the discrete optimum within 3 %."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "section42_translation.json")))
    assert abs(g["emd_distance"] - math.hypot(*g["translation"])) < 1e-15
    f0, f1 = synth.translated_discs(48)
    st = O.emd_solve(f0, f1, tol=1e-4, max_iters=20000)
    assert abs(st["primal"] - g["emd_distance"]) < 0.03 * g["emd_distance"]


@pytest.mark.parametrize("N", [16, 64])
def test_dual_of_a_gradient_field_is_its_potential(N):
    """Closed form of the dual bound (weak duality, section 2.1, for the
    constraint of section 3.2): for p = D phi with phi = 0.6 x + 0.8 y at the
    cell centres (forward differences, zero last slots), div p is the
    5-point Neumann Laplacian of phi, so Lap^-1 div p is phi less its mean,
    max |D phi| = |(0.6, 0.8)| = 1 (no normalisation), and the bound is
    h^2 sum (phi - mean) (f1 - f0)."""
    h = 1.0 / N
    x = (np.arange(N) + 0.5) * h
    phi = 0.6 * x[None, :] + 0.8 * x[:, None]
    px, py = O.grad(phi, h)
    f0, f1 = synth.gaussian_mixture_pair(N, 7)
    D, pot, s = O.emd_dual(px, py, f0, f1)
    c = phi - phi.mean()
    assert np.abs(pot - c).max() < 1e-12
    assert abs(s - 1.0) < 1e-12
    exact = h * h * float(np.sum(c * (f1.astype(np.float64) - f0.astype(np.float64))))
    assert abs(D - exact) <= 1e-12 * abs(exact)
