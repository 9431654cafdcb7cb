"""Pins of the oracle's ROF iteration (section 3.1) against facts the paper and
the mathematics fix:

* mean preservation: summing the u-update, sum(div pbar) = sum(Lap u) = 0
  under Neumann conditions, so mean(u_n) = mean(I) at every iterate;
* a constant image is a fixed point with p = 0;
* the duality gap is non-negative and falls to zero (section 2.1);
* lambda-strong convexity (Corollary 3.4): lam/2 ||u - u*||^2 <= P(u) - P(u*)
  <= gap;
* exact 1-D solution: for an image varying along x only the minimiser is
  row-constant and equals the 1-D ROF solution, computed exactly from the
  box-constrained dual least squares (scipy BVLS);
* 8 x 8 brute force: the dual QCQP max D(p) s.t. |p| <= 1 solved by SLSQP;
* the corrected disc closed form (section 3.1 / 4.1; the printed one is
  garbled): plateau values a = 1 - 2/(lam r), b = 2 pi r / (lam (1 - pi r^2))
  approached as N grows;
* the step rule on a straight edge: ||I||_TV = 1, ||grad I|| = sqrt(N),
  lam/2 ||I - mean I||^2 = lam / 8.
"""
import math

import numpy as np
import pytest
from scipy.optimize import lsq_linear, minimize

from oracle import gprox_oracle as O
from paper_1805_09453_gb300 import synth


def test_mean_preserved_every_iterate():
    I = synth.rof_image(32, 3).astype(np.float64)
    tau, sigma, _ = O.rof_step_rule(I, 8.0)
    means = []
    st = O.rof_init(I)
    O.rof_iterate(st, I, 8.0, tau, sigma, 40, callback=lambda n, u, px, py: means.append(u.mean()))
    assert np.max(np.abs(np.array(means) - I.mean())) < 1e-12


def test_constant_image_fixed_point():
    I = np.full((16, 16), 0.37)
    st = O.rof_solve(I, 8.0, n_iters=5)
    np.testing.assert_allclose(st["u"], I, atol=1e-13)
    assert np.abs(st["px"]).max() < 1e-12 and np.abs(st["py"]).max() < 1e-12


def test_gap_nonneg_and_to_zero_and_strong_convexity():
    I = synth.rof_image(32, 5).astype(np.float64)
    lam = 8.0
    ref = O.rof_solve(I, lam, tol=1e-12, max_iters=50000)
    assert ref["rel_gap"] <= 1e-12
    u_star, P_star = ref["u"], ref["primal"]
    tau, sigma, _ = O.rof_step_rule(I, lam)
    st = O.rof_init(I)
    h = 1.0 / 32
    gaps = []
    for _ in range(30):
        O.rof_iterate(st, I, lam, tau, sigma, 5)
        P, D, g = O.rof_gap(st["u"], st["px"], st["py"], I, lam)
        assert P - D >= -1e-12
        assert D <= P_star + 1e-12 <= P + 2e-12
        err2 = h * h * np.sum((st["u"] - u_star) ** 2)
        assert 0.5 * lam * err2 <= (P - D) + 1e-12
        gaps.append(g)
    assert gaps[-1] < 1e-3 * gaps[0]


def _div_matrix_1d(N, h):
    A = np.zeros((N, N - 1))
    for k in range(N - 1):
        A[k, k] += 1.0 / h
        A[k + 1, k] -= 1.0 / h
    return A


@pytest.mark.parametrize("seed,lam", [(1, 10.0), (2, 40.0)])
def test_exact_1d_solution(seed, lam):
    N = 32
    h = 1.0 / N
    rng = np.random.default_rng(seed)
    g = np.repeat(rng.uniform(0, 1, N // 4), 4) + 0.1 * rng.normal(size=N)
    A = _div_matrix_1d(N, h)
    # 1-D dual: min ||div p + lam g||^2, |p_j| <= 1; u = g + div p / lam
    res = lsq_linear(A, -lam * g, bounds=(-1, 1), method="bvls", tol=1e-15)
    w = g + A @ res.x / lam
    I = np.tile(g, (N, 1))
    st = O.rof_solve(I, lam, tol=1e-13, max_iters=100000)
    assert np.max(np.abs(st["u"] - w[None, :])) < 1e-10


def test_brute_force_8x8_dual_qcqp():
    N, lam = 8, 20.0
    h = 1.0 / N
    rng = np.random.default_rng(3)
    I = rng.uniform(0, 1, (N, N))
    nv = 2 * N * (N - 1)

    def unpack(z):
        px = np.zeros((N, N))
        py = np.zeros((N, N))
        px[:, :-1] = z[: N * (N - 1)].reshape(N, N - 1)
        py[:-1, :] = z[N * (N - 1):].reshape(N - 1, N)
        return px, py

    A = np.zeros((N * N, nv))
    for k in range(nv):
        e = np.zeros(nv)
        e[k] = 1.0
        A[:, k] = O.div(*unpack(e), h).ravel()
    Iv = I.ravel()

    def negD(z):
        d = A @ z
        return h * h * (Iv @ d) + h * h * (d @ d) / (2 * lam)

    def negD_grad(z):
        return h * h * (A.T @ Iv) + h * h * (A.T @ (A @ z)) / lam

    def cons(z):
        px, py = unpack(z)
        return (1 - px ** 2 - py ** 2).ravel()

    res = minimize(negD, np.zeros(nv), jac=negD_grad, method="SLSQP",
                   constraints=[{"type": "ineq", "fun": cons}],
                   options={"ftol": 1e-14, "maxiter": 1000})
    assert res.success
    st = O.rof_solve(I, lam, tol=1e-12, max_iters=100000)
    assert abs(st["primal"] - (-res.fun)) <= 1e-7 * abs(st["primal"])


def test_disc_closed_form_plateaus():
    lam, r = 20.0, 0.25
    a = 1 - 2 / (lam * r)
    b = 2 * math.pi * r / (lam * (1 - math.pi * r * r))
    assert a > b  # the two-valued solution exists for this lambda
    # mean of the two-valued solution equals the disc area (mass preserved)
    assert abs(math.pi * r * r * a + (1 - math.pi * r * r) * b - math.pi * r * r) < 1e-12
    errs = []
    for N in (16, 32, 64):
        I = synth.disc_image(N).astype(np.float64)
        u = O.rof_solve(I, lam, n_iters=3000)["u"]
        errs.append((abs(u[N // 2, N // 2] - a), abs(u[0, 0] - b)))
    assert all(e[0] < 0.02 and e[1] < 0.012 for e in errs)
    assert errs[2][0] < errs[0][0] and errs[2][1] < errs[1][1] < errs[0][1]


def test_printed_disc_solution_is_the_garbled_one():
    """Section 4.1 prints the disc's continuum solution (cited fixture
    tests/golden/section41_disc.json) as (1 - 8/lambda) I + 8 pi/(lambda (16 - pi)).
    An ROF minimiser keeps the mean of I (the fidelity's optimality condition
    sums to zero), and the printed form does not; the oracle's converged
    plateaus at lambda = 20 sit at the two-valued form (reading R12), not at
    the printed values."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "section41_disc.json")))
    r = g["radius"]
    area = math.pi * r * r
    for lam in (10.0, 20.0):
        inside = (1 - 8 / lam) + 8 * math.pi / (lam * (16 - math.pi))
        outside = 8 * math.pi / (lam * (16 - math.pi))
        assert abs(area * inside + (1 - area) * outside - area) > 0.05 * area  # mean off by 10-20 %
    lam, N = 20.0, 64
    I = synth.disc_image(N).astype(np.float64)
    u = O.rof_solve(I, lam, n_iters=3000)["u"]
    a = 1 - 2 / (lam * r)
    printed_inside = (1 - 8 / lam) + 8 * math.pi / (lam * (16 - math.pi))
    assert abs(u[N // 2, N // 2] - a) < 0.02 < abs(u[N // 2, N // 2] - printed_inside)


@pytest.mark.parametrize("N", [8, 32])
def test_step_rule_straight_edge(N):
    lam = 10.0
    I = np.zeros((N, N))
    I[:, N // 2:] = 1.0
    tau, sigma, s = O.rof_step_rule(I, lam, eps=1e-3)
    assert abs(s["tv"] - 1.0) < 1e-12
    assert abs(s["grad_l2"] - math.sqrt(N)) < 1e-12
    assert abs(s["fid"] - lam / 8) < 1e-12
    expect = min(math.sqrt(lam) * min(1.0, lam / 8) / math.sqrt(1e-3), math.sqrt(N))
    assert abs(tau - expect) < 1e-12 and abs(sigma * tau - 1) < 1e-15
