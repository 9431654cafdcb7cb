"""Pins of the oracle's CP2 iteration (the accelerated primal-dual method the
paper compares G-prox PDHG with in section 4.1, Tables 4-5) against facts that
do not come from the oracle itself:

* the initial steps tau0 = sigma0 = 1 / sqrt(||Lap||) (section 4.1) against
  the largest eigenvalue of the 5-point Neumann matrix, assembled here from
  the stencil and diagonalised by numpy;
* the step-size recursion: tau_n sigma_n stays tau0 sigma0, and
  1/tau_{n+1}^2 = 1/tau_n^2 + 2 gamma / tau_n, whence gamma n tau_n -> 1;
* a constant image is a fixed point with p = 0;
* the limit is the ROF minimiser: the optimum of the (independently pinned)
  G-prox iteration, by value and by iterate (u* is unique: the energy is
  lambda-strongly convex), with a duality gap falling towards zero;
* the 8 x 8 dual optimum from SLSQP (as for the G-prox oracle).
"""
import numpy as np
from scipy.optimize import minimize

from oracle import gprox_oracle as O
from paper_1805_09453_gb300 import synth


def _neumann_matrix(N):
    """-Lap on an N x N cell grid (h = 1/N), 5-point stencil, zero-flux sides."""
    h2 = 1.0 / (N * N)
    M = np.zeros((N * N, N * N))
    for i in range(N):
        for j in range(N):
            r = i * N + j
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < N and 0 <= jj < N:
                    M[r, r] += 1.0 / h2
                    M[r, ii * N + jj] -= 1.0 / h2
    return M


def test_initial_steps_match_the_laplacian_norm():
    for N in (4, 8, 12):
        lmax = np.linalg.eigvalsh(_neumann_matrix(N)).max()
        t0, s0 = O.rof_cp2_steps(N)
        assert abs(t0 * s0 * lmax - 1.0) < 1e-12 and t0 == s0


def test_step_recursion_and_its_asymptote():
    N, lam = 8, 12.0
    I = np.zeros((N, N))
    st = O.rof_cp2_init(I)
    t0, s0 = st["tau"], st["sigma"]
    taus = [st["tau"]]
    for _ in range(4000):
        O.rof_cp2_iterate(st, I, lam, 1)
        taus.append(st["tau"])
        assert abs(st["tau"] * st["sigma"] - t0 * s0) <= 1e-12 * t0 * s0
    t = np.array(taus)
    np.testing.assert_allclose(1.0 / t[1:] ** 2, 1.0 / t[:-1] ** 2 + 2.0 * lam / t[:-1], rtol=1e-10)
    n = len(t) - 1
    assert abs(lam * n * t[-1] - 1.0) < 0.02  # the decay rate of tau behind the O(1/n^2) gap


def test_constant_image_fixed_point():
    I = np.full((16, 16), 0.37)
    st = O.rof_cp2_init(I, u0=I)
    O.rof_cp2_iterate(st, I, 8.0, 25)
    np.testing.assert_allclose(st["u"], I, atol=1e-13)
    assert np.abs(st["px"]).max() < 1e-12 and np.abs(st["py"]).max() < 1e-12


def test_limit_is_the_rof_minimiser():
    N, lam = 16, 8.0
    I = synth.rof_image(N, 2).astype(np.float64)
    ref = O.rof_solve(I, lam, tol=1e-12, max_iters=100000)
    st = O.rof_cp2_init(I)
    gaps = []
    for _ in range(60):
        O.rof_cp2_iterate(st, I, lam, 250)
        P, D, g = O.rof_gap(st["u"], st["px"], st["py"], I, lam)
        assert P - D >= -1e-12
        gaps.append(P - D)
    assert gaps[-1] < 1e-3 * gaps[0]
    assert abs(P - ref["primal"]) <= 1e-7 * abs(ref["primal"])
    # lambda-strong convexity: lam/2 ||u - u*||^2 <= P(u) - P(u*)
    h2 = 1.0 / (N * N)
    assert 0.5 * lam * h2 * np.sum((st["u"] - ref["u"]) ** 2) <= P - ref["primal"] + 1e-12


def test_brute_force_8x8_dual():
    """max D(p) s.t. |p| <= 1 by SLSQP on the 8 x 8 dual, against CP2's limit."""
    N, lam = 8, 6.0
    rng = np.random.default_rng(11)
    I = rng.uniform(0, 1, (N, N))
    h = 1.0 / N
    nx = N * (N - 1)  # free components: px[:, :-1], py[:-1, :]

    def unpack(z):
        px = np.zeros((N, N))
        py = np.zeros((N, N))
        px[:, :-1] = z[:nx].reshape(N, N - 1)
        py[:-1, :] = z[nx:].reshape(N - 1, N)
        return px, py

    def negD(z):
        px, py = unpack(z)
        d = (np.pad(px[:, :-1], ((0, 0), (0, 1))) - np.pad(px[:, :-1], ((0, 0), (1, 0)))
             + np.pad(py[:-1, :], ((0, 1), (0, 0))) - np.pad(py[:-1, :], ((1, 0), (0, 0)))) / h
        return h * h * np.sum(I * d) + h * h * np.sum(d * d) / (2.0 * lam)

    def cons(z):
        px, py = unpack(z)
        return 1.0 - (px * px + py * py).ravel()

    res = minimize(negD, np.zeros(2 * nx), method="SLSQP", constraints=[{"type": "ineq", "fun": cons}],
                   options={"maxiter": 2000, "ftol": 1e-14})
    assert res.success
    st = O.rof_cp2_solve(I, lam, n_iters=40000)
    assert abs(st["primal"] - (-res.fun)) <= 1e-7 * abs(res.fun)
