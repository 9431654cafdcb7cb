"""Pins of the three-dimensional FP64 oracle (CPU only), each against
something other than the oracle itself: adjointness of grad and div, the
cosine eigenvectors of the 7-point Neumann Laplacian (Appendix A), a dense
linear solve, ROF invariants (mean, fixed point, weak duality) and the ball's
two-valued minimiser, EMD feasibility and the one-dimensional identity
W1 = h sum |F0 - F1| for densities that vary along one axis only."""
import math

import numpy as np
import pytest

from oracle import gprox_oracle3d as O3
from paper_1805_09453_gb300 import synth


def test_grad_div_adjoint_and_zero_slots():
    rng = np.random.default_rng(0)
    N, h = 7, 1.0 / 7
    u = rng.normal(size=(N, N, N))
    p = [rng.normal(size=(N, N, N)) for _ in range(3)]
    g = O3.grad3(u, h)
    lhs = sum((gi * pi).sum() for gi, pi in zip(g, p))
    rhs = -(u * O3.div3(*p, h)).sum()
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    assert np.all(g[0][:, :, -1] == 0) and np.all(g[1][:, -1, :] == 0) and np.all(g[2][-1, :, :] == 0)


def test_cosine_eigenvectors():
    N, h = 8, 1.0 / 8
    c = (np.arange(N) + 0.5) / N
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    a, b, k = 3, 1, 5
    u = np.cos(math.pi * a * x) * np.cos(math.pi * b * y) * np.cos(math.pi * k * z)
    mu = lambda q: (4 / h ** 2) * math.sin(math.pi * q / (2 * N)) ** 2
    np.testing.assert_allclose(O3.laplacian3(u, h), -(mu(a) + mu(b) + mu(k)) * u, atol=1e-9)


@pytest.mark.parametrize("alpha", [0.7, 0.0])
def test_helmholtz_against_dense_solve(alpha):
    N, h = 4, 1.0 / 4
    n = N ** 3
    L = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        L[:, i] = O3.laplacian3(e.reshape(N, N, N), h).ravel()
    rng = np.random.default_rng(1)
    b = rng.normal(size=n)
    A = alpha * np.eye(n) - L
    if alpha == 0.0:
        b -= b.mean()
        x, *_ = np.linalg.lstsq(A, b, rcond=None)
        x -= x.mean()
    else:
        x = np.linalg.solve(A, b)
    np.testing.assert_allclose(O3.helmholtz_solve3(b.reshape(N, N, N), alpha, h).ravel(), x, atol=1e-10)


def test_rof_invariants():
    rng = np.random.default_rng(2)
    N, lam = 10, 8.0
    I = rng.uniform(size=(N, N, N))
    means = []
    res = O3.rof_solve3(I, lam, 200, callback=lambda n, u, *p: means.append(u.mean()))
    assert np.allclose(means, I.mean(), atol=1e-13)  # the fidelity keeps the mean
    P, D = res["primal"], res["dual"]
    assert P >= D and (P - D) / abs(P) < 1e-2  # weak duality, gap closing
    J = np.full((N, N, N), 0.3)
    r = O3.rof_solve3(J, lam, 5)
    np.testing.assert_allclose(r["u"], J, atol=1e-14)  # a constant image is the fixed point
    assert all(np.all(pc == 0) for pc in r["p"])


def test_rof_ball_two_valued_minimiser():
    """For the indicator of a ball of radius r, the two-valued function a
    inside, b outside that minimises TV + lambda/2 ||u - I||^2 has
    a = 1 - 3/(lambda r) (perimeter / volume = 3/r) and
    b = 4 pi r^2 / (lambda (1 - 4/3 pi r^3)); it keeps the mean.  On the
    grid the converged plateaus sit near it: the outer one approaches b as the
    grid refines (1.0e-2 off at 12^3, 4.6e-3 at 24^3), the inner one stays
    about 1-1.5 % below a (4.7e-3 at 12^3, 9.5e-3 at 24^3: the isotropic
    forward-difference TV of a staircase sphere exceeds its area, as the
    digitised disc's does in two dimensions)."""
    lam, r = 30.0, 0.3
    a = 1 - 3 / (lam * r)
    b = 4 * math.pi * r * r / (lam * (1 - 4 / 3 * math.pi * r ** 3))
    vol = 4 / 3 * math.pi * r ** 3
    assert a > b and abs(vol * a + (1 - vol) * b - vol) < 1e-12
    errs = []
    for N in (12, 24):
        c = (np.arange(N) + 0.5) / N
        z, y, x = np.meshgrid(c, c, c, indexing="ij")
        I = ((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2 <= r * r).astype(np.float64)
        u = O3.rof_solve3(I, lam, 1500)["u"]
        errs.append((abs(u[N // 2, N // 2, N // 2] - a), abs(u[0, 0, 0] - b)))
    assert errs[0][0] < 0.015 * a and errs[1][0] < 0.015 * a, errs
    assert errs[1][1] < 0.006 and errs[1][1] < 0.5 * errs[0][1], errs


def test_emd_feasible_and_one_dimensional_identity():
    N = 12
    h = 1.0 / N
    xs = (np.arange(N) + 0.5) / N
    f0x = np.exp(-((xs - 0.3) / 0.1) ** 2) + 0.05
    f1x = np.exp(-((xs - 0.7) / 0.15) ** 2) + 0.05
    f0x /= f0x.sum() * h
    f1x /= f1x.sum() * h
    f0 = np.broadcast_to(f0x, (N, N, N)).copy()
    f1 = np.broadcast_to(f1x, (N, N, N)).copy()
    res = []
    st = O3.emd_init3(f0, f1)
    O3.emd_iterate3(st, 1.0, 1.0, 3000,
                    callback=lambda n, mx, my, mz, *p: res.append(
                        np.abs(O3.div3(mx, my, mz, h) - (f0 - f1)).max()) if n % 500 == 0 else None)
    assert max(res) < 1e-10  # every iterate feasible
    F = h * np.cumsum(f0x - f1x)
    W1 = h * np.abs(F).sum()
    P = O3.emd_primal3(*st["m"])
    D = O3.emd_dual3(*st["p"], f0, f1)
    assert D <= P + 1e-12 and abs(P - W1) < 1e-4 * W1 and (P - D) < 1e-3 * P, (P, D, W1)


def test_three_dimensional_inputs():
    N = 16
    I = synth.ball_image3(N)
    assert I.shape == (N, N, N) and abs(I.mean() - 4 / 3 * math.pi / 64) < 0.02  # ball of radius 1/4
    f0, f1 = synth.translated_balls3(N)
    for f in (f0, f1):
        assert abs(f.astype(np.float64).sum() / N ** 3 - 1) < 1e-6
    np.testing.assert_array_equal(np.roll(f0, (N // 4,) * 3, axis=(0, 1, 2)), f1)
    g0, g1 = synth.gaussian_mixture_pair3(N, 0)
    assert g0.min() > 0 and abs(g0.astype(np.float64).sum() / N ** 3 - 1) < 1e-6
    assert not np.array_equal(g0, g1)


def test_translated_balls_near_the_translation_length():
    """A measure and its translate by v are |v| apart (section 4.2's argument
    holds in any dimension): |(1/4, 1/4, 1/4)| = sqrt(3)/4; at 16^3 the grid's
    anisotropy leaves the discrete optimum within 10 %, and the gap certifies
    the value."""
    f0, f1 = synth.translated_balls3(16)
    res = O3.emd_solve3(f0, f1, 1500)
    v = math.sqrt(3) / 4
    assert res["dual"] <= res["primal"] and (res["primal"] - res["dual"]) < 1e-2 * res["primal"]
    assert abs(res["primal"] - v) < 0.1 * v, res["primal"]
