"""Pins of the oracle's discrete operators against textbook objects.

* grad / div adjointness, the defining property of div = -grad^T (reading R2);
* -Laplacian equals the combinatorial Laplacian of the N x N grid graph / h^2
  (built by networkx, independent of the oracle's stencils);
* the Neumann Helmholtz solve equals a dense linear solve with that matrix;
* cosine vectors cos(pi k (j + 1/2) / N) are eigenvectors of the 1-D Neumann
  second difference with mu_k = (4/h^2) sin^2(pi k / 2N) (Appendix A's even
  reflection), checked without scipy.fft;
* the unit-ball projection (sections 3.1 and 3.2) on hand-computed cases.
"""
import math

import networkx as nx
import numpy as np
import pytest

from oracle import gprox_oracle as O


def _grid_laplacian(N):
    G = nx.grid_2d_graph(N, N)  # nodes (i, j)
    nodes = [(i, j) for i in range(N) for j in range(N)]
    L = nx.laplacian_matrix(G, nodelist=nodes).toarray().astype(np.float64)
    return L


@pytest.mark.parametrize("N", [1, 2, 5, 8, 13])
def test_grad_div_adjoint(N):
    rng = np.random.default_rng(N)
    h = 1.0 / N
    u = rng.normal(size=(N, N))
    px, py = rng.normal(size=(N, N)), rng.normal(size=(N, N))  # slots deliberately non-zero
    gx, gy = O.grad(u, h)
    lhs = h * h * np.sum(gx * px + gy * py)
    rhs = -h * h * np.sum(u * O.div(px, py, h))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    # zero-flux slots of the gradient
    assert np.all(gx[:, -1] == 0) and np.all(gy[-1, :] == 0)


@pytest.mark.parametrize("N", [2, 3, 6, 9])
def test_laplacian_is_grid_graph_laplacian(N):
    h = 1.0 / N
    L = _grid_laplacian(N)
    M = np.zeros((N * N, N * N))
    for k in range(N * N):
        e = np.zeros(N * N)
        e[k] = 1.0
        M[:, k] = -O.laplacian(e.reshape(N, N), h).ravel()
    np.testing.assert_allclose(M, L / (h * h), rtol=0, atol=1e-9)


@pytest.mark.parametrize("N,alpha", [(4, 3.0), (7, 0.5), (12, 100.0), (16, 1e-3), (9, 0.0), (16, 0.0)])
def test_helmholtz_solve_matches_dense(N, alpha):
    h = 1.0 / N
    rng = np.random.default_rng(100 + N)
    b = rng.normal(size=(N, N))
    A = alpha * np.eye(N * N) + _grid_laplacian(N) / (h * h)
    if alpha == 0.0:
        bc = b - b.mean()  # the solve drops the constant mode of b
        x_ref = np.linalg.lstsq(A, bc.ravel(), rcond=None)[0]
        x_ref -= x_ref.mean()
    else:
        x_ref = np.linalg.solve(A, b.ravel())
    x = O.helmholtz_solve(b, alpha, h)
    np.testing.assert_allclose(x.ravel(), x_ref, rtol=0, atol=1e-10 * max(1.0, np.abs(x_ref).max()))
    if alpha == 0.0:
        assert abs(x.mean()) < 1e-12


@pytest.mark.parametrize("N", [5, 8, 16])
def test_cosine_eigenvectors(N):
    h = 1.0 / N
    mu = O.eigenvalues(N, h)
    j = np.arange(N)
    for k in range(N):
        v = np.cos(math.pi * k * (j + 0.5) / N)
        # 1-D Neumann second difference
        lap = np.zeros(N)
        lap[:-1] += v[1:] - v[:-1]
        lap[1:] -= v[1:] - v[:-1]
        lap /= h * h
        np.testing.assert_allclose(-lap, mu[k] * v, atol=1e-8 * (1 + mu[k]))
        # and the 2-D Laplacian on an outer product
        V = np.outer(v, np.cos(math.pi * 1 * (j + 0.5) / N))
        np.testing.assert_allclose(-O.laplacian(V, h), (mu[k] + mu[1]) * V, atol=1e-8 * (1 + mu[k] + mu[1]))


def test_projection_cases():
    qx = np.array([3.0, 0.3, 1.0, -0.6, 0.0])
    qy = np.array([4.0, 0.4, 0.0, 0.8, -2.0])
    px, py = O.project(qx, qy)
    np.testing.assert_allclose(px, [0.6, 0.3, 1.0, -0.6, 0.0])
    np.testing.assert_allclose(py, [0.8, 0.4, 0.0, 0.8, -1.0])
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=1000) * 3, rng.normal(size=1000) * 3
    px, py = O.project(a, b)
    assert np.all(np.hypot(px, py) <= 1 + 1e-15)
    inside = np.hypot(a, b) <= 1
    assert np.all(px[inside] == a[inside]) and np.all(py[inside] == b[inside])
    # l1 variant: componentwise clip
    cx, cy = O.project(np.array([2.0, -0.5]), np.array([-3.0, 0.25]), norm="l1")
    np.testing.assert_array_equal(cx, [1.0, -0.5])
    np.testing.assert_array_equal(cy, [-1.0, 0.25])
