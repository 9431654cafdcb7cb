"""Pins of the warm-start network's FP64 oracle (CPU only).

Each piece is checked against something other than itself: scipy's 2-D
correlation, reshaping / Kronecker forms of pooling and upsampling, adjoint
identities, central finite differences of the whole network's loss, Adam's
closed form under a constant gradient, torch's bfloat16 rounding, scipy's
cell-centred zoom for the coarse-start interpolation, and -- for the premise
of the warm start (section 4.2: the dual iterate converges to the gradient of
the Kantorovich potential) -- the iteration count of the EMD oracle started
from the converged dual potential and from the coarse-grid potential.
"""
import numpy as np
import pytest
import scipy.ndimage
import scipy.signal

from oracle import cnn_oracle as K
from oracle import gprox_oracle as O
from paper_1805_09453_gb300 import synth


def _rand_params(C, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    w = []
    for ci, co in K.conv_specs(C):
        w.append(rng.uniform(-1, 1, ci * co * 9) * scale * np.sqrt(6.0 / (9 * ci)))
        w.append(rng.uniform(-0.1, 0.1, co))
    return np.concatenate(w)


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 9, 7))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = K.conv3x3(x, W, b)
    for bb in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.signal.correlate2d(x[bb, c], W[o, c], mode="same", boundary="fill")
                             for c in range(3))
            np.testing.assert_allclose(y[bb, o], ref, rtol=1e-12, atol=1e-12)


def test_pool_and_upsample_closed_forms():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 8, 6))
    np.testing.assert_allclose(K.pool2(x), x.reshape(2, 3, 4, 2, 3, 2).mean(axis=(3, 5)), rtol=1e-14)
    z = rng.normal(size=(2, 3, 4, 3))
    np.testing.assert_array_equal(K.up2(z), np.kron(z, np.ones((1, 1, 2, 2))))


def test_linear_pieces_are_adjoint():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 3, 8, 8))
    W = rng.normal(size=(5, 3, 3, 3))
    dy = rng.normal(size=(2, 5, 8, 8))
    lhs = np.sum(K.conv3x3(x, W, None) * dy)
    assert abs(lhs - np.sum(x * K.conv3x3_adjoint(dy, W, x.shape))) < 1e-10 * abs(lhs)
    # weight gradient: <conv(x; W2, b2), dy> = <W2, dW> + <b2, db> (linear in W, b)
    W2 = rng.normal(size=W.shape)
    b2 = rng.normal(size=5)
    dW, db = K.conv3x3_wgrad(dy, x)
    lhs = np.sum(K.conv3x3(x, W2, b2) * dy)
    assert abs(lhs - (np.sum(W2 * dW) + np.sum(b2 * db))) < 1e-10 * abs(lhs)
    z = rng.normal(size=(2, 3, 4, 4))
    assert abs(np.sum(K.pool2(x) * z) - np.sum(x * K.pool2_adjoint(z))) < 1e-12
    assert abs(np.sum(K.up2(z) * x) - np.sum(z * K.up2_adjoint(x))) < 1e-12


def test_loss_gradient_wrt_phi_by_finite_differences():
    rng = np.random.default_rng(3)
    phi = rng.normal(size=(2, 8, 8))
    phi -= phi.mean(axis=(1, 2), keepdims=True)
    t = rng.normal(size=(2, 8, 8)) + 3.0
    g = K.loss_grad_phi(phi, t)
    eps = 1e-6
    for _ in range(20):
        b, i, j = rng.integers(2), rng.integers(8), rng.integers(8)
        d = np.zeros_like(phi)
        d[b, i, j] = eps
        d[b] -= d[b].mean()  # stay mean-free: the gradient is taken on mean-free fields
        fd = (K.loss(phi + d, t) - K.loss(phi - d, t)) / (2 * eps)
        assert abs(fd - np.sum(g * d) / eps) < 1e-7


@pytest.mark.parametrize("bf16", [False, True])
def test_network_gradient_by_finite_differences(bf16):
    """Whole-network parameter gradient vs central differences of the loss.
    In the BF16 emulation the rounding makes the loss piecewise constant, so
    the finite differences are taken through the FP64 network and only the
    forward pass is compared for the emulation (it must stay within the BF16
    error of the FP64 output)."""
    C, N, B = 2, 8, 2
    rng = np.random.default_rng(4)
    w = _rand_params(C, 5, scale=1.5)
    f = [synth.gaussian_mixture_pair(N, s) for s in range(B)]
    x = np.stack([K.features(a, b, 0.1 * rng.normal(size=(N, N))) for a, b in f])
    t = rng.normal(size=(B, N, N))
    if bf16:
        phi64, _ = K.forward(w, x, C, bf16=False)
        phi16, _ = K.forward(w, x, C, bf16=True)
        rel = np.linalg.norm(phi16 - phi64) / np.linalg.norm(phi64)
        assert 1e-5 < rel < 5e-2, rel  # rounding happened, and it is BF16-sized
        return
    L, g, _ = K.loss_and_grad(w, x, t, C)
    assert np.isfinite(L) and g.shape == w.shape
    eps = 1e-6
    idx = rng.choice(w.size, 60, replace=False)
    off = 0
    for ci, co in K.conv_specs(C):  # every conv's bias and one weight included
        idx = np.append(idx, [off + rng.integers(ci * co * 9), off + ci * co * 9 + rng.integers(co)])
        off += ci * co * 9 + co
    gmax = np.max(np.abs(g))
    for k in idx:
        d = np.zeros_like(w)
        d[k] = eps
        fd = (K.loss(K.forward(w + d, x, C)[0], t) - K.loss(K.forward(w - d, x, C)[0], t)) / (2 * eps)
        assert abs(fd - g[k]) < 1e-6 * max(gmax, 1.0), (k, fd, g[k])


def test_adam_constant_gradient_closed_form():
    """With a constant gradient the bias-corrected moments equal g and g^2 at
    every step, so w_k = w_0 - k lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    w0 = rng.normal(size=50)
    g = rng.normal(size=50)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for k in range(1, 8):
        w, m, v = K.adam_step(w, m, v, g, k, 1e-2)
        np.testing.assert_allclose(w, w0 - k * 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-12)


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-30, 30, 4000), [0.0, -0.0, 1.0, 3.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(K.round_bf16(x), ref)


def test_features_prior_and_warm_dual():
    N = 16
    f0, f1 = synth.gaussian_mixture_pair(N, 3)
    prior = np.linspace(0, 1, N)[None, :] * np.ones((N, 1))
    x = K.features(f0, f1, prior)
    np.testing.assert_allclose(x[0], (f0 - f1) / 16)
    np.testing.assert_allclose(x[1], (f0 + f1) / 16)
    np.testing.assert_array_equal(x[2], prior)
    # a network whose head is zero returns its prior (mean removed)
    w = _rand_params(2, 1)
    off = sum(ci * co * 9 + co for ci, co in K.conv_specs(2)[:-1])
    w[off:] = 0.0
    phi, _ = K.forward(w, x[None], 2)
    np.testing.assert_allclose(phi[0], prior - prior.mean(), atol=1e-15)
    px, py = K.warm_dual(0.5 * prior)
    assert np.max(np.hypot(px, py)) <= 1 + 1e-12


def test_upsample_matches_scipy_zoom_and_restrict_keeps_mass():
    rng = np.random.default_rng(8)
    c = rng.normal(size=(8, 8))
    for k in (2, 4, 8):
        ref = scipy.ndimage.zoom(c, k, order=1, grid_mode=True, mode="nearest")
        np.testing.assert_allclose(K.upsample_bilinear(c, k), ref, atol=1e-14)
    f = rng.random((32, 32))
    for k in (2, 4):
        r = K.restrict_mean(f, k)
        assert r.shape == (32 // k, 32 // k)
        assert abs(r.sum() * k * k - f.sum()) < 1e-12 * f.sum()  # same mass with h_c = k h
        np.testing.assert_allclose(K.upsample_bilinear(np.full((4, 4), 2.5), k), 2.5)


def test_dual_potential_start_cuts_iterations():
    """Premise of the warm start: the EMD oracle started from
    p_0 = proj(grad phi*), phi* the converged dual potential, reaches a
    relative gap of 1e-5 in far fewer iterations than from p_0 = 0 (here
    ~500 against ~5000)."""
    N = 16
    f0, f1 = synth.gaussian_mixture_pair(N, 3)
    st = O.emd_solve(f0, f1, tol=1e-8, gap_every=10, max_iters=40000)
    _, phi, s = O.emd_dual(st["px"], st["py"], f0, f1)
    p0 = K.warm_dual(phi / max(1.0, s))

    def iters(p):
        s2 = O.emd_init(f0, f1, p0=p, pbar0=p)
        for n in range(10, 20001, 10):
            O.emd_iterate(s2, 1.0, 1.0, 10)
            if O.emd_gap(s2, f0, f1)[2] <= 1e-5:
                return n
        return 20000

    zero, warm = iters(None), iters(p0)
    assert warm < 0.5 * zero, (warm, zero)


def test_coarse_start_cuts_iterations():
    """The coarse-grid potential (2x coarser, 4000 oracle iterations there)
    as the start: fewer fine iterations to a relative gap of 1e-5 than the
    zero start (here about a third)."""
    N = 32
    f0, f1 = synth.gaussian_mixture_pair(N, 3)
    px, py = K.warm_dual(K.coarse_start(f0, f1, 2, 4000))

    def iters(p):
        s2 = O.emd_init(f0, f1, p0=p, pbar0=p)
        for n in range(10, 20001, 10):
            O.emd_iterate(s2, 1.0, 1.0, 10)
            if O.emd_gap(s2, f0, f1)[2] <= 1e-5:
                return n
        return 20000

    zero, warm = iters(None), iters((px, py))
    assert warm < 0.6 * zero, (warm, zero)
