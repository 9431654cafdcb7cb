"""Learned warm start: the network's GPU kernels against the FP64 oracle, the
zero-start fallback, and what a trained network gains.

Tolerances.  FP32 mode: the kernels accumulate in FP32 (unit roundoff 6e-8)
over at most 12C * 9 terms per output and through 15 layers; a relative L2
error of 1e-5 on phi and 1e-4 on the parameter gradient (whose wgrad sums run
over B * N^2 terms with atomics) leaves an order of magnitude of headroom.
The BF16 mode runs the same templated kernels with BF16 storage.  There an
element-wise bar does not exist: a BF16 rounding decision flips under an
FP32-vs-FP64 accumulation difference, and the random network's mean-free
output is a small difference of large terms, so each flip is amplified (in
the oracle alone, a 1e-6 relative perturbation of one input channel moves the
BF16 output by up to 2.5e-3 and the gradient by up to half of its whole BF16
error).  The bar is the BF16 error envelope measured on the oracle: the GPU
result is no farther from the oracle's BF16 emulation than that emulation is
from FP64, and no more than twice as far from FP64.
"""
import numpy as np
import pytest
import torch

from oracle import cnn_oracle as K
from paper_1805_09453_gb300 import synth
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    hh = gprox.Handle(0)
    yield hh
    hh.close()


def _batch(N, seeds):
    f = [synth.gaussian_mixture_pair(N, s) for s in seeds]
    f0 = [torch.from_numpy(a).cuda() for a, _ in f]
    f1 = [torch.from_numpy(b).cuda() for _, b in f]
    x = np.stack([K.features(a, b) for a, b in f])
    return f0, f1, x


def _net(h, C, bf16, seed=1):
    from paper_1805_09453_gb300 import gprox

    net = gprox.Cnn(h, C, bf16=bf16, seed=seed)
    # small random biases so that every ReLU sees both signs
    w = net.get_params()
    rng = np.random.default_rng(seed)
    off = 0
    for ci, co in K.conv_specs(C):
        off += ci * co * 9
        w[off:off + co] = rng.uniform(-0.05, 0.05, co)
        off += co
    net.set_params(w)
    return net


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("N,C,B", [(64, 4, 2), (40, 4, 1), (8, 2, 3), (128, 8, 1)])
def test_cnn_forward_matches_oracle(h, bf16, N, C, B):
    net = _net(h, C, bf16)
    assert net.num_params == K.num_params(C)
    f0, f1, x = _batch(N, range(B))
    phi = net.forward(f0, f1).cpu().numpy()
    w = net.get_params().astype(np.float64)
    ref, _ = K.forward(w, x, C, bf16=bf16)
    assert np.abs(phi.mean(axis=(1, 2))).max() < 1e-6 * np.abs(ref).max()
    if not bf16:
        assert rel_l2(phi, ref) < 1e-5, rel_l2(phi, ref)
        return
    exact, _ = K.forward(w, x, C)
    env = rel_l2(ref, exact)
    assert rel_l2(phi, ref) <= env and rel_l2(phi, exact) <= 2 * env, (rel_l2(phi, ref), rel_l2(phi, exact), env)


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("N,C,B", [(64, 4, 2), (40, 4, 2), (128, 8, 1)])
def test_cnn_loss_grad_matches_oracle(h, bf16, N, C, B):
    net = _net(h, C, bf16, seed=3)
    f0, f1, x = _batch(N, range(10, 10 + B))
    rng = np.random.default_rng(N)
    t = np.stack([K.features(*synth.gaussian_mixture_pair(N, 50 + b))[2] * 0.05 + 0.01 * rng.normal(size=(N, N))
                  for b in range(B)])
    tt = [torch.from_numpy(t[b].astype(np.float32)).cuda() for b in range(B)]
    L, g = net.loss_grad(f0, f1, tt, want_grad=True)
    w = net.get_params().astype(np.float64)
    t64 = t.astype(np.float32).astype(np.float64)
    Lr, gr, _ = K.loss_and_grad(w, x, t64, C, bf16=bf16)
    if not bf16:
        assert abs(L - Lr) < 1e-6 * abs(Lr)
        assert rel_l2(g, gr) < 1e-4, rel_l2(g, gr)
        # every convolution's slice, not just the whole vector
        off = 0
        for ci, co in K.conv_specs(C):
            n = ci * co * 9 + co
            assert rel_l2(g[off:off + n], gr[off:off + n]) < 1e-4
            off += n
        return
    Le, ge, _ = K.loss_and_grad(w, x, t64, C)
    assert abs(L - Lr) <= 2 * abs(Lr - Le) + 1e-4 * abs(Le), (L, Lr, Le)
    env = rel_l2(gr, ge)
    assert rel_l2(g, gr) <= env and rel_l2(g, ge) <= 2 * env, (rel_l2(g, gr), rel_l2(g, ge), env)


def test_cnn_adam_matches_oracle(h):
    net = _net(h, 4, True, seed=5)
    f0, f1, _ = _batch(32, [0, 1])
    tt = [torch.randn(32, 32, device="cuda") for _ in range(2)]
    w = net.get_params().astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for k in range(1, 4):
        _, g = net.loss_grad(f0, f1, tt, want_grad=True, want_loss=False)
        net.adam_step(1e-3)
        w, m, v = K.adam_step(w, m, v, g.astype(np.float64), k, 1e-3)
        got = net.get_params()
        assert np.max(np.abs(got - w)) < 1e-6 * max(1.0, np.max(np.abs(w)))
        w = got.astype(np.float64)  # follow the GPU's FP32 weights


def test_cnn_errors(h):
    from paper_1805_09453_gb300 import gprox

    net = gprox.Cnn(h, 2)
    f = torch.zeros(12, 12, device="cuda")
    phi = torch.zeros(1, 12, 12, device="cuda")
    assert gprox.lib().gp_cnn_forward(net._n, 1, gprox._ptr_array([f]), gprox._ptr_array([f]), 12, gprox._ptr(phi),
                                      None) == gprox.GP_ERR_ARG
    assert "multiple of 8" in net.last_error()
    fh = torch.zeros(16, 16)
    assert gprox.lib().gp_cnn_forward(net._n, 1, gprox._ptr_array([fh]), gprox._ptr_array([fh]), 16,
                                      gprox._ptr(phi), None) == gprox.GP_ERR_ARG
    with pytest.raises(ValueError):
        net.set_params(np.zeros(3, np.float32))
    assert gprox.lib().gp_cnn_adam_step(net._n, -1.0, None) == gprox.GP_ERR_ARG


def test_learned_start_matches_warm_dual_and_zero_net_falls_back(h):
    """A network whose output is zero gives p_0 = 0: the gap probe keeps the
    zero start and the result equals emd_solve from zero bit for bit.  And a
    random network's start p_0 equals proj(grad phi_0) of its own output."""
    from paper_1805_09453_gb300 import gprox

    N = 64
    net = gprox.Cnn(h, 4, seed=2)
    f0, f1, _ = _batch(N, [7])
    o = gprox.default_opts(max_iters=200, tol_rel_gap=0.0, gap_every=20)
    phi0 = net.forward(f0, f1)[0].cpu().numpy().astype(np.float64)
    p = torch.zeros((2, N, N), device="cuda")
    m = torch.zeros((2, N, N), device="cuda")
    o0 = gprox.default_opts(max_iters=0, tol_rel_gap=0.0)
    st, rep = gprox.emd_solve_learned(h, net, f0[0], f1[0], m, p, None, o0)
    net.check(st)
    if rep["used_warm"]:
        px, py = K.warm_dual(phi0)
        assert rel_l2(p.cpu().numpy(), np.stack([px, py])) < 1e-5
    net.set_params(np.zeros(net.num_params, np.float32))
    m1 = torch.zeros((2, N, N), device="cuda")
    st, rep = gprox.emd_solve_learned(h, net, f0[0], f1[0], m1, None, None, o)
    net.check(st)
    assert not rep["used_warm"]
    m2 = torch.zeros((2, N, N), device="cuda")
    st, rep2 = gprox.emd_solve(h, f0[0], f1[0], m2, None, None, o)
    h.check(st)
    assert torch.equal(m1, m2)
    assert rep["primal"] == rep2["primal"] and rep["iters"] == rep2["iters"] == 200


def test_trained_network_cuts_iterations(h):
    """Train a small network (C = 8) on 96 solved 64^2 pairs with the library's
    own kernels, then solve 12 held-out pairs to a relative gap of 1e-5 from
    the zero start and from the learned start."""
    from paper_1805_09453_gb300 import gprox, learn

    N = 64
    # targets: dual potentials solved to a gap of 2e-6 (or 20000 iterations; a
    # start needs no more than ~1e-4)
    f0, f1, phi, iters, gaps = learn.generate(h, N, range(96), tol=2e-6, max_iters=20000)
    assert max(gaps) < 1e-4
    g0, g1, gphi, _, _ = learn.generate(h, N, range(learn.TEST_SEED0, learn.TEST_SEED0 + 12), tol=2e-6,
                                        max_iters=20000)
    net = gprox.Cnn(h, 8, seed=0)
    L0 = learn.test_loss(net, g0, g1, gphi)
    hist = learn.train(net, f0, f1, phi, steps=600, batch=16, lr=2e-3)
    L1 = learn.test_loss(net, g0, g1, gphi)
    assert L1 < 0.5 * L0, (L0, L1, hist[-3:])
    s = learn.summarize(learn.evaluate(h, net, g0, g1, tol=1e-5))
    print(s)
    assert s["median_warm_iters"] < 0.8 * s["median_zero_iters"], s
