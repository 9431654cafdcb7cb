"""Learned warm start: the network's GPU kernels against the FP64 oracle, the
zero-start fallback, and what a trained network gains.

Tolerances.  FP32 mode: the kernels accumulate in FP32 (unit roundoff 6e-8)
over at most 12C * 9 terms per output and through 15 layers; a relative L2
error of 1e-5 on phi and 1e-4 on the parameter gradient (whose wgrad sums run
over B * N^2 terms with atomics) leaves an order of magnitude of headroom.
The BF16 mode stores weights and activations in BF16 and runs every
convolution product (forward, weight and data gradients) as a tcgen05
implicit GEMM (FP32 accumulation in tensor memory; the FP32 gradient dY
enters as a hi + lo BF16 pair).  There an
element-wise bar does not exist: a BF16 rounding decision flips under an
FP32-vs-FP64 accumulation difference, and the random network's mean-free
output is a small difference of large terms, so each flip is amplified (in
the oracle alone, a 1e-6 relative perturbation of one input channel moves the
BF16 output by up to 2.5e-3 and the gradient by up to half of its whole BF16
error).  The bar is the BF16 error envelope measured on the oracle: the GPU
result is no farther from the oracle's BF16 emulation than that emulation is
from FP64, and no more than twice as far from FP64.  The sizes include
C = 32, the workloads' width (up to 256 output channels, K = 9 Cin up to
3 456, full 256-column tensor-core tiles), at 64^2 (vector gathers at every
level) and 32^2 (the coarsest level, 4 x 4, takes the scalar gather).
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


def _batch(N, seeds, with_prior=True):
    """Device pairs, smooth random priors (or None) and the oracle's input stack."""
    f = [synth.gaussian_mixture_pair(N, s) for s in seeds]
    f0 = [torch.from_numpy(a).cuda() for a, _ in f]
    f1 = [torch.from_numpy(b).cuda() for _, b in f]
    pri = None
    if with_prior:
        xs = (np.arange(N) + 0.5) / N
        pri = [(0.3 * np.sin(2.0 + s + 3 * xs)[None, :] * np.cos(1.0 + 2 * xs - s)[:, None]).astype(np.float32)
               for s in seeds]
    x = np.stack([K.features(a, b, None if pri is None else pri[i]) for i, (a, b) in enumerate(f)])
    return f0, f1, (None if pri is None else [torch.from_numpy(q).cuda() for q in pri]), x


def _net(h, C, bf16, seed=1):
    from paper_1805_09453_gb300 import gprox

    net = gprox.Cnn(h, C, bf16=bf16, seed=seed)
    # small random biases so that every ReLU sees both signs, and a non-zero head
    w = net.get_params()
    rng = np.random.default_rng(seed)
    off = 0
    for ci, co in K.conv_specs(C):
        if co == 1:
            w[off:off + ci * 9] = rng.uniform(-1, 1, ci * 9) * np.sqrt(6.0 / (9 * ci))
        off += ci * co * 9
        w[off:off + co] = rng.uniform(-0.05, 0.05, co)
        off += co
    net.set_params(w)
    return net


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("N,C,B", [(64, 4, 2), (40, 4, 1), (8, 2, 3), (128, 8, 1), (64, 32, 1)])
def test_cnn_forward_matches_oracle(h, bf16, N, C, B):
    net = _net(h, C, bf16)
    assert net.num_params == K.num_params(C)
    f0, f1, pri, x = _batch(N, range(B), with_prior=(N != 8))
    phi = net.forward(f0, f1, pri).cpu().numpy()
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
@pytest.mark.parametrize("N,C,B", [(64, 4, 2), (40, 4, 2), (128, 8, 1), (32, 32, 2)])
def test_cnn_loss_grad_matches_oracle(h, bf16, N, C, B):
    net = _net(h, C, bf16, seed=3)
    f0, f1, pri, x = _batch(N, range(10, 10 + B))
    rng = np.random.default_rng(N)
    t = np.stack([x[b, 2] + 0.02 * rng.normal(size=(N, N)) for b in range(B)])
    tt = [torch.from_numpy(t[b].astype(np.float32)).cuda() for b in range(B)]
    L, g = net.loss_grad(f0, f1, tt, pri, want_grad=True)
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
    f0, f1, pri, _ = _batch(32, [0, 1])
    tt = [torch.randn(32, 32, device="cuda") for _ in range(2)]
    w = net.get_params().astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for k in range(1, 4):
        _, g = net.loss_grad(f0, f1, tt, pri, want_grad=True, want_loss=False)
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
    assert gprox.lib().gp_cnn_forward(net._n, 1, gprox._ptr_array([f]), gprox._ptr_array([f]), None, 12,
                                      gprox._ptr(phi), None) == gprox.GP_ERR_ARG
    assert "multiple of 8" in net.last_error()
    fh = torch.zeros(16, 16)
    assert gprox.lib().gp_cnn_forward(net._n, 1, gprox._ptr_array([fh]), gprox._ptr_array([fh]), None, 16,
                                      gprox._ptr(phi), None) == gprox.GP_ERR_ARG
    fd = torch.zeros(16, 16, device="cuda")
    assert gprox.lib().gp_cnn_forward(net._n, 1, gprox._ptr_array([fd]), gprox._ptr_array([fd]),
                                      gprox._ptr_array([fh]), 16, gprox._ptr(phi), None) == gprox.GP_ERR_ARG
    assert "prior" in net.last_error()
    st, _, _ = gprox.emd_coarse_start(h, fd, fd, 3)
    assert st == gprox.GP_ERR_ARG
    with pytest.raises(ValueError):
        net.set_params(np.zeros(3, np.float32))
    assert gprox.lib().gp_cnn_adam_step(net._n, -1.0, None) == gprox.GP_ERR_ARG


@pytest.mark.parametrize("N,k", [(64, 2), (64, 4), (96, 4)])
def test_coarse_start_matches_oracle(h, N, k):
    """Restriction, the coarse EMD iteration (300 iterations) and the
    interpolation against the oracle's coarse_start; potentials compared
    mean-free at the EMD potential bar of 1e-3."""
    from paper_1805_09453_gb300 import gprox

    f0, f1 = synth.gaussian_mixture_pair(N, 21)
    st, phi, rep = gprox.emd_coarse_start(h, torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), k,
                                          gprox.default_opts(max_iters=300, tol_rel_gap=0.0, gap_every=300))
    h.check(st)
    assert rep["iters"] == 300
    ref = K.coarse_start(f0, f1, k, 300)
    got = phi.cpu().numpy()
    assert rel_l2(got - got.mean(), ref - ref.mean()) < 1e-3


def test_learned_start_matches_warm_dual_and_zero_net_falls_back(h):
    """A network whose output is zero gives p_0 = 0: the gap probe keeps the
    zero start and the result equals emd_solve from zero bit for bit.  A new
    network (zero head) returns its prior, the coarse start."""
    from paper_1805_09453_gb300 import gprox

    N = 64
    net = gprox.Cnn(h, 4, seed=2)
    f0, f1, _, _ = _batch(N, [7], with_prior=False)
    o = gprox.default_opts(max_iters=200, tol_rel_gap=0.0, gap_every=20)
    p = torch.zeros((2, N, N), device="cuda")
    m = torch.zeros((2, N, N), device="cuda")
    oc = gprox.default_opts(max_iters=400, tol_rel_gap=0.0, gap_every=400)
    st, prior, _ = gprox.emd_coarse_start(h, f0[0], f1[0], 4, oc)
    h.check(st)
    phi0 = net.forward(f0, f1, [prior])[0].cpu().numpy().astype(np.float64)
    pr = prior.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(phi0, pr - pr.mean(), atol=1e-6)
    o0 = gprox.default_opts(max_iters=0, tol_rel_gap=0.0)
    st, rep = gprox.emd_solve_learned(h, net, f0[0], f1[0], m, p, None, o0, coarse_factor=4, coarse_opts=oc)
    net.check(st)
    assert rep["start"] in ("learned", "prior")  # identical potentials; the first one wins the tie
    px, py = K.warm_dual(phi0)
    assert rel_l2(p.cpu().numpy(), np.stack([px, py])) < 1e-5
    net.set_params(np.zeros(net.num_params, np.float32))
    m1 = torch.zeros((2, N, N), device="cuda")
    st, rep = gprox.emd_solve_learned(h, net, f0[0], f1[0], m1, None, None, o, coarse_factor=0)
    net.check(st)
    assert rep["start"] == "zero"
    m2 = torch.zeros((2, N, N), device="cuda")
    st, rep2 = gprox.emd_solve(h, f0[0], f1[0], m2, None, None, o)
    h.check(st)
    assert torch.equal(m1, m2)
    assert rep["primal"] == rep2["primal"] and rep["iters"] == rep2["iters"] == 200


def test_trained_network_cuts_iterations(h):
    """Train a small network (C = 8) on 96 solved 64^2 pairs with the library's
    own kernels, its prior the 4x coarser solve, then solve 12 held-out pairs
    to a relative gap of 1e-5 from the zero start and from the learned start.
    The trained network must fit the held-out potentials better than its
    prior does (the untrained network) and the learned start must save
    iterations over the zero start."""
    from paper_1805_09453_gb300 import gprox, learn

    N, k = 64, 4
    # targets: dual potentials solved to a gap of 2e-6 (or 20000 iterations; a
    # start needs no more than ~1e-4)
    f0, f1, phi, pri, iters, gaps = learn.generate(h, N, range(96), tol=2e-6, max_iters=20000, coarse_factor=k)
    assert max(gaps) < 1e-4
    g0, g1, gphi, gpri, _, _ = learn.generate(h, N, range(learn.TEST_SEED0, learn.TEST_SEED0 + 12), tol=2e-6,
                                              max_iters=20000, coarse_factor=k)
    net = gprox.Cnn(h, 8, seed=0)
    L0 = learn.test_loss(net, g0, g1, gphi, gpri)
    hist = learn.train(net, f0, f1, phi, pri, steps=600, batch=16, lr=1e-3)
    L1 = learn.test_loss(net, g0, g1, gphi, gpri)
    print("held-out loss: prior", L0, "trained", L1)
    assert L1 < L0, (L0, L1, hist[-3:])
    rows = learn.evaluate(h, net, g0, g1, tol=1e-5, coarse_factor=k)
    s = learn.summarize(rows)
    print(s)
    assert all(r["warm_status"] in ("GP_OK",) for r in rows), rows
    assert s["median_warm_iters"] < 0.8 * s["median_zero_iters"], s
    # what the network adds over its prior (the coarse-grid start alone, the
    # same network with its head zeroed): the learned start is chosen for some
    # pairs and saves iterations over the prior on the median pair
    assert s["fallback_rate"] < 1.0, s
    assert s["median_warm_iters"] < s["median_prior_iters"], s


def test_coarse_start_at_2048(h):
    """2048^2 with the 4x coarser start (the 512^2 problem solved to gap 1e-6):
    the warm-started solve reaches the relative gap 1e-5 in fewer fine
    iterations than the zero start."""
    from paper_1805_09453_gb300 import gprox

    N = 2048
    f0, f1 = (torch.from_numpy(a).cuda() for a in synth.gaussian_mixture_pair(N, 4))
    base = gprox.Cnn(h, 1, seed=0)
    base.set_params(np.zeros(base.num_params, np.float32))
    m = torch.empty((2, N, N), device="cuda")
    o = gprox.default_opts(max_iters=60000, tol_rel_gap=1e-5, gap_every=10, use_graph=1)
    oc = gprox.default_opts(max_iters=200000, tol_rel_gap=1e-6, gap_every=50, use_graph=1)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        st, rz = gprox.emd_solve(h, f0, f1, m, None, None, o)
        h.check(st)
        st, rw = gprox.emd_solve_learned(h, base, f0, f1, m, None, None, o, 4, oc)
        base.check(st)
        stream.synchronize()
    print(f"2048^2: zero {rz['iters']} it {rz['seconds']:.2f} s, coarse start {rw['iters']} it {rw['seconds']:.2f} s")
    assert rw["start"] in ("prior", "learned") and rw["rel_gap"] <= 1e-5  # both are the prior here
    assert rw["iters"] < rz["iters"]
    base.close()
