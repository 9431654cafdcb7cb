"""ROF warm starts (section 3.1 with a start other than zero): the coarse-grid
start against the FP64 oracle, the gap-decided choice among the learned, the
prior and the zero start, and what a trained network gains.

The coarse start is restriction by block means, the coarse ROF iteration and
cell-centred bilinear interpolation of u and p (p then made feasible).  The
test rebuilds it from the oracle's coarse iteration with its own numpy
interpolation; bars as the ROF parity tests (u 1e-4 relative L2, p 1e-3
absolute).  Whatever the start, the solve must land on the same minimiser:
two solves that each certify a relative gap of 1e-5 have primal values within
2e-5 of each other (both lie within 1e-5 of the optimum).
"""
import numpy as np
import pytest
import torch

from oracle import gprox_oracle as O
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


def _block_mean(a, k):
    n = a.shape[0] // k
    return a.reshape(n, k, n, k).mean(axis=(1, 3))


def _upsample(c, k):
    """Cell-centred bilinear interpolation n -> n k, clamped at the outer centres."""
    n = c.shape[0]
    x = np.clip((np.arange(n * k) + 0.5) / k - 0.5, 0, n - 1)
    i0 = np.minimum(np.floor(x).astype(int), n - 1)
    i1 = np.minimum(i0 + 1, n - 1)
    t = x - i0
    rows = c[i0, :] * (1 - t)[:, None] + c[i1, :] * t[:, None]
    return rows[:, i0] * (1 - t)[None, :] + rows[:, i1] * t[None, :]


@pytest.mark.parametrize("N,k", [(64, 2), (64, 4), (128, 4)])
def test_rof_coarse_start_matches_oracle(h, N, k):
    from paper_1805_09453_gb300 import gprox

    lam, iters = 8.0, 120
    I = synth.rof_image(N, 31)
    st, u, p, rep = gprox.rof_coarse_start(h, torch.from_numpy(I).cuda(), k, lam,
                                           gprox.default_opts(max_iters=iters, tol_rel_gap=0.0, gap_every=iters))
    h.check(st)
    assert rep["iters"] == iters
    ref = O.rof_solve(_block_mean(I.astype(np.float64), k), lam, n_iters=iters)
    uref = _upsample(ref["u"], k)
    px, py = _upsample(ref["px"], k), _upsample(ref["py"], k)
    px[:, -1] = 0.0
    py[-1, :] = 0.0
    nrm = np.maximum(1.0, np.hypot(px, py))
    assert rel_l2(u.cpu().numpy(), uref) < 1e-4
    pc = p.cpu().numpy()
    assert np.abs(pc[0] - px / nrm).max() < 1e-3 and np.abs(pc[1] - py / nrm).max() < 1e-3
    assert np.hypot(pc[0], pc[1]).max() <= 1.0 + 1e-6


def test_rof_learned_start_choice_and_optimum(h):
    """A new network (zero head) returns its prior: the learned and prior starts
    coincide, one of them is kept, and the solve reaches the same minimiser as
    the zero start.  Without a prior the learned start is mean(I) + the
    network's correction, again judged by the gap at n = 0."""
    from paper_1805_09453_gb300 import gprox

    N, lam = 128, 8.0
    I = torch.from_numpy(synth.rof_image(N, 5)).cuda()
    net = gprox.Cnn(h, 4, seed=3)
    o = gprox.default_opts(max_iters=5000, tol_rel_gap=1e-5, gap_every=10)
    u0 = torch.empty((N, N), device="cuda")
    st, rz = gprox.rof_solve(h, I, u0, None, lam, o)
    h.check(st)
    u1 = torch.empty((N, N), device="cuda")
    p1 = torch.empty((2, N, N), device="cuda")
    st, rw = gprox.rof_solve_learned(h, net, I, u1, p1, lam, o, coarse_factor=4)
    net.check(st)
    assert rw["start"] in ("learned", "prior")
    assert st == gprox.GP_OK and rw["rel_gap"] <= 1e-5
    assert abs(rw["primal"] - rz["primal"]) <= 2e-5 * rz["primal"]
    assert rel_l2(u1.cpu().numpy(), u0.cpu().numpy()) < 1e-3
    assert rw["iters"] < rz["iters"]  # the coarse solution is a better start than zero
    st, rn = gprox.rof_solve_learned(h, net, I, u1, None, lam, o, coarse_factor=0)
    net.check(st)
    assert rn["start"] in ("learned", "zero") and st == gprox.GP_OK
    assert abs(rn["primal"] - rz["primal"]) <= 2e-5 * rz["primal"]


def test_rof_trained_network_start_is_gap_decided(h):
    """Train a small network (C = 8) on 64 solved 128^2 images, its prior the 4x
    coarser solve, and solve 8 held-out images to a relative gap of 1e-5 from
    the zero start, the prior and the learned start.  Every arm reaches the
    same minimiser, the warm starts save iterations over zero, and training
    does not worsen the held-out fit of u*.  (Measured: the held-out loss
    barely moves from the prior's, FP32 and BF16 alike: at lambda = 40 the
    minimiser keeps noise-shaped small plateaus that the coarse prior lacks
    and that dominate the gradient term of the loss; the gap at n = 0 then
    keeps whichever of the prior and the learned start is closer.)"""
    from paper_1805_09453_gb300 import gprox, learn

    N, k, lam = 128, 4, 40.0
    f0, f1, tgt, pri, _, iters, gaps = learn.generate_rof(h, N, range(64), lam, tol=1e-5, max_iters=5000,
                                                          coarse_factor=k)
    assert max(gaps) <= 1e-4  # training targets: a start needs no more
    g0, g1, gt, gp, gI, _, _ = learn.generate_rof(h, N, range(learn.TEST_SEED0, learn.TEST_SEED0 + 8), lam,
                                                  tol=1e-5, max_iters=5000, coarse_factor=k)
    net = gprox.Cnn(h, 8, seed=0)
    L0 = learn.test_loss(net, g0, g1, gt, gp)
    hist = learn.train(net, f0, f1, tgt, pri, steps=400, batch=16, lr=1e-3)
    L1 = learn.test_loss(net, g0, g1, gt, gp)
    print("held-out loss: prior", L0, "trained", L1)
    assert L1 <= L0 * (1 + 1e-2), (L0, L1, hist[-3:])
    rows = learn.evaluate_rof(h, net, gI, lam, tol=1e-5, max_iters=40000, coarse_factor=k)
    s = learn.summarize(rows)
    print(s)
    assert all(r["warm_status"] == "GP_OK" and r["zero_status"] == "GP_OK" for r in rows), rows
    assert all(abs(r["warm_primal"] - r["zero_primal"]) <= 2e-5 * r["zero_primal"] for r in rows), rows
    assert all(r["warm_start"] in ("learned", "prior") for r in rows), rows
    assert s["median_warm_iters"] < s["median_zero_iters"], s
    assert s["median_prior_iters"] < s["median_zero_iters"], s
