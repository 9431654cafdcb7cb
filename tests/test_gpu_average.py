"""Ergodic averages (the iterate averages u^n = (1/n) sum_{k=1..n} u_k,
p^n = (1/n) sum p_k of the convergence theorems, sections 3.1 / 3.2) on the
GPU against the FP64 oracle's iterates averaged by definition.

The library never stores the primal iterates: it sums the right-hand sides
(ROF r_k, EMD s_k and d_k) in FP64 and takes the primal average through the
solve's linearity at read time, so this checks that identity as well as the
bookkeeping (steps over several pd_step calls, restart, errors).  Bars: the
FP32 iterate bars of the single-step tests (primal relative L2 1e-4; p
absolute 3e-4 EMD, 1e-3 ROF, where the 1/h of the gradient amplifies FP32
rounding in p over the steps).
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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("N", [64, 129, 512])
def test_rof_average_matches_oracle(h, N):
    from paper_1805_09453_gb300 import gprox

    lam = 8.0
    I = synth.rof_image(N, 1)
    tau, sigma, _ = O.rof_step_rule(I, lam)
    s = gprox.State(h, "rof", N, I=_t(I), lam=lam, tau=tau, sigma=sigma)
    s.step(3)  # not averaged
    s.average(True)
    s.step(7)
    s.step(13)
    ub, pb, n = s.read_average()
    assert n == 20
    ref = O.rof_init(I)
    us, pxs, pys = [], [], []
    O.rof_iterate(ref, I, lam, tau, sigma, 3)
    O.rof_iterate(ref, I, lam, tau, sigma, 20,
                  callback=lambda k, u, px, py: (us.append(u), pxs.append(px), pys.append(py)))
    u_avg = np.mean(us, axis=0)
    assert rel_l2(ub.cpu().numpy(), u_avg) < 1e-4
    p = pb.cpu().numpy()
    assert np.abs(p[0] - np.mean(pxs, axis=0)).max() < 1e-3 and np.abs(p[1] - np.mean(pys, axis=0)).max() < 1e-3
    s.close()


@pytest.mark.parametrize("N", [64, 512])
def test_emd_average_matches_oracle(h, N):
    from paper_1805_09453_gb300 import gprox

    f0, f1 = synth.gaussian_mixture_pair(N, 2)
    s = gprox.State(h, "emd", N, f0=_t(f0), f1=_t(f1), tau=1.0)
    s.average(True)
    s.step(10)
    s.step(15)
    mb, pb, n = s.read_average()
    assert n == 25
    ref = O.emd_init(f0, f1)
    ms, ps = [], []
    O.emd_iterate(ref, 1.0, 1.0, 25, callback=lambda k, mx, my, px, py: (ms.append((mx, my)), ps.append((px, py))))
    m_avg = np.mean(np.array(ms), axis=0)
    p_avg = np.mean(np.array(ps), axis=0)
    assert rel_l2(mb.cpu().numpy(), m_avg) < 1e-4
    assert np.abs(pb.cpu().numpy() - p_avg).max() < 3e-4
    # the average of feasible fluxes is feasible: div m = f0 - f1
    mc = mb.cpu().numpy().astype(np.float64)
    res = O.div(mc[0], mc[1], 1.0 / N) - (f0.astype(np.float64) - f1)
    assert np.abs(res).sum() / np.abs(f0.astype(np.float64) - f1).sum() < 1e-3
    s.close()


def test_average_restart_and_errors(h):
    from paper_1805_09453_gb300 import gprox

    N = 32
    f0, f1 = synth.gaussian_mixture_pair(N, 3)
    s = gprox.State(h, "emd", N, f0=_t(f0), f1=_t(f1), tau=1.0)
    with pytest.raises(gprox.GproxError):
        s.read_average()  # averaging not started
    s.average(True)
    with pytest.raises(gprox.GproxError):
        s.read_average()  # no averaged step yet
    s.step(4)
    assert s.read_average()[2] == 4
    s.average(True)  # restart
    s.step(2)
    m2, p2, n = s.read_average()
    assert n == 2 and torch.isfinite(m2).all() and torch.isfinite(p2).all()
    s.average(False)
    with pytest.raises(gprox.GproxError):
        s.read_average()
    s.close()
