"""Three-dimensional G-prox PDHG (the d = 3 instance of Algorithm 2; ROF of
section 3.1, L1-EMD of section 3.2) on the GPU through the C ABI against the
FP64 three-dimensional oracle:

* fixed iteration counts from the zero start, element by element, at 16^3,
  32^3 and 64^3 (one to four CTAs of lines per plane), and at 256^3 for two
  iterations; FP32 bars as the two-dimensional tests: ROF u 1e-4 relative L2,
  p 1e-3 absolute, P 1e-5 relative; EMD m 1e-3 relative L2, P 1e-5, D 1e-4;
* the step rule's tau, the mean of u, a constant volume as the fixed point;
* run to a relative gap: translated balls land near the translation length
  |(1/4, 1/4, 1/4)| (section 4.2's argument holds in any dimension);
* argument errors.
"""
import math

import numpy as np
import pytest
import torch

from oracle import gprox_oracle3d as O3
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


def _noisy_ball(N, seed):
    rng = np.random.default_rng(seed)
    return (synth.ball_image3(N) + 0.1 * rng.normal(size=(N, N, N))).astype(np.float32)


@pytest.mark.parametrize("N,lam,iters", [(16, 8.0, 30), (32, 8.0, 30), (64, 20.0, 20)])
def test_rof3_fixed_iterations_match_oracle(h, N, lam, iters):
    from paper_1805_09453_gb300 import gprox

    I = _noisy_ball(N, N)
    u = torch.empty((N, N, N), device="cuda")
    p = torch.empty((3, N, N, N), device="cuda")
    st, rep = gprox.rof_solve3d(h, _t(I), u, p, lam,
                                gprox.default_opts(max_iters=iters, tol_rel_gap=0.0, gap_every=10))
    h.check(st)
    ref = O3.rof_solve3(I.astype(np.float64), lam, iters)
    assert rep["iters"] == iters
    assert abs(rep["tau"] - ref["tau"]) < 1e-6 * ref["tau"]
    assert rel_l2(u.cpu().numpy(), ref["u"]) <= 1e-4
    pc = p.cpu().numpy()
    for k in range(3):
        assert np.abs(pc[k] - ref["p"][k]).max() < 1e-3
    assert abs(rep["primal"] - ref["primal"]) <= 1e-5 * abs(ref["primal"])
    assert abs(rep["dual"] - ref["dual"]) <= 1e-5 * abs(ref["primal"])
    assert abs(u.double().mean().item() - I.astype(np.float64).mean()) < 1e-5


@pytest.mark.parametrize("N,iters", [(16, 40), (32, 40), (64, 20)])
def test_emd3_fixed_iterations_match_oracle(h, N, iters):
    from paper_1805_09453_gb300 import gprox

    f0, f1 = synth.gaussian_mixture_pair3(N, N)
    m = torch.empty((3, N, N, N), device="cuda")
    p = torch.empty((3, N, N, N), device="cuda")
    st, rep = gprox.emd_solve3d(h, _t(f0), _t(f1), m, p,
                                gprox.default_opts(max_iters=iters, tol_rel_gap=0.0, gap_every=10))
    h.check(st)
    ref = O3.emd_solve3(f0, f1, iters)
    assert rep["iters"] == iters
    mc = m.cpu().numpy()
    assert rel_l2(mc, np.stack(ref["m"])) < 1e-3
    pc = p.cpu().numpy()
    for k in range(3):
        assert np.abs(pc[k] - ref["p"][k]).max() < 1e-3
    assert abs(rep["primal"] - ref["primal"]) < 1e-5 * ref["primal"]
    assert abs(rep["dual"] - ref["dual"]) < 1e-4 * abs(ref["primal"])
    # every iterate is feasible up to FP32 rounding (the Leray step keeps div m = f0 - f1)
    assert rep["mass_residual"] < 1e-4
    assert math.isnan(rep["rel_gap_feasible"])


def test_emd3_zero_iterations_is_the_hodge_start(h):
    from paper_1805_09453_gb300 import gprox

    N = 32
    f0, f1 = synth.gaussian_mixture_pair3(N, 5)
    m = torch.empty((3, N, N, N), device="cuda")
    st, rep = gprox.emd_solve3d(h, _t(f0), _t(f1), m, None, gprox.default_opts(max_iters=0, tol_rel_gap=0.0))
    h.check(st)
    ref = O3.emd_init3(f0, f1)
    assert rep["iters"] == 0
    assert rel_l2(m.cpu().numpy(), np.stack(ref["m"])) < 1e-4
    assert rep["dual"] == 0.0


def test_rof3_constant_volume_is_the_fixed_point(h):
    from paper_1805_09453_gb300 import gprox

    N = 32
    I = np.full((N, N, N), 0.3, np.float32)
    u = torch.empty((N, N, N), device="cuda")
    p = torch.empty((3, N, N, N), device="cuda")
    st, rep = gprox.rof_solve3d(h, _t(I), u, p, 8.0, gprox.default_opts(max_iters=5, tol_rel_gap=0.0))
    h.check(st)
    assert torch.allclose(u, _t(I), atol=1e-6)
    assert p.abs().max().item() < 1e-6


def test_3d_256_two_iterations_match_oracle(h):
    """The largest grid the three-dimensional benchmark runs, two iterations."""
    from paper_1805_09453_gb300 import gprox

    N, lam = 256, 20.0
    I = _noisy_ball(N, 1)
    u = torch.empty((N, N, N), device="cuda")
    st, rep = gprox.rof_solve3d(h, _t(I), u, None, lam, gprox.default_opts(max_iters=2, tol_rel_gap=0.0))
    h.check(st)
    ref = O3.rof_solve3(I.astype(np.float64), lam, 2)
    assert rel_l2(u.cpu().numpy(), ref["u"]) <= 1e-4
    assert abs(rep["primal"] - ref["primal"]) <= 1e-5 * abs(ref["primal"])
    del ref
    f0, f1 = synth.translated_balls3(N)
    m = torch.empty((3, N, N, N), device="cuda")
    st, rep = gprox.emd_solve3d(h, _t(f0), _t(f1), m, None, gprox.default_opts(max_iters=2, tol_rel_gap=0.0))
    h.check(st)
    ref = O3.emd_solve3(f0, f1, 2)
    assert rel_l2(m.cpu().numpy(), np.stack(ref["m"])) < 1e-3
    assert abs(rep["primal"] - ref["primal"]) < 1e-5 * ref["primal"]


def test_emd3_translated_balls_to_gap(h):
    from paper_1805_09453_gb300 import gprox

    N = 32
    f0, f1 = synth.translated_balls3(N)
    m = torch.empty((3, N, N, N), device="cuda")
    st, rep = gprox.emd_solve3d(h, _t(f0), _t(f1), m, None,
                                gprox.default_opts(max_iters=20000, tol_rel_gap=1e-4, gap_every=0))
    h.check(st)
    assert st == gprox.GP_OK and 0.0 <= rep["rel_gap"] <= 1e-4
    assert abs(rep["primal"] - math.sqrt(3) / 4) < 0.1 * math.sqrt(3) / 4, rep


def test_3d_argument_errors(h):
    from paper_1805_09453_gb300 import gprox

    N = 16
    I = torch.zeros((N, N, N), device="cuda")
    u = torch.empty_like(I)
    with pytest.raises(ValueError):
        gprox.rof_solve3d(h, I, torch.empty((N, N), device="cuda"))
    with pytest.raises(ValueError):
        gprox.emd_solve3d(h, I, I, torch.empty((2, N, N, N), device="cuda"))
    J = torch.zeros((24, 24, 24), device="cuda")
    st, _ = gprox.rof_solve3d(h, J, torch.empty_like(J))
    assert st == gprox.GP_ERR_ARG
    st, _ = gprox.rof_solve3d(h, I, u, None, 8.0, gprox.default_opts(prec="split_bf16"))
    assert st == gprox.GP_ERR_UNSUPPORTED
    st, _ = gprox.rof_solve3d(h, I, u, None, 8.0, gprox.default_opts(warm_start=1))
    assert st == gprox.GP_ERR_UNSUPPORTED
    f1 = torch.full((N, N, N), 2.0, device="cuda")
    st, _ = gprox.emd_solve3d(h, torch.ones((N, N, N), device="cuda"), f1, torch.empty((3, N, N, N), device="cuda"))
    assert st == gprox.GP_ERR_MASS
