"""CP2 (the accelerated PDHG comparison method of section 4.1) on the GPU
through the C ABI against the FP64 oracle's CP2:

* fixed iteration counts from the zero start, element by element at sizes
  from 2 to 129 (ragged and power-of-two), and at 4096^2 (the benchmark
  size) for two iterations; FP32 bars: u 1e-5 relative L2, p 1e-4 absolute,
  P 1e-6 relative;
* run to a relative gap: the value agrees with the G-prox optimum (both
  methods solve the same ROF problem, whose minimiser is unique);
* argument errors.
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


@pytest.mark.parametrize("N", [2, 7, 16, 33, 64, 128, 129])
def test_cp2_fixed_iterations_match_oracle(h, N):
    from paper_1805_09453_gb300 import gprox

    lam, iters = 8.0, 150
    I = synth.rof_image(N, N)
    u = torch.empty((N, N), device="cuda")
    p = torch.empty((2, N, N), device="cuda")
    st, rep = gprox.rof_solve_cp2(h, _t(I), u, p, lam, gprox.default_opts(max_iters=iters, tol_rel_gap=0.0,
                                                                           gap_every=50))
    h.check(st)
    ref = O.rof_cp2_solve(I, lam, n_iters=iters)
    assert rep["iters"] == iters
    assert rel_l2(u.cpu().numpy(), ref["u"]) < 1e-5
    pc = p.cpu().numpy()
    assert np.abs(pc[0] - ref["px"]).max() < 1e-4 and np.abs(pc[1] - ref["py"]).max() < 1e-4
    assert abs(rep["primal"] - ref["primal"]) <= 1e-6 * abs(ref["primal"])
    assert abs(rep["tau"] - ref["tau"]) <= 1e-12 * ref["tau"]


def test_cp2_reaches_the_gprox_optimum(h):
    from paper_1805_09453_gb300 import gprox

    N, lam = 64, 8.0
    I = synth.rof_image(N, 1)
    u = torch.empty((N, N), device="cuda")
    st, rep = gprox.rof_solve_cp2(h, _t(I), u, None, lam, gprox.default_opts(max_iters=200000, tol_rel_gap=1e-5))
    assert st == gprox.GP_OK and rep["rel_gap"] <= 1e-5
    ref = O.rof_solve(I, lam, tol=1e-9, max_iters=100000)
    assert abs(rep["primal"] - ref["primal"]) <= 1.1e-5 * ref["primal"]
    assert rep["dual"] <= ref["primal"] * (1 + 1e-6)


def test_cp2_full_size_two_iterations(h):
    from paper_1805_09453_gb300 import gprox

    N, lam = 4096, 8.0
    I = synth.rof_image(N, 0)
    u = torch.empty((N, N), device="cuda")
    p = torch.empty((2, N, N), device="cuda")
    st, rep = gprox.rof_solve_cp2(h, _t(I), u, p, lam, gprox.default_opts(max_iters=2, tol_rel_gap=0.0))
    h.check(st)
    ref = O.rof_cp2_solve(I, lam, n_iters=2)
    assert rel_l2(u.cpu().numpy(), ref["u"]) < 1e-5
    pc = p.cpu().numpy()
    assert np.abs(pc[0] - ref["px"]).max() < 1e-4 and np.abs(pc[1] - ref["py"]).max() < 1e-4


def test_cp2_errors(h):
    from paper_1805_09453_gb300 import gprox

    I = torch.zeros((8, 8), device="cuda")
    u = torch.empty_like(I)
    assert gprox.rof_solve_cp2(h, I, u, None, -1.0)[0] == gprox.GP_ERR_ARG
    assert gprox.rof_solve_cp2(h, I, u, None, 1.0, gprox.default_opts(warm_start=1))[0] == gprox.GP_ERR_ARG
