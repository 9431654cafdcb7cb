"""ROF G-prox PDHG (section 3.1) on the GPU through the C ABI vs the FP64 oracle.

Bars (FP32 plain path): relative L2 iterate error <= 1e-4 after a fixed
number of iterations and relative objective error <= 1e-6 on the 128 x 128
noisy-shapes workload (lambda = 8, 500 iterations); single steps from random
states agree to FP32 rounding (u: 2e-5 relative L2, p: 3e-4 absolute -- p is
the projection of p + sigma grad u, whose FP32 rounding is amplified by the
1/h of the gradient on random, non-smooth states).
"""
import numpy as np
import pytest
import torch

from oracle import gprox_oracle as O
from paper_1805_09453_gb300 import synth
from tests.gpu_common import random_unit_field, rel_l2

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


def test_rof_128_500_iterations_parity(h):
    from paper_1805_09453_gb300 import gprox

    N, lam = 128, 8.0
    I = synth.rof_image(N, 0)
    u = torch.empty((N, N), device="cuda")
    p = torch.empty((2, N, N), device="cuda")
    st, rep = gprox.rof_solve(h, _t(I), u, p, lam, gprox.default_opts(max_iters=500, tol_rel_gap=0.0))
    h.check(st)
    ref = O.rof_solve(I, lam, n_iters=500)
    assert abs(rep["tau"] - ref["tau"]) < 1e-6 * ref["tau"]
    assert rel_l2(u.cpu().numpy(), ref["u"]) <= 1e-4
    assert abs(rep["primal"] - ref["primal"]) <= 1e-6 * abs(ref["primal"])
    assert rep["iters"] == 500
    pc = p.cpu().numpy()
    assert np.abs(pc[0] - ref["px"]).max() < 1e-3 and np.abs(pc[1] - ref["py"]).max() < 1e-3


@pytest.mark.parametrize("N", [1, 2, 5, 16, 33, 64, 128, 129])
@pytest.mark.parametrize("n_steps", [1, 3])
def test_rof_steps_from_random_state(h, N, n_steps):
    from paper_1805_09453_gb300 import gprox

    rng = np.random.default_rng(10 * N + n_steps)
    lam, tau, sigma = 8.0, 2.0, 0.5
    I = rng.uniform(0, 1, (N, N)).astype(np.float32)
    u0 = rng.uniform(0, 1, (N, N)).astype(np.float32)
    p0 = random_unit_field(N, N + 1)
    pb0 = random_unit_field(N, N + 2, scale=2.0)
    Id = _t(I)
    s = gprox.State(h, "rof", N, I=Id, lam=lam, tau=tau, sigma=sigma, primal0=_t(u0),
                    p0=_t(np.stack(p0)), pbar0=_t(np.stack(pb0)))
    s.step(n_steps)
    u, p = s.read()
    ref = O.rof_init(I, u0, p0, pb0)
    O.rof_iterate(ref, I, lam, tau, sigma, n_steps)
    assert rel_l2(u.cpu().numpy(), ref["u"]) < 2e-5
    pc = p.cpu().numpy()
    assert np.abs(pc[0] - ref["px"]).max() < 3e-4 and np.abs(pc[1] - ref["py"]).max() < 3e-4
    g = s.gap()
    P, D, gg = O.rof_gap(ref["u"], ref["px"], ref["py"], I, lam)
    assert abs(g["primal"] - P) < 1e-5 * max(1.0, abs(P)) and abs(g["dual"] - D) < 1e-5 * max(1.0, abs(D))
    s.close()


def test_rof_converges_and_state_gap_matches_report(h):
    from paper_1805_09453_gb300 import gprox

    N, lam = 96, 10.0
    I = synth.rof_image(N, 3)
    Id = _t(I)
    u = torch.empty((N, N), device="cuda")
    p = torch.empty((2, N, N), device="cuda")
    st, rep = gprox.rof_solve(h, Id, u, p, lam, gprox.default_opts(max_iters=5000, tol_rel_gap=1e-6))
    assert st == gprox.GP_OK and rep["rel_gap"] <= 1e-6
    ref = O.rof_solve(I, lam, tol=1e-10)
    # lambda-strong convexity (Corollary 3.4): ||u - u*||^2 <= 2 gap / lambda
    err2 = np.sum((u.cpu().numpy() - ref["u"]) ** 2) / N ** 2
    assert err2 <= 2.0 * (rep["primal"] - rep["dual"]) / lam + 1e-9
    # mean preserved (sum of the u-update)
    assert abs(u.mean().item() - I.mean()) < 1e-5
    # a warm start from the returned state starts from that state: its initial
    # objective equals the final one of the first solve
    st2, rep2 = gprox.rof_solve(h, Id, u, p, lam, gprox.default_opts(max_iters=0, tol_rel_gap=0.0, warm_start=1))
    assert st2 == gprox.GP_OK and rep2["iters"] == 0
    assert abs(rep2["primal"] - rep["primal"]) < 1e-6 * abs(rep["primal"])


def test_rof_constant_image_and_errors(h):
    from paper_1805_09453_gb300 import gprox

    N = 32
    I = torch.full((N, N), 0.25, device="cuda")
    u = torch.empty_like(I)
    st, rep = gprox.rof_solve(h, I, u, None, 8.0, gprox.default_opts(max_iters=20, tol_rel_gap=0.0))
    h.check(st)
    assert rep["tau"] == 1.0  # constant image: the rule's tau is 0, 1 is used
    assert torch.allclose(u, I, atol=1e-6)
    assert gprox.rof_solve(h, I, u, None, -1.0)[0] == gprox.GP_ERR_ARG
    assert gprox.rof_solve(h, I, u, None, 8.0, gprox.default_opts(gap_every=-1))[0] == gprox.GP_ERR_ARG
    # gap_every = 0 selects the adaptive check schedule
    st, rep = gprox.rof_solve(h, I, u, None, 8.0, gprox.default_opts(max_iters=50, gap_every=0, tol_rel_gap=1e-5))
    assert st == gprox.GP_OK and rep["iters"] % 10 == 0
    bad = I.clone()
    bad[3, 3] = float("nan")
    st, _ = gprox.rof_solve(h, bad, u, None, 8.0, gprox.default_opts(max_iters=10, tau=1.0))
    assert st == gprox.GP_ERR_NONFINITE


def test_rof_full_size_two_iterations(h):
    """4096 x 4096 (the benchmark size): two iterations element by element."""
    from paper_1805_09453_gb300 import gprox

    N, lam = 4096, 8.0
    I = synth.rof_image(N, 2)
    u = torch.empty((N, N), device="cuda")
    p = torch.empty((2, N, N), device="cuda")
    st, rep = gprox.rof_solve(h, _t(I), u, p, lam, gprox.default_opts(max_iters=2, gap_every=2, tol_rel_gap=0.0))
    h.check(st)
    ref = O.rof_solve(I, lam, n_iters=2)
    assert abs(rep["tau"] - ref["tau"]) < 1e-6 * ref["tau"]
    assert rel_l2(u.cpu().numpy(), ref["u"]) < 2e-5
    assert abs(rep["primal"] - ref["primal"]) < 1e-5 * abs(ref["primal"])
    assert abs(u.double().mean().item() - I.astype(np.float64).mean()) < 1e-5
