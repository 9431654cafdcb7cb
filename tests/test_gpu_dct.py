"""dct2_poisson (the u-step solve of sections 3.1 / 3.2, Appendix A cosine
basis) through the C ABI against the oracle's solve, element by element.

Tolerance: FP32 transforms have relative error O(log N * 2^-24); the bar is a
relative L2 error of 2e-5 (an order of magnitude of headroom), on power-of-two
(fast) and ragged / odd (dense) sizes, with and without the constant mode.
"""
import numpy as np
import pytest
import torch

from oracle import gprox_oracle as O
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    hh = gprox.Handle(0)
    yield hh
    hh.close()


@pytest.mark.parametrize("N", [1, 2, 7, 16, 32, 33, 64, 128, 129, 256, 512, 1000, 1024, 2048])
@pytest.mark.parametrize("alpha", [0.0, 3.7, 1e4])
def test_dct2_poisson_matches_oracle(h, N, alpha):
    from paper_1805_09453_gb300 import gprox

    rng = np.random.default_rng(N + int(alpha))
    b = rng.normal(size=(N, N)).astype(np.float32)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    h.check(gprox.dct2_poisson(h, bd, xd, alpha))
    x = xd.cpu().numpy()
    ref = O.helmholtz_solve(b.astype(np.float64), alpha, 1.0 / N)
    if N == 1 and alpha == 0.0:
        assert np.all(x == 0)
        return
    assert rel_l2(x, ref) < 2e-5, rel_l2(x, ref)


def test_dct2_poisson_in_place_and_full_size(h):
    from paper_1805_09453_gb300 import gprox

    N = 4096
    rng = np.random.default_rng(4096)
    b = rng.normal(size=(N, N)).astype(np.float32)
    ref = O.helmholtz_solve(b.astype(np.float64), 50.0, 1.0 / N)
    bd = torch.from_numpy(b).cuda()
    h.check(gprox.dct2_poisson(h, bd, bd, 50.0))  # x aliases b
    assert rel_l2(bd.cpu().numpy(), ref) < 2e-5


def test_dct2_poisson_largest_fast_size(h):
    """8192 x 8192 (the largest fast-transform size; column pass on bulk
    tensor copies with 8 boxes per column pair) against the FP64 oracle."""
    from paper_1805_09453_gb300 import gprox

    N = 8192
    rng = np.random.default_rng(8192)
    b = rng.normal(size=(N, N)).astype(np.float32)
    ref = O.helmholtz_solve(b.astype(np.float64), 3.7, 1.0 / N)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    h.check(gprox.dct2_poisson(h, bd, xd, 3.7))
    assert rel_l2(xd.cpu().numpy(), ref) < 2e-5


def test_dct2_poisson_errors(h):
    from paper_1805_09453_gb300 import gprox

    b = torch.zeros((8, 8), device="cuda")
    x = torch.empty_like(b)
    assert gprox.dct2_poisson(h, b, x, -1.0) == gprox.GP_ERR_ARG
    assert gprox.dct2_poisson(h, b, x, 0.0, prec=9) == gprox.GP_ERR_ARG
    host = torch.zeros((8, 8))
    assert gprox.dct2_poisson(h, host, x, 1.0) == gprox.GP_ERR_ARG
    assert "device pointer" in h.last_error()


@pytest.mark.parametrize("N", [7, 16, 33, 64, 128, 512, 1024, 2048, 4096, 8192])
@pytest.mark.parametrize("alpha", [0.0, 3.7])
def test_dct2_poisson_grad_matches_oracle(h, N, alpha):
    """Spectral gradient of the solve vs the FP64 oracle's forward differences:
    relative L2 2e-5 at every size (differencing an FP32 solution would lose
    ~log2(N) bits: ~1e-4 at 4096)."""
    from paper_1805_09453_gb300 import gprox

    rng = np.random.default_rng(7 * N + int(alpha))
    b = rng.normal(size=(N, N)).astype(np.float32)
    if N >= 1024:  # smooth right-hand side (the EMD regime): the potential dwarfs its grid-scale variation
        x = (np.arange(N) + 0.5) / N
        X, Y = np.meshgrid(x, x)
        b = (np.exp(-((X - 0.3) ** 2 + (Y - 0.6) ** 2) / 0.01) - np.exp(-((X - 0.7) ** 2 + (Y - 0.4) ** 2) / 0.02)).astype(np.float32)
    bd = torch.from_numpy(b).cuda()
    g = torch.empty((2, N, N), device="cuda")
    h.check(gprox.dct2_poisson_grad(h, bd, g, alpha))
    ref = O.helmholtz_solve(b.astype(np.float64), alpha, 1.0 / N)
    gx, gy = O.grad(ref, 1.0 / N)
    assert rel_l2(g.cpu().numpy(), np.stack([gx, gy])) < 2e-5
