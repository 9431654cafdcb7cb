"""dct2_poisson_static: the cosine-basis solve for callers that may not call
cudaMalloc (a host framework that owns all device memory through its own pool,
a real-time loop that may not allocate).  Its scratch lives in static device
arrays inside the library; the caller passes only input and output.

Checked through the C ABI against the allocating dct2_poisson, with the same
tolerance as the other solve tests (relative L2 2e-5), on two calls in a row
(the second reuses the static scratch the first one left behind, with a new
input and a new alpha).  Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    a = a.double()
    b = b.double()
    return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()


def test_static_solve_matches_allocating_solve_on_two_calls():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    h = gprox.Handle(0)
    rng = np.random.default_rng(2024)
    for N, alpha in ((1024, 0.0), (1024, 7.5)):
        b = torch.from_numpy(rng.normal(size=(N, N)).astype(np.float32)).cuda()
        ref = torch.empty_like(b)
        out = torch.full_like(b, float("nan"))
        h.check(gprox.dct2_poisson(h, b, ref, alpha))
        st = gprox.dct2_poisson_static(b, out, alpha)
        assert st == gprox.GP_OK, gprox.static_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel_l2(out, ref) < 2e-5
    h.close()


def test_static_solve_rejects_sizes_beyond_its_maximum():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    b = torch.zeros((2048, 2048), device="cuda")
    x = torch.empty_like(b)
    assert gprox.dct2_poisson_static(b, x, 1.0) == gprox.GP_ERR_ARG
    assert "power-of-two N in [16, 1024]" in gprox.static_last_error()
