"""dct2_poisson_static: the cosine-basis solve for callers that may not call
cudaMalloc (a host framework that owns all device memory through its own pool,
a real-time loop that may not allocate).  Its scratch lives in static device
arrays inside the library; the caller passes only input and output.

Checked through the C ABI against the allocating dct2_poisson and against the
FP64 oracle's solve, with the same tolerance as the other solve tests
(relative L2 2e-5), on calls in a row that change N and come back to an
earlier one (each size change rebuilds the static tables; each call reuses
the scratch the previous one left behind).  Kept in a file of its own that
pytest collects last.
"""
import numpy as np
import pytest
import torch

from oracle import gprox_oracle as O

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_solve_matches_allocating_solve_and_oracle_on_calls_in_a_row():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    h = gprox.Handle(0)
    rng = np.random.default_rng(2024)
    for N, alpha in ((256, 0.0), (1024, 7.5), (64, 1.0), (1024, 0.0), (1024, 7.5)):
        bh = rng.normal(size=(N, N)).astype(np.float32)
        b = torch.from_numpy(bh).cuda()
        ref = torch.empty_like(b)
        out = torch.full_like(b, float("nan"))
        h.check(gprox.dct2_poisson(h, b, ref, alpha))
        st = gprox.dct2_poisson_static(b, out, alpha)
        assert st == gprox.GP_OK, gprox.static_last_error()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.isfinite(o).all()
        assert _rel_l2(o, ref.cpu().numpy()) < 2e-5, (N, alpha)
        exact = O.helmholtz_solve(bh.astype(np.float64), alpha, 1.0 / N)
        if alpha == 0.0:  # the oracle drops b's mean and returns the zero-mean solution
            o = o - o.mean()
        assert _rel_l2(o, exact) < 2e-5, (N, alpha)
    h.close()


def test_static_solve_rejects_sizes_beyond_its_maximum():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    b = torch.zeros((2048, 2048), device="cuda")
    x = torch.empty_like(b)
    assert gprox.dct2_poisson_static(b, x, 1.0) == gprox.GP_ERR_ARG
    assert "power-of-two N in [16, 1024]" in gprox.static_last_error()
    with pytest.raises(ValueError):  # the binding refuses a short output before the library sees it
        gprox.dct2_poisson_static(torch.zeros((64, 64), device="cuda"), torch.empty((32, 32), device="cuda"), 1.0)
