"""Split-precision cosine solves on the tcgen05 tensor cores, through the C
ABI, against the FP64 oracle.

Three 16-bit products per contraction (hi*hi + hi*lo + lo*hi) with FP32
accumulation in tensor memory.  BF16 parts carry 8 significant bits each, a
relative error of order 2^-16 per contraction; four contractions per solve:
bar 1e-4 (the FP32 fast transform reaches ~3e-7).  FP16 parts carry 11 bits
(after a power-of-two scale that keeps each operand inside FP16's range), but
the measured error is hardly smaller than BF16's and grows linearly with N
(256^2: 4.9e-6, 1024^2: 1.1e-5, 4096^2: 4.5e-5): the tensor core's FP32
accumulation, about one biased rounding per K = 16 step, dominates both.
Bar 1e-4 as BF16.  One step of residual correction (r = b - (alpha - Lap) x
in FP64 from the stored x, x += solve(r)) removes most of it: bar 5e-6 at
these sizes and at least 5x below the plain BF16 split; the refined gradient
(differences of the stored first solution plus the split gradient of the
correction) 1e-5.  The measured errors are part of the precision study."""
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


@pytest.mark.parametrize("N", [128, 256, 384, 1024])
@pytest.mark.parametrize("alpha", [0.0, 3.7, 1e4])
def test_split_bf16_solve_matches_oracle(h, N, alpha):
    from paper_1805_09453_gb300 import gprox

    rng = np.random.default_rng(N + int(alpha))
    b = rng.normal(size=(N, N)).astype(np.float32)
    bd = torch.from_numpy(b).cuda()
    x = torch.empty_like(bd)
    h.check(gprox.dct2_poisson(h, bd, x, alpha, prec="split_bf16"))
    ref = O.helmholtz_solve(b.astype(np.float64), alpha, 1.0 / N)
    err = rel_l2(x.cpu().numpy(), ref)
    assert err < 1e-4, err


@pytest.mark.parametrize("N", [128, 384, 1024])
@pytest.mark.parametrize("alpha", [0.0, 3.7, 1e4])
@pytest.mark.parametrize("prec,bar,ratio", [("split_fp16", 1e-4, 2.0), ("split_bf16_refined", 5e-6, 0.2),
                                            ("split_fp16_refined", 5e-6, 0.2)])
def test_split_modes_match_oracle(h, N, alpha, prec, bar, ratio):
    from paper_1805_09453_gb300 import gprox

    rng = np.random.default_rng(N + int(alpha) + 7)
    b = (rng.normal(size=(N, N)) * 3.0 + 1.0).astype(np.float32)
    bd = torch.from_numpy(b).cuda()
    x = torch.empty_like(bd)
    h.check(gprox.dct2_poisson(h, bd, x, alpha, prec=prec))
    ref = O.helmholtz_solve(b.astype(np.float64), alpha, 1.0 / N)
    err = rel_l2(x.cpu().numpy(), ref)
    xb = torch.empty_like(bd)
    h.check(gprox.dct2_poisson(h, bd, xb, alpha, prec="split_bf16"))
    err_bf16 = rel_l2(xb.cpu().numpy(), ref)
    print(f"N={N} alpha={alpha} {prec}: {err:.3e} (split_bf16 {err_bf16:.3e})")
    assert err < bar and err < ratio * err_bf16, (err, err_bf16)


@pytest.mark.parametrize("prec,bar", [("split_fp16", 1e-4), ("split_bf16_refined", 1e-5),
                                      ("split_fp16_refined", 1e-5)])
def test_split_modes_in_place_and_gradient(h, prec, bar):
    """b may alias x (the refined modes keep a copy of b for the residual), and
    the spectral gradient of the split solve matches the oracle's forward
    differences of its solution."""
    from paper_1805_09453_gb300 import gprox

    N, alpha = 256, 0.0
    rng = np.random.default_rng(11)
    b = rng.normal(size=(N, N)).astype(np.float32)
    ref = O.helmholtz_solve(b.astype(np.float64), alpha, 1.0 / N)
    x = torch.from_numpy(b.copy()).cuda()
    h.check(gprox.dct2_poisson(h, x, x, alpha, prec=prec))
    assert rel_l2(x.cpu().numpy(), ref) < bar
    g = torch.empty((2, N, N), device="cuda")
    h.check(gprox.dct2_poisson_grad(h, torch.from_numpy(b).cuda(), g, alpha, prec=prec))
    gx, gy = O.grad(ref, 1.0 / N)
    assert rel_l2(g.cpu().numpy(), np.stack([gx, gy])) < bar


def test_split_bf16_rejects_unsupported_sizes(h):
    from paper_1805_09453_gb300 import gprox

    b = torch.zeros((96, 96), device="cuda")
    x = torch.empty_like(b)
    assert gprox.dct2_poisson(h, b, x, 1.0, prec="split_bf16") == gprox.GP_ERR_UNSUPPORTED
    for prec in ("split_fp16", "split_bf16_refined", "split_fp16_refined"):
        assert gprox.dct2_poisson(h, b, x, 1.0, prec=prec) == gprox.GP_ERR_UNSUPPORTED
    assert gprox.lib().dct2_poisson(h.ptr, gprox._ptr(b), gprox._ptr(x), 96, 1.0, 5, None) == gprox.GP_ERR_ARG
