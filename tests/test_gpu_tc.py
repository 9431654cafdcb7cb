"""Split-precision (hi + lo BF16) cosine solve on the tcgen05 tensor cores,
through the C ABI, against the FP64 oracle.

Three BF16 products per contraction (hi*hi + hi*lo + lo*hi) with FP32
accumulation leave a relative error of order 2^-16 per contraction; four
contractions per solve: the bar is relative L2 1e-4 (the FP32 fast transform
reaches ~1e-6).  The measured error is part of the precision study of the
split-precision mode."""
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


def test_split_bf16_rejects_unsupported_sizes(h):
    from paper_1805_09453_gb300 import gprox

    b = torch.zeros((96, 96), device="cuda")
    x = torch.empty_like(b)
    assert gprox.dct2_poisson(h, b, x, 1.0, prec="split_bf16") == gprox.GP_ERR_UNSUPPORTED
    assert gprox.dct2_poisson(h, b, x, 1.0, prec="split_fp16") == gprox.GP_ERR_UNSUPPORTED
