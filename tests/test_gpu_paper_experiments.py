"""The paper-experiment driver on the GPU (section 4): the image norms its
ROF step rules take, reduced on the GPU, against the FP64 oracle's gradient;
and a small run of the protocol (ground truth certified by the gap, iteration
counts to F(u_n) - F* < eps) at 128^2."""
import math

import numpy as np
import pytest
import torch

from oracle import gprox_oracle as O
from paper_1805_09453_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    hh = gprox.Handle(0)
    yield hh
    hh.close()


@pytest.mark.parametrize("kind", ["disc", "noisy"])
def test_rof_image_stats_match_oracle(h, kind):
    from paper_1805_09453_gb300 import gprox

    N = 96
    I = synth.disc_image(N) if kind == "disc" else synth.rof_image(N, 5)
    tv, gl2, dev2 = gprox.rof_image_stats(h, torch.from_numpy(I).cuda())
    I64 = I.astype(np.float64)
    gx, gy = O.grad(I64, 1.0 / N)
    mag = np.hypot(gx, gy)
    h2 = 1.0 / N ** 2
    assert tv == pytest.approx(h2 * mag.sum(), rel=1e-6)
    assert gl2 == pytest.approx(math.sqrt(h2 * (mag ** 2).sum()), rel=1e-6)
    assert dev2 == pytest.approx(h2 * ((I64 - I64.mean()) ** 2).sum(), rel=1e-6)


def test_protocol_small_grid(h):
    from paper_1805_09453_gb300 import paper_experiments as PE

    N = 128
    I = torch.from_numpy(synth.disc_image(N)).cuda()
    from paper_1805_09453_gb300 import gprox

    stats = gprox.rof_image_stats(h, I)
    gt = PE.ground_truth(h, "rof", N, (I,), PE.rof_tau(stats, 10.0, 1e-3), 1e-3, lam=10.0)
    assert gt["certified"] and gt["gap"] < 1e-4
    counts = []
    for eps in (1e-2, 1e-3):
        o, _ = PE.first_below(h, "rof", N, (I,), PE.rof_tau(stats, 10.0, eps), gt["F"], [eps], lam=10.0)
        counts.append(o[eps])
    assert None not in counts and counts[0] <= counts[1], counts
    f0, f1 = (torch.from_numpy(a).cuda() for a in synth.translated_discs(N))
    gt = PE.ground_truth(h, "emd", N, (f0, f1), 1.0, 1e-3)
    assert gt["certified"]
    # the translated discs' distance is |v| = 1/sqrt(8) in the continuum (section 4.2); the grid's
    # anisotropy moves it by a few percent at 128^2
    assert abs(gt["F"] - 1 / math.sqrt(8)) < 0.05 / math.sqrt(8), gt["F"]
    o, _ = PE.first_below(h, "emd", N, (f0, f1), 1.0, gt["F"], [1e-2, 1e-3])
    assert None not in o.values() and o[1e-2] <= o[1e-3], o


def test_delta_measures_tau1_reproduce_the_papers_table():
    """Section 4.2, delta measures with tau = sigma = 1 (the paper's Table 8,
    cited fixture tests/golden/section4_iterations.json): at 512^2 the
    iterations to F(m_n) - F* < eps for eps = 1e-2, 1e-3, 1e-4 agree with the
    printed 93 / 611 / 1864 within 5 % (the same iteration on the same
    problem; the paper's discretisation is unprinted, ours is R1-R4)."""
    import json
    import os

    from paper_1805_09453_gb300 import build, gprox
    from paper_1805_09453_gb300 import paper_experiments as PE

    build.build()
    h = gprox.Handle(0)
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "section4_iterations.json")))
    printed = g["tables"]["emd_deltas_tau1"]["iters"]["512"]
    N = 512
    d0, d1 = (torch.from_numpy(a).cuda() for a in synth.delta_pair(N))
    gt = PE.ground_truth(h, "emd", N, (d0, d1), PE.emd_delta_tau(N, 1e-4), 1e-4, max_iters=20000)
    assert gt["certified"], gt
    o, _ = PE.first_below(h, "emd", N, (d0, d1), 1.0, gt["F"], [1e-2, 1e-3, 1e-4])
    got = [o[1e-2], o[1e-3], o[1e-4]]
    print("delta measures, tau = 1, 512^2:", got, "paper", printed)
    for a, b in zip(got, printed):
        assert a is not None and abs(a - b) <= 0.05 * b, (got, printed)
    h.close()
