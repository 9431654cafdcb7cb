"""Host side of the paper-experiment driver (section 4), CPU only: the step
rules against the paper's own statements about them, and the inputs.

Section 4.2 states, for the delta-measure rule
tau = min(sqrt(1/(eps |log eps|)), 2 M^(1/4)): at eps = 1e-2 the first term
is the smaller on every grid (512^2 .. 4096^2); at 1e-3 it is larger on
512^2, about equal on 1024^2 and smaller on 2048^2 and 4096^2; at 1e-4 the
second term is the smaller on every grid.  Those statements hold for M = N,
the points per side, and are the pins of that form of the rule below; with
M = N^2, the number of grid points the paper's definition names (the
driver's default, which reproduces the paper's delta table more closely),
the second term is the larger everywhere at these tolerances.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1805_09453_gb300 import paper_experiments as PE
from paper_1805_09453_gb300 import synth

SIZES = [512, 1024, 2048, 4096]


def _terms(N, eps):
    return math.sqrt(1.0 / (eps * abs(math.log(eps)))), 2.0 * N ** 0.25


def test_delta_rule_eps_1e2_first_term_everywhere():
    for N in SIZES:
        a, b = _terms(N, 1e-2)
        assert a < b and PE.emd_delta_tau(N, 1e-2, m_points=False) == a


def test_delta_rule_eps_1e3_crosses_at_1024():
    a, b = _terms(512, 1e-3)
    assert a > b and PE.emd_delta_tau(512, 1e-3, m_points=False) == b
    a, b = _terms(1024, 1e-3)
    assert abs(a - b) / b < 0.1  # "approximately equal"
    for N in (2048, 4096):
        a, b = _terms(N, 1e-3)
        assert a < b and PE.emd_delta_tau(N, 1e-3, m_points=False) == a


def test_delta_rule_eps_1e4_grid_term_everywhere():
    for N in SIZES:
        a, b = _terms(N, 1e-4)
        assert b < a and PE.emd_delta_tau(N, 1e-4, m_points=False) == b


def test_delta_rule_with_grid_points():
    # M = N^2: 2 M^(1/4) = 2 sqrt(N) >= 45 exceeds sqrt(1/(eps |log eps|)) (<= 33) for eps >= 1e-4
    for N in SIZES:
        for eps in (1e-2, 1e-3, 1e-4):
            assert PE.emd_delta_tau(N, eps) == pytest.approx(math.sqrt(1.0 / (eps * abs(math.log(eps)))))


@pytest.mark.parametrize("lam,eps", [(10.0, 1e-2), (20.0, 1e-3)])
def test_rof_rule_forms(lam, eps):
    stats = (1.5, 30.0, 0.2)
    free = math.sqrt(lam) * 1.5 / math.sqrt(eps)
    assert PE.rof_tau(stats, lam, eps, grid_dependent=False) == pytest.approx(free, rel=1e-15)
    assert PE.rof_tau(stats, lam, eps) == pytest.approx(min(free, 30.0), rel=1e-15)


def test_inputs_of_the_experiments():
    N = 64
    I = synth.disc_image(N)
    assert set(np.unique(I)) == {0.0, 1.0}
    assert abs(I.mean() - math.pi / 16) < 0.01  # disc of radius 1/4
    f0, f1 = synth.translated_discs(N)
    assert abs(f0.astype(np.float64).sum() / N ** 2 - 1) < 1e-6 and abs(f1.astype(np.float64).sum() / N ** 2 - 1) < 1e-6
    # f1 is f0 translated by (1/4, 1/4): N/4 cells along both axes
    np.testing.assert_array_equal(np.roll(f0, (N // 4, N // 4), axis=(0, 1)), f1)
    d0, d1 = synth.delta_pair(N)
    assert np.count_nonzero(d0) == 1 and d0.max() == N * N and np.count_nonzero(d1) == 1
    np.testing.assert_array_equal(np.roll(d0, (N // 4, N // 4), axis=(0, 1)), d1)


def test_paper_tables_match_the_cited_fixture():
    """The experiments module's copy of the paper's section-4 iteration counts equals the
    cited fixture tests/golden/section4_iterations.json."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "section4_iterations.json")))
    assert set(g["tables"]) == set(PE.PAPER_TABLES)
    for name, t in g["tables"].items():
        assert t["eps"] == PE.PAPER_TABLES[name]["eps"]
        assert {int(k): v for k, v in t["iters"].items()} == PE.PAPER_TABLES[name]["iters"], name


def test_paper_tables_are_consistent():
    for name, t in PE.PAPER_TABLES.items():
        for N, row in t["iters"].items():
            assert len(row) == len(t["eps"]), name
            vals = [v for v in row if v is not None]
            assert vals == sorted(vals), (name, N)  # tighter tolerance, more iterations


class _FakeState:
    """Scripted objective sequence: after k steps the primal is P(k), the dual D(k)."""

    def __init__(self, P, D):
        self.P, self.D, self.k = P, D, 0

    def step(self, n):
        self.k += n

    def gap(self):
        return {"primal": self.P(self.k), "dual": self.D(self.k)}

    def close(self):
        pass


def test_protocol_counts_first_iterate_below_each_tolerance(monkeypatch):
    # F(u_n) - F* = 1/n  ->  first n with 1/n < eps is floor(1/eps) + 1 (tolerances off the reciprocals)
    monkeypatch.setattr(PE, "_state", lambda *a, **k: _FakeState(lambda n: 2.0 + 1.0 / n, lambda n: 2.0 - 1.0 / n))
    out, _ = PE.first_below(None, "emd", 8, None, 1.0, 2.0, [0.15, 1.5e-2, 3e-3])
    assert out == {0.15: 7, 1.5e-2: 67, 3e-3: 334}
    out, _ = PE.first_below(None, "emd", 8, None, 1.0, 2.0, [1e-4], max_iters=50)
    assert out == {1e-4: None}


def test_ground_truth_certified_by_the_gap(monkeypatch):
    # gap 2/n: below eps/10 = 1.5e-4 first at n > 13333.3, checked in chunks of 50 -> 13350
    monkeypatch.setattr(PE, "_state", lambda *a, **k: _FakeState(lambda n: 2.0 + 1.0 / n, lambda n: 2.0 - 1.0 / n))
    gt = PE.ground_truth(None, "emd", 8, None, 1.0, 1.5e-3)
    assert gt["certified"] and gt["iters"] == 13350 and abs(gt["F"] - (2.0 + 1.0 / 13350)) < 1e-15
    gt = PE.ground_truth(None, "emd", 8, None, 1.0, 1e-3, max_iters=1000)
    assert not gt["certified"] and gt["iters"] == 1000 and abs(gt["F"] - 2.001) < 1e-12  # smallest primal seen


@pytest.mark.parametrize("N,lam,eps", [(32, 8.0, 1e-3), (64, 20.0, 1e-2), (48, 0.5, 1e-3)])
def test_rof_step_rule_in_the_library_matches_the_oracle(N, lam, eps):
    """gp_rof_step_tau (host only) with both flags is rof_solve's rule; on the
    oracle's image norms it gives the oracle's tau, and without the flags the
    plain section-4.1 rule sqrt(lam) ||I||_TV / sqrt(eps)."""
    from oracle import gprox_oracle as O
    from paper_1805_09453_gb300 import gprox

    I = synth.rof_image(N, N).astype(np.float64)
    tau, _, st = O.rof_step_rule(I, lam, eps)
    stats = (st["tv"], st["grad_l2"], st["fid"] / (0.5 * lam))
    got = gprox.rof_step_tau(stats, lam, eps, grid_cap=True, fidelity_bound=True)
    assert abs(got - tau) <= 1e-14 * tau
    plain = gprox.rof_step_tau(stats, lam, eps, grid_cap=False)
    assert abs(plain - math.sqrt(lam) * st["tv"] / math.sqrt(eps)) <= 1e-14 * plain
    assert gprox.rof_step_tau((0.0, 0.0, 0.0), lam, eps) == 1.0  # a constant image
    assert math.isnan(gprox.rof_step_tau(stats, -1.0, eps))
    assert math.isnan(gprox.emd_delta_tau(0, eps))
