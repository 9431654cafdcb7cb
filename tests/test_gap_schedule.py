"""Host logic of the adaptive gap-check schedule (gap_every = 0), CPU only.

While the relative gap is above 3 x the tolerance, the schedule fits its
decay between two checks as g = c n^-a and runs half the iterations the fit
predicts to the tolerance, as a chunk of 10 * 2^j <= 320; within 3 x, and
in the fallbacks (no previous check, no decrease, converged), 10.  Checked
against the closed form of that rule on exact power laws and its bounds.
"""
import math

import pytest

from paper_1805_09453_gb300 import gprox


def _rule(n_prev, g_prev, n, g, tol):
    if g <= 3 * tol:
        return 10
    a = math.log(g_prev / g) / math.log(n / n_prev)
    half = 0.5 * (n * (g / tol) ** (1.0 / a) - n)
    k = 10
    while 2 * k <= 320 and 2 * k <= half:
        k *= 2
    return k


@pytest.mark.parametrize("a", [0.5, 1.0, 2.0])
@pytest.mark.parametrize("n", [20, 100, 1000])
def test_power_law_decay_matches_closed_form(a, n):
    c, tol = 1.0, 1e-5
    g_prev, g = c * (n / 2) ** -a, c * n ** -a
    k = gprox.gap_schedule_next(n // 2, g_prev, n, g, tol)
    assert k == _rule(n // 2, g_prev, n, g, tol)
    assert k in (10, 20, 40, 80, 160, 320)
    # never past the predicted crossing: the chunk is at most half the distance (or the minimum 10)
    n_star = (c / tol) ** (1.0 / a)
    assert k == 10 or n + k <= n + 0.5 * (n_star - n) + 1e-9


def test_far_from_target_takes_the_longest_chunk():
    assert gprox.gap_schedule_next(100, 1e-1, 200, 5e-2, 1e-5) == 320


def test_chunk_halves_towards_the_predicted_crossing():
    # g ~ 1/n: from 8e-5 at n = 1000 the tolerance 1e-5 is 7000 iterations away -> half 3500 -> 320;
    # from 4e-5 at n = 1000 it is 3000 away -> half 1500 -> 320; g ~ n^-4 from 4e-5 at n = 1000:
    # 1000 (4^(1/4) - 1) = 414 away -> half 207 -> 160
    assert gprox.gap_schedule_next(500, 16e-5, 1000, 8e-5, 1e-5) == 320
    assert gprox.gap_schedule_next(500, 8e-5, 1000, 4e-5, 1e-5) == 320
    assert gprox.gap_schedule_next(500, 4e-5 * 16, 1000, 4e-5, 1e-5) == 160


def test_within_three_tolerances_checks_every_ten():
    assert gprox.gap_schedule_next(500, 6e-5, 1000, 3e-5, 1e-5) == 10
    assert gprox.gap_schedule_next(500, 2.2e-5, 1000, 1.1e-5, 1e-5) == 10


@pytest.mark.parametrize("args", [
    (-1, 0.0, 10, 1e-2, 1e-5),      # no previous check
    (10, 1e-3, 20, 2e-3, 1e-5),     # gap grew
    (10, 1e-3, 20, 1e-3, 1e-5),     # no decrease
    (10, 1e-3, 20, 1e-6, 1e-5),     # converged
    (10, 1e-3, 20, 1e-4, 0.0),      # no tolerance
    (20, 1e-3, 20, 1e-4, 1e-5),     # same iteration
])
def test_fallback_is_ten(args):
    assert gprox.gap_schedule_next(*args) == 10
