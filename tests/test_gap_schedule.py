"""Host logic of the adaptive gap-check schedule (gap_every = 0), CPU only.

The schedule fits the relative gap's decay between two checks as
g = c n^-a and runs half the iterations the fit predicts to the tolerance,
as a chunk of 10 * 2^j <= 320.  Checked against the closed form of that
rule on exact power laws, its bounds, and the fallbacks (no previous check,
no decrease, already converged).
"""
import math

import pytest

from paper_1805_09453_gb300 import gprox


def _rule(n_prev, g_prev, n, g, tol):
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


def test_close_to_target_takes_the_shortest_chunk():
    # g ~ 1/n: from 2e-5 at n = 1000 the tolerance 1e-5 is 1000 iterations away -> half = 500 -> 320;
    # from 1.1e-5 at n = 1000 it is 100 away -> half = 50 -> 40
    assert gprox.gap_schedule_next(500, 4e-5, 1000, 2e-5, 1e-5) == 320
    assert gprox.gap_schedule_next(500, 2.2e-5, 1000, 1.1e-5, 1e-5) == 40
    assert gprox.gap_schedule_next(990, 1.0101e-5, 1000, 1.0001e-5, 1e-5) == 10


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
