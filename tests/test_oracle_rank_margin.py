"""Pin of the oracle's rank-decision margin (``oracle.update.rank_margin``).

The GPU parity tests compare ranks only where the oracle's rank decision is
not close to flipping, so the margin decides which rank checks run.  Its
definition here is the brute-force one: the rank rule of Section 4 (reading:
keep the smallest r with sum_{i>=r} sigma_i^2 <= (eps/2)^2) is re-evaluated
with the threshold scaled by a factor f, and the margin is the distance of
the nearest f at which the chosen rank changes, min(f_up - 1, 1 - f_down),
found by bisection on the rule itself (no tail sums are formed here).  A
rank that no positive threshold changes has an infinite margin; margins are
compared up to 1 (the gate is 1e-6).
"""
import math

import numpy as np
import pytest

from oracle.update import rank_margin, rank_rule


def _rank_at(sigma, eps, f):
    # threshold (eps/2)^2 scaled by f  <=>  eps scaled by sqrt(f)
    return rank_rule(sigma, eps * math.sqrt(f))


def _flip_factor(sigma, eps, r, lo, hi):
    """Bisection for the boundary factor between lo (rank r) and hi (rank
    different from r)."""
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _rank_at(sigma, eps, mid) == r:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def brute_margin(sigma, eps):
    r = rank_rule(sigma, eps)
    up, down = math.inf, math.inf
    # larger thresholds: rank can only fall; look for the first factor that
    # changes it (none if the rank is 0 already)
    f = 2.0
    while f < 1e40 and _rank_at(sigma, eps, f) == r:
        f *= 2.0
    if _rank_at(sigma, eps, f) != r:
        up = _flip_factor(sigma, eps, r, 1.0, f) - 1.0
    # smaller thresholds: rank can only grow
    f = 0.5
    while f > 1e-300 and _rank_at(sigma, eps, f) == r:
        f *= 0.5
    if _rank_at(sigma, eps, f) != r:
        down = 1.0 - _flip_factor(sigma, eps, r, 1.0, f)
    return min(up, down)


def _cases():
    rng = np.random.default_rng(20140520)
    out = []
    for n in (1, 2, 3, 5, 8, 13, 24, 32):
        for _ in range(6):
            s = np.sort(np.abs(rng.standard_normal(n)) * 10.0 ** rng.uniform(-3, 1, n))[::-1]
            # thresholds placed among the tail sums, and far above / below
            tails = np.cumsum((s ** 2)[::-1])[::-1]
            pick = tails[rng.integers(0, n)] * 10.0 ** rng.uniform(-0.5, 0.5)
            for thr in (pick, tails[0] * 3.0, tails[-1] * 0.1):
                out.append((s.copy(), 2.0 * math.sqrt(thr)))
    # graded spectra with a clear gap, the benchmark's shape
    for k in (4, 16, 24):
        s = np.concatenate([np.linspace(2.0, 1.0, k), 1e-6 * np.ones(8)])
        out.append((s, 1e-4))
        out.append((s, 1e-8))
    return out


@pytest.mark.parametrize("idx", range(len(_cases())))
def test_margin_equals_brute_force(idx):
    sigma, eps = _cases()[idx]
    r = rank_rule(sigma, eps)
    # margins of 1 and above all mean "far from flipping"; the oracle caps a
    # side that no threshold reaches at 1, so compare min(margin, 1)
    got = min(rank_margin(sigma, eps, r), 1.0)
    want = min(brute_margin(sigma, eps), 1.0)
    assert abs(got - want) <= 1e-9, (got, want, r)


def test_margin_special_cases():
    # every singular value zero: no positive threshold changes rank 0
    assert math.isinf(rank_margin(np.zeros(5), 0.1, 0))
    # eps = 0 keeps every nonzero value and never flips
    s = np.array([3.0, 2.0, 1.0])
    assert rank_rule(s, 0.0) == 3 and math.isinf(rank_margin(s, 0.0, 3))
    # threshold exactly between the two adjacent tails, by hand:
    # tails (from r): r=2 -> 1, r=1 -> 5; thr = 3 -> margin = 2/3 both ways
    s = np.array([3.0, 2.0, 1.0])
    eps = 2.0 * math.sqrt(3.0)
    assert rank_rule(s, eps) == 2
    assert abs(rank_margin(s, eps, 2) - 2.0 / 3.0) < 1e-15


def test_margin_gate_is_not_always_closed():
    # on the benchmark-shaped spectra the gate (margin >= 1e-6) lets the
    # rank check through; on a threshold placed on a tail sum it does not
    s = np.concatenate([np.linspace(2.0, 1.0, 24), 1e-6 * np.ones(8)])
    assert rank_margin(s, 1e-4, rank_rule(s, 1e-4)) >= 1e-6
    tails = np.cumsum((s ** 2)[::-1])[::-1]
    eps = 2.0 * math.sqrt(tails[20] * (1 + 1e-9))
    assert rank_margin(s, eps, rank_rule(s, eps)) < 1e-6
