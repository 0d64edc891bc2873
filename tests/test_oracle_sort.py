"""Pins for the oracle's greedy sort (Algorithm 1)."""
from fractions import Fraction
import itertools

import numpy as np
import pytest

from oracle import sort


def _exact_sqdist(a, b):
    return sum((Fraction(float(x)) - Fraction(float(y))) ** 2 for x, y in zip(a, b))


def _exact_greedy(P, start):
    """Algorithm 1 with exact rational distances (brute force for tiny inputs)."""
    N = len(P)
    remaining = [j for j in range(N) if j != start]
    order, i0 = [start], start
    while remaining:
        best, jmin = None, None
        for j in remaining:
            d = _exact_sqdist(P[i0], P[j])
            if best is None or d < best:
                best, jmin = d, j
        remaining.remove(jmin)
        order.append(jmin)
        i0 = jmin
    return order


@pytest.mark.parametrize("seed,N,p", [(0, 7, 5), (1, 9, 300), (2, 12, 17), (3, 6, 600)])
def test_matches_exact_rational_greedy(seed, N, p):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((N, p))
    for start in (0, N - 1):
        assert sort.greedy_sort(P, start) == _exact_greedy(P, start)


def test_canonical_sum_close_to_exact_and_order_defined():
    rng = np.random.default_rng(5)
    a, b = rng.standard_normal(1000), rng.standard_normal(1000)
    d = sort.canonical_sqdist(a, b)
    exact = float(_exact_sqdist(a, b))
    assert abs(d - exact) <= 1e-13 * exact
    # lane structure: element t goes to lane t % 256 and is added left to
    # right inside its lane; lanes are then combined pairwise.  Lane 0 holds
    # 1 + 2^-54 (rounds to 1); lane 1 holds 3 * 2^-54 exactly; their sum
    # rounds to 1 + 2^-52.  A plain left-to-right sum would give exactly 1.
    x = np.zeros(768)
    x[0] = 1.0
    x[256] = 2.0 ** -27
    x[1] = x[257] = x[513] = 2.0 ** -27
    assert sort.canonical_sqdist(x, np.zeros(768)) == 1.0 + 2.0 ** -52
    seq = 0.0
    for v in x:
        seq = seq + v * v
    assert seq == 1.0


def test_ties_go_to_lowest_index():
    base = np.array([0.0, 0.0])
    P = np.array([base, [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0], [1.0, 0.0]])
    # from 0, rows 1, 2, 3, 4 are all at distance 1: lowest index 1 wins
    order = sort.greedy_sort(P, 0)
    assert order[1] == 1
    # from row 1 the duplicate row 4 is at distance 0
    assert order[2] == 4


def test_duplicate_rows_and_permutation_property():
    rng = np.random.default_rng(9)
    P = rng.standard_normal((10, 4))
    P[7] = P[2]
    P[5] = P[2]
    for start in range(10):
        order = sort.greedy_sort(P, start)
        assert sorted(order) == list(range(10))
        assert order[0] == start
        if start == 2:
            assert order[1:3] == [5, 7]


def test_one_dimensional_parameters_follow_the_line():
    # points on a line: the greedy chain from the smallest walks up the line
    xs = np.array([3.0, -1.0, 0.5, 7.0, 2.0, -4.0])
    P = xs[:, None]
    order = sort.greedy_sort(P, int(np.argmin(xs)))
    assert list(xs[order]) == sorted(xs)


def test_edge_cases():
    assert sort.greedy_sort(np.zeros((0, 3))) == []
    assert sort.greedy_sort(np.ones((1, 3))) == [0]
    with pytest.raises(ValueError):
        sort.greedy_sort(np.array([[np.nan], [1.0]]))
    with pytest.raises(ValueError):
        sort.greedy_sort(np.ones((2, 2)), start=2)


def test_large_distances_not_stale():
    # every distance far above the paper's "e.g. 1000" initial value
    P = np.array([[0.0], [1e5], [3e5], [2e5]])
    assert sort.greedy_sort(P, 0) == [0, 1, 3, 2]
