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


# ------------------------------------------------------------------ large-N grouped sort (Sec. 4.1)

def test_grouped_sort_hand_derived_bisection():
    # top split on x (spread 13 > 8); each half then splits on y (spread 7 > 3)
    P = np.array([[0, 0], [10, 1], [1, 5], [11, 6], [2, 2], [12, 3], [3, 7], [13, 8]], dtype=float)
    assert sort.coordinate_groups(P, 2) == [[0, 4], [2, 6], [1, 5], [3, 7]]
    order, offs = sort.grouped_sort(P, 2)
    assert order == [0, 4, 2, 6, 1, 5, 3, 7] and offs == [0, 2, 4, 6, 8]


def test_grouped_sort_odd_sizes_put_the_smaller_half_first():
    # 5 = 2 + 3 by value, then 3 = 1 + 2
    P = np.array([[5.0], [1.0], [4.0], [2.0], [3.0]])
    assert sort.coordinate_groups(P, 2) == [[1, 3], [4], [0, 2]]
    assert sort.grouped_sort(P, 2) == ([1, 3, 4, 0, 2], [0, 2, 3, 5])


def test_grouped_sort_ties_lowest_coordinate_and_lowest_index():
    # equal spreads (3 and 3): the split is along coordinate 0
    P = np.array([[0, 3], [3, 0], [1, 2], [2, 1]], dtype=float)
    assert sort.coordinate_groups(P, 2) == [[0, 2], [1, 3]]
    # equal values along the split coordinate: index order decides
    assert sort.coordinate_groups(np.full((4, 1), 7.0), 2) == [[0, 1], [2, 3]]
    # -0.0 and +0.0 are equal values
    Z = np.array([[0.0], [-0.0], [0.0], [-0.0]])
    assert sort.coordinate_groups(Z, 2) == [[0, 1], [2, 3]]


def test_grouped_sort_one_group_is_algorithm_1():
    rng = np.random.default_rng(7)
    P = rng.standard_normal((23, 40))
    for G in (23, 100):
        order, offs = sort.grouped_sort(P, G)
        assert order == _exact_greedy(P, 0) and offs == [0, 23]


def test_grouped_sort_one_dimensional_groups_are_value_quantiles():
    rng = np.random.default_rng(8)
    v = rng.permutation(64).astype(float) * 0.5 - 3.0
    groups = sort.coordinate_groups(v[:, None], 8)
    ranks = np.argsort(v, kind="stable")
    assert groups == [sorted(ranks[8 * q:8 * q + 8].tolist()) for q in range(8)]
    order, offs = sort.grouped_sort(v[:, None], 8)
    for q, g in enumerate(groups):
        seg = order[offs[q]:offs[q + 1]]
        assert seg == [g[a] for a in _exact_greedy(v[g][:, None], 0)]


def test_grouped_sort_recovers_separated_clusters():
    rng = np.random.default_rng(9)
    centres = np.array([[0.0, 0.0], [100.0, 0.0], [0.0, 60.0], [100.0, 60.0]])
    lab = rng.permutation(np.repeat(np.arange(4), 8))
    P = centres[lab] + rng.uniform(-1, 1, size=(32, 2))
    groups = sort.coordinate_groups(P, 8)
    assert sorted(sorted(g) for g in groups) == sorted(np.flatnonzero(lab == c).tolist() for c in range(4))


@pytest.mark.parametrize("seed,N,p,G", [(0, 37, 6, 5), (1, 100, 3, 7), (2, 64, 50, 1), (3, 11, 2, 3), (4, 7, 4, 3)])
def test_grouped_sort_sizes_and_permutation(seed, N, p, G):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((N, p))
    groups = sort.coordinate_groups(P, G)
    order, offs = sort.grouped_sort(P, G)
    assert sorted(order) == list(range(N))
    if (N, G) == (7, 3):
        assert sorted(len(g) for g in groups) == [2, 2, 3]
    sizes = [len(g) for g in groups]
    assert max(sizes) <= G and sum(sizes) == N and np.diff(offs).tolist() == sizes
    # halving at every level: sets at depth d hold floor(N / 2^d) or
    # ceil(N / 2^d) systems, and no group is deeper than the first depth at
    # which every set fits
    depth = 0
    while -(-N // 2 ** depth) > G:
        depth += 1
    assert min(sizes) >= N // 2 ** depth
    for q, g in enumerate(groups):
        assert order[offs[q]] == g[0]   # each group starts at its lowest index


def test_sort_walks_a_closed_curve_of_fields():
    # fields cos(t) G1 + sin(t) G2: the distance between two of them grows
    # with |t_i - t_j| (mod 2 pi), so Algorithm 1's chain walks the curve and
    # its tour in t is short, while the input order jumps about
    from workloads import darcy2d_circle_sequence
    L, t = darcy2d_circle_sequence(14, 40, 0.2, seed=3)
    assert abs(L.reshape(40, -1).var(axis=1).mean() - 1.0) < 0.6   # GRF marginal, sigma = 1
    order = sort.greedy_sort(L.reshape(40, -1), 0)

    def tour(o):
        d = np.abs(np.diff(t[o]))
        return float(np.minimum(d, 2 * np.pi - d).sum())

    assert tour(order) <= 4 * np.pi
    assert tour(list(range(40))) > 3 * tour(order)


def test_convdiff_keys_are_standardised():
    # the z-scores have mean 0 and variance 1 under the drawing distributions,
    # so nu (range 0.09) weighs as much as beta (range 100) in the distance
    from workloads import convdiff2d_sequence, convdiff_keys
    nu, beta, _ = convdiff2d_sequence(4, 20000, seed=11)
    K = convdiff_keys(nu, beta)
    np.testing.assert_allclose(K.mean(axis=0), 0.0, atol=0.03)
    np.testing.assert_allclose(K.std(axis=0), 1.0, atol=0.03)
    # closed form at the ends of the nu range: +-sqrt(3)
    K2 = convdiff_keys(np.array([0.01, 0.1]), np.zeros((2, 2)))
    np.testing.assert_allclose(K2[:, 0], [-np.sqrt(3.0), np.sqrt(3.0)], rtol=1e-12)
