"""Greedy nearest-neighbour sort of a sequence of systems (oracle).

Follows Algorithm 1 (Sec. 4.1): start from the first system, then N-1 times
scan the systems not yet placed in ascending index order and append the one
whose parameter matrix is nearest (Frobenius norm of the difference) to the
last placed one, keeping the first strictly smaller distance.

Readings:
  * the running minimum starts at +inf (the paper's "e.g. 1000" would keep a
    stale index once every distance exceeds 1000);
  * the scan order is ascending index, so ties go to the lowest index;
  * the start index is a parameter (0 = the paper's system 1);
  * the parameter matrix is compared as its flattened float64 array; squared
    distances are compared (monotone in the norm, no square root rounding);
  * the squared distance is summed in one fixed order, so that any two
    implementations that follow it agree bit for bit: element t goes to lane
    t mod 256; each lane adds its squares left to right (separate multiply
    and add, no fused multiply-add); the 256 lane sums are then added
    pairwise, lane l with lane l + half, for half = 128, 64, ..., 1.

Large N (the paragraph after Algorithm 1 in Sec. 4.1): divide the systems
into groups of bounded size by their coordinates, run Algorithm 1 inside each
group, and concatenate the groups' orders.  Readings:
  * "by their coordinates" is recursive coordinate bisection: a set of more
    than G systems is split along the coordinate (entry of the flattened
    parameter array) whose spread max - min over the set is largest (the
    lowest coordinate on ties), at the median: with the set ordered by
    (value of that coordinate, index), the first floor(s/2) go to the first
    half and the rest to the second; sets of at most G systems are groups;
  * groups are concatenated in the order of the recursion, first half first;
  * inside a group, Algorithm 1 scans the group's systems in ascending index
    order and starts from the group's lowest index.

Pins: brute force with exact rational distances on small inputs; hand-made
ties; permutation and start properties; hand-derived bisections; the
grouped order with G >= N equals Algorithm 1's.
"""
import numpy as np

LANES = 256


def canonical_sqdist_many(P_rows, p_ref):
    """Squared distances of each row of P_rows to p_ref, in the fixed order above."""
    P_rows = np.atleast_2d(np.asarray(P_rows, dtype=np.float64))
    p_ref = np.asarray(p_ref, dtype=np.float64).reshape(-1)
    R, plen = P_rows.shape
    T = (plen + LANES - 1) // LANES
    d = np.zeros((R, T * LANES))
    d[:, :plen] = P_rows - p_ref[None, :]
    sq = (d * d).reshape(R, T, LANES)
    s = np.zeros((R, LANES))
    for t in range(T):
        s = s + sq[:, t, :]
    half = LANES // 2
    while half >= 1:
        s = s[:, :half] + s[:, half:2 * half]
        half //= 2
    return s[:, 0]


def canonical_sqdist(a, b):
    """Squared Frobenius distance of two parameter arrays in the fixed order."""
    return float(canonical_sqdist_many(np.asarray(a).reshape(1, -1), b)[0])


def greedy_sort(P, start=0):
    """Algorithm 1: the order in which to solve the N systems.

    P      (N, p) float64: row i is the flattened parameter matrix of system i
    start  index of the first system
    Returns a list of N distinct indices beginning with `start`.
    """
    P = np.asarray(P, dtype=np.float64)
    N = P.shape[0]
    if N == 0:
        return []
    if not (0 <= start < N):
        raise ValueError("start out of range")
    if not np.all(np.isfinite(P)):
        raise ValueError("non-finite parameters")
    remaining = list(range(N))
    remaining.remove(start)
    order = [start]
    i0 = start
    for _ in range(N - 1):
        dists = canonical_sqdist_many(P[remaining], P[i0])
        best = np.inf
        jmin = -1
        for pos, j in enumerate(remaining):
            if dists[pos] < best:
                best = dists[pos]
                jmin = j
        remaining.remove(jmin)
        order.append(jmin)
        i0 = jmin
    return order


def coordinate_groups(P, group_max):
    """Groups of the large-N sort (Sec. 4.1): recursive coordinate bisection.

    P          (N, p) float64
    group_max  G >= 1, the largest group size
    Returns a list of groups, each a list of indices in ascending order, in
    concatenation order.
    """
    P = np.asarray(P, dtype=np.float64)
    N = P.shape[0]
    if group_max < 1:
        raise ValueError("group_max < 1")
    if not np.all(np.isfinite(P)):
        raise ValueError("non-finite parameters")

    def split(members):
        if len(members) <= group_max:
            return [sorted(members)]
        X = P[members]
        spread = X.max(axis=0) - X.min(axis=0)
        c = int(np.argmax(spread))          # first maximum: lowest coordinate on ties
        ordered = sorted(members, key=lambda i: (P[i, c], i))
        h = len(members) // 2
        return split(ordered[:h]) + split(ordered[h:])

    return split(list(range(N))) if N else []


def grouped_sort(P, group_max):
    """The large-N order (Sec. 4.1): Algorithm 1 inside each coordinate group.

    Returns (order, offsets): the concatenated order (N indices) and the
    ngroups + 1 offsets of the groups in it.
    """
    P = np.asarray(P, dtype=np.float64)
    order, offsets = [], [0]
    for g in coordinate_groups(P, group_max):
        local = greedy_sort(P[g], start=0)
        order.extend(g[a] for a in local)
        offsets.append(len(order))
    return order, offsets
