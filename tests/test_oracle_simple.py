"""Pins of the oracle's graph without parallel edges (section 4: the targets already
generated for a node are kept in a table and a duplicate target is rejected).

Reading under test: chains follow the array without rejection; node u takes its edges in
order, and while an edge's candidate target is already one of the node's accepted targets
(and a new one exists: edge index j < reach(u)), it is redrawn over the same range as the
plain draw.  Under an ideal hash the accepted target is then node v outside the table with
probability w_v / (W - w_table), w the occurrences in the array without rejection.  The
brute-force test enumerates that process on degrees -- the with-duplicates attachment
process of section 1 drives the chains, each node's output replaces a duplicate by a draw
from the same weights restricted to nodes not yet taken -- and never touches positions, so
it does not restate the oracle's array algorithm.
"""
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle


def reach(u, n0, no_loops):
    if no_loops:
        return u
    return u if n0 == 1 else u + 1


def exact_distribution(n, d, n0, no_loops):
    """{tuple of new-edge targets: probability} of the rejection process, enumerated."""
    m0 = n0 * (n0 - 1) // 2
    m = m0 + (n - n0) * d
    degree = Counter()
    for v in range(1, n0):
        for u in range(v):
            degree[v] += 1
            degree[u] += 1
    dist = {}

    def walk(i, deg, arrival, taken, prob, targets):
        if i == m:
            key = tuple(targets)
            dist[key] = dist.get(key, 0) + prob
            return
        s = n0 + (i - m0) // d
        j = (i - m0) % d
        if j == 0:
            taken, arrival = (), Counter(deg)
        if no_loops:
            weights = arrival                      # edges of earlier nodes only
        else:
            weights = Counter(deg)
            weights[s] += 1                        # the edge's own first end point
        total = sum(weights.values())
        assert total == (2 * (m0 + (s - n0) * d) if no_loops else 2 * i + 1)
        for t0, w in sorted(weights.items()):
            if w == 0:
                continue
            nd = Counter(deg)
            nd[s] += 1
            nd[t0] += 1                            # the array keeps the first draw
            p0 = prob * Fraction(w, total)
            if j < reach(s, n0, no_loops) and t0 in taken:
                w_taken = sum(weights[x] for x in taken)
                for v, wv in sorted(weights.items()):
                    if wv and v not in taken:
                        walk(i + 1, nd, arrival, taken + (v,), p0 * Fraction(wv, total - w_taken),
                             targets + [v])
            else:
                walk(i + 1, nd, arrival, taken + (t0,), p0, targets + [t0])

    walk(m0, degree, Counter(degree), (), Fraction(1), [])
    return dist


def test_enumeration_by_hand():
    # n=2, d=2, n0=0: node 0 owns edges 0 and 1, both (0, 0) (reach(0) = 1, so the second
    # keeps its duplicate); node 1's first edge sees node 0 with weight 4 and itself with 1,
    # its second edge must take the other node.
    dist = exact_distribution(2, 2, 0, False)
    assert dist == {(0, 0, 0, 1): Fraction(4, 5), (0, 0, 1, 0): Fraction(1, 5)}


CASES = [(3, 2, 0, False, 150_000), (4, 2, 0, False, 200_000), (5, 2, 3, False, 200_000),
         (6, 2, 3, False, 200_000), (5, 2, 3, True, 100_000), (4, 3, 2, True, 100_000),
         (6, 3, 4, True, 200_000), (3, 3, 1, False, 100_000)]


@pytest.mark.parametrize("n,d,n0,no_loops,S", CASES)
def test_oracle_matches_exact_rejection_distribution(n, d, n0, no_loops, S):
    dist = exact_distribution(n, d, n0, no_loops)
    assert sum(dist.values()) == 1
    m0 = n0 * (n0 - 1) // 2
    seen = Counter()
    for seed in range(S):
        out = oracle.edges_simple(seed, n, d, n0, no_loops)
        seen[tuple(int(x) for x in out[m0:, 1])] += 1
    assert set(seen) <= set(dist), "oracle produced an edge list the process forbids"
    # bins with an expected count below 5 are pooled
    keys = sorted(dist, key=lambda k: -dist[k])
    big = [k for k in keys if float(dist[k]) * S >= 5]
    obs = [seen.get(k, 0) for k in big]
    exp = [float(dist[k]) * S for k in big]
    rest_exp = S - sum(exp)
    if rest_exp >= 5:
        obs.append(S - sum(obs))
        exp.append(rest_exp)
    obs, exp = np.array(obs, dtype=float), np.array(exp)
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < stats.chi2.ppf(1 - 1e-6, len(exp) - 1), (chi2, len(exp))


GRAPHS = [(7, 300, 4, 0, False), (8, 300, 5, 6, False), (9, 300, 4, 5, True),
          (10, 200, 3, 1, False), (11, 60, 32, 0, False), (12, 90, 32, 33, True),
          (13, 2000, 1, 0, False), (14, 500, 7, 2, True), (15, 100, 6, 1, False)]


@pytest.mark.parametrize("seed,n,d,n0,no_loops", GRAPHS)
def test_structure(seed, n, d, n0, no_loops):
    out = oracle.edges_simple(seed, n, d, n0, no_loops)
    plain = oracle.bb_array_variant(seed, n, d, n0, oracle.HASH_SPLITMIX, no_loops).reshape(-1, 2)
    m0 = n0 * (n0 - 1) // 2
    np.testing.assert_array_equal(out[:, 0], plain[:, 0])          # sources unchanged
    np.testing.assert_array_equal(out[:m0], plain[:m0])            # the seed clique too
    if no_loops:
        assert (out[m0:, 1] < out[m0:, 0]).all()
    else:
        assert (out[:, 1] <= out[:, 0]).all()
    changed = 0
    for u in range(n0, n):
        lo = m0 + (u - n0) * d
        t, p = out[lo:lo + d, 1].tolist(), plain[lo:lo + d, 1].tolist()
        k = min(d, reach(u, n0, no_loops))
        assert len(set(t[:k])) == k, u                              # no parallel edges
        assert t[k:] == p[k:], u                                    # beyond reach: plain
        # up to the first plain duplicate the node is unchanged
        first_dup = next((j for j in range(k) if p[j] in p[:j]), k)
        assert t[:first_dup] == p[:first_dup], u
        changed += t != p
    assert changed > 0 if d > 1 else changed == 0     # one edge per node: nothing to reject
    deg = np.bincount(out.ravel(), minlength=n)
    assert deg.sum() == 2 * len(out)


@pytest.mark.parametrize("seed,n,d,n0,no_loops", GRAPHS)
def test_recomputation_equals_array_on_every_split(seed, n, d, n0, no_loops):
    out = oracle.edges_simple(seed, n, d, n0, no_loops)
    m = len(out)
    np.testing.assert_array_equal(oracle.edges_range_simple(seed, n, d, n0, no_loops, 0, m), out)
    rng = np.random.default_rng(seed)
    for _ in range(6):
        a, b = sorted(int(x) for x in rng.integers(0, m + 1, 2))
        np.testing.assert_array_equal(
            oracle.edges_range_simple(seed, n, d, n0, no_loops, a, b), out[a:b])
    counts = np.zeros(n, dtype=np.uint64)
    for a, b in [(0, m // 3), (m // 3, m - 5), (m - 5, m)]:
        oracle.degree_count_range_simple(seed, n, d, n0, no_loops, a, b, n, counts)
    np.testing.assert_array_equal(counts, np.bincount(out.ravel(), minlength=n).astype(np.uint64))


def test_reach_rule_on_the_first_nodes():
    # n0 = 0: node 0 reaches only itself, so all d of its edges are (0, 0); node 1 reaches
    # nodes 0 and 1, so its first two targets are {0, 1} and the rest keep the plain draw.
    for seed in range(50):
        out = oracle.edges_simple(seed, 30, 4, 0, False)
        plain = oracle.bb_array(seed, 30, 4, 0).reshape(-1, 2)
        assert out[:4].tolist() == [[0, 0]] * 4
        assert sorted(out[4:6, 1].tolist()) == [0, 1]
        assert out[6:8, 1].tolist() == plain[6:8, 1].tolist()
        # n0 = 1: node 0 has no end point and is never drawn; node 1 reaches only itself,
        # node 2 reaches nodes 1 and 2
        out = oracle.edges_simple(seed, 30, 4, 1, False)
        plain = oracle.bb_array(seed, 30, 4, 1).reshape(-1, 2)
        assert out[:4].tolist() == [[1, 1]] * 4
        assert sorted(out[4:6, 1].tolist()) == [1, 2]
        assert out[6:8, 1].tolist() == plain[6:8, 1].tolist()


def test_invalid_parameters_are_rejected():
    with pytest.raises(ValueError):
        oracle.edges_range_simple(1, 10, 2, 1, True, 0, 4)           # no seed edge
    with pytest.raises(ValueError):
        oracle.edges_range_simple(1, 10, 2, 0, False, 5, 4)          # a > b
