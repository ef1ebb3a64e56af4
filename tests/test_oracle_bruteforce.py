"""Brute-force pin of the oracle against preferential attachment (section 1).

For tiny graphs the exact distribution of the edge list is enumerated from the model as
section 1 states it -- each new edge of node s picks node j with probability proportional
to j's current degree, where the new edge's own first end point already counts for s
(so the weights sum to 2i+1 and self-loops are possible, section 2) -- with exact
fractions.  The oracle, run over many hash seeds, must reproduce that distribution
(chi^2 at a fixed threshold; the seeds are fixed, so the result is deterministic).
The enumeration works on degrees, not on array positions, so it does not restate the
oracle's array algorithm.
"""
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle


def exact_distribution(n, d, n0):
    """{tuple of new-edge targets: probability} by enumerating the attachment process."""
    m0 = n0 * (n0 - 1) // 2
    m = m0 + (n - n0) * d
    degree = Counter()
    for v in range(1, n0):
        for u in range(v):
            degree[v] += 1
            degree[u] += 1
    dist = {}

    def walk(i, deg, prob, targets):
        if i == m:
            dist[tuple(targets)] = dist.get(tuple(targets), 0) + prob
            return
        s = n0 + (i - m0) // d
        weights = Counter(deg)
        weights[s] += 1                    # the new edge's own first end point
        total = sum(weights.values())
        assert total == 2 * i + 1
        for j, w in sorted(weights.items()):
            if w == 0:
                continue
            nd = Counter(deg)
            nd[s] += 1
            nd[j] += 1
            walk(i + 1, nd, prob * Fraction(w, total), targets + [j])

    walk(m0, degree, Fraction(1), [])
    return dist


@pytest.mark.parametrize("n,d,n0,S", [(3, 1, 0, 100_000), (4, 1, 0, 150_000),
                                      (5, 1, 0, 200_000), (3, 2, 0, 200_000),
                                      (5, 1, 3, 100_000), (5, 2, 3, 200_000)])
def test_oracle_matches_exact_attachment_distribution(n, d, n0, S):
    dist = exact_distribution(n, d, n0)
    assert sum(dist.values()) == 1
    m0 = n0 * (n0 - 1) // 2
    seen = Counter()
    for seed in range(S):
        E = oracle.bb_array(seed, n, d, n0)
        seen[tuple(int(x) for x in E[2 * m0 + 1::2])] += 1
    assert set(seen) <= set(dist), "oracle produced an edge list the model forbids"
    keys = sorted(dist)
    obs = np.array([seen.get(k, 0) for k in keys], dtype=float)
    exp = np.array([float(dist[k]) * S for k in keys])
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < stats.chi2.ppf(1 - 1e-6, len(keys) - 1), chi2


def test_exact_distribution_small_cases_by_hand():
    # n=2, d=1: edge 0 is (0,0); edge 1 (node 1) sees node 0 with weight 2 and itself 1.
    dist = exact_distribution(2, 1, 0)
    assert dist == {(0, 0): Fraction(2, 3), (0, 1): Fraction(1, 3)}


def test_attachment_probability_is_degree_over_2i_plus_1():
    # Batagelj-Brandes lemma (section 2): given the first i edges, the target of edge i
    # is node j with probability (occurrences of j in E[0..2i]) / (2i+1).  Checked over
    # seeds for i = 4 of (n=8, d=1) by conditioning on the prefix E[0..2i].
    i = 4
    by_prefix = {}
    for seed in range(60_000):
        E = oracle.bb_array(seed, 8, 1, 0)
        key = tuple(int(x) for x in E[:2 * i + 1])
        by_prefix.setdefault(key, Counter())[int(E[2 * i + 1])] += 1
    checked = 0
    for prefix, hist in by_prefix.items():
        total = sum(hist.values())
        if total < 3000:
            continue
        counts = Counter(prefix)
        keys = sorted(counts)
        obs = np.array([hist.get(j, 0) for j in keys], dtype=float)
        exp = np.array([counts[j] / (2 * i + 1) * total for j in keys])
        assert set(hist) <= set(keys)
        chi2 = float(((obs - exp) ** 2 / exp).sum())
        assert chi2 < stats.chi2.ppf(1 - 1e-6, max(len(keys) - 1, 1))
        checked += 1
    assert checked >= 3
