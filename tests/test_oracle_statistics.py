"""Statistical pins of the oracle against what the paper and the model fix.

* Section 2 work bound: the expected number of array positions visited per edge is at
  most 2.  Under an ideal hash it has an exact recursion: for the chain started at
  r = 2j+1, the first draw is uniform on 0..2j; j+1 of the 2j+1 values are even (stop)
  and odd value 2k+1 restarts from k, so A_j = 1 + (sum_{k<j} A_k) / (2j+1).
  The oracle's mean chain length, averaged over hash seeds, must sit within 5 standard
  errors of the exact mean.
* Section 1 (scale-free): the degree distribution of this process (the LCD model of
  Bollobas, Riordan, Spencer & Tusnady 2001, which allows loops as section 2 does) has
  P(K >= k) = d(d+1) / (k(k+1)) for k >= d, a power-law tail of exponent 3.
* Fig. 2 shape: the expected degree of node j grows like d sqrt(n/j), a log-log slope
  of -1/2 over the early nodes.
"""
import numpy as np
import pytest

import oracle


def exact_mean_chain_length(m):
    """Mean over edges 0..m-1 of A_j (empty seed graph, ideal uniform hash)."""
    s = 0.0
    total = 0.0
    for j in range(m):
        a = 1.0 + s / (2 * j + 1)
        total += a
        s += a
    return total / m


def test_exact_recursion_small_values():
    # A_0 = 1 (h(1) = 0 is even); A_1 = 1 + 1/3; below 2 for every m.
    assert exact_mean_chain_length(1) == 1.0
    assert abs(exact_mean_chain_length(2) - (1 + 4 / 3) / 2) < 1e-15
    for m in (10, 1000, 100_000):
        assert exact_mean_chain_length(m) < 2.0


@pytest.mark.parametrize("m,seeds", [(1000, 400), (100_000, 60), (1_000_000, 16)])
def test_mean_chain_length_within_five_sigma_of_exact(m, seeds):
    # Chains share suffixes (a chain that reaches odd position 2k+1 continues exactly as
    # edge k's chain), so the lengths inside one graph are correlated and the spread of a
    # single graph's mean is far above sqrt(Var/m).  The expectation is over the hash, so
    # it is estimated over many seeds, with the standard error measured across seeds.
    means = []
    for seed in range(seeds):
        lens = oracle.chain_lengths(1000 + seed, m, 1, 0, 0, m)
        assert lens.min() >= 1
        means.append(lens.mean())
    means = np.array(means)
    exact = exact_mean_chain_length(m)
    se = means.std(ddof=1) / np.sqrt(seeds)
    assert abs(means.mean() - exact) <= 5 * se, (means.mean(), exact, se)
    assert means.mean() < 2.0 + 5 * se


def test_chain_lengths_are_geometric():
    # P(len >= k) ~ 2^(1-k) away from the first few edges.
    lens = oracle.chain_lengths(4, 10**6, 1, 0, 10**5, 10**6)
    for k in range(2, 9):
        p = (lens >= k).mean()
        assert abs(p - 2.0 ** (1 - k)) < 5 * np.sqrt(2.0 ** (1 - k) / lens.size) + 1e-3


@pytest.fixture(scope="module")
def degrees_1e6_d4():
    E = oracle.bb_array(1, 10**6, 4, 0)
    return oracle.degrees_of_array(E, 10**6).astype(np.int64)


def test_degree_ccdf_matches_lcd_closed_form(degrees_1e6_d4):
    d = 4
    deg = degrees_1e6_d4
    assert deg.min() >= d
    ks = np.arange(d, 200)
    emp = np.array([(deg >= k).mean() for k in ks])
    closed = d * (d + 1) / (ks * (ks + 1.0))
    assert np.abs(emp - closed).max() < 0.003


def test_degree_tail_exponent_near_three(degrees_1e6_d4):
    deg = degrees_1e6_d4
    kmin = 30
    tail = deg[deg >= kmin]
    alpha = 1 + tail.size / np.log(tail / (kmin - 0.5)).sum()   # discrete MLE (CSN 2009)
    assert 2.7 <= alpha <= 3.3, alpha


def test_degree_of_early_nodes_falls_like_inverse_sqrt():
    n, d = 2 * 10**6, 4
    deg = oracle.degrees_of_array(oracle.bb_array(7, n, d, 0), n).astype(float)
    j = np.arange(n)
    cuts = np.unique(np.logspace(np.log10(30), np.log10(3e4), 25).astype(int))
    xs = [np.log(j[a:b].mean()) for a, b in zip(cuts[:-1], cuts[1:])]
    ys = [np.log(deg[a:b].mean()) for a, b in zip(cuts[:-1], cuts[1:])]
    slope = np.polyfit(xs, ys, 1)[0]
    assert -0.55 <= slope <= -0.45, slope
