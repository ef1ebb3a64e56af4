"""GPU side of section 2's work bound: the device's chain lengths (draws per edge) equal the
oracle's edge for edge, and their mean over seeds lies within 5 standard errors of the
exact expectation A_j = 1 + S_j/(2j+1), S_{j+1} = S_j + A_j (the recursion the oracle's
statistics test pins)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1602_07106_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BINS = 64


def _hist(ba, seed, n, d, n0, a, b, bins=BINS):
    h = torch.full((bins,), 5, dtype=torch.int64, device="cuda")
    ba.ba_chain_lengths(seed, n, d, n0, a, b, bins, h)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.uint64)


def _want(lens, bins=BINS):
    return np.bincount(np.minimum(lens.astype(np.int64), bins - 1), minlength=bins).astype(np.uint64)


@pytest.mark.parametrize("seed,n,d,n0,a,b", [
    (1, 10**6, 4, 0, 0, 4 * 10**6), (3, 20_000, 7, 8, 0, 28 + 19_992 * 7),
    (5, 2**29, 16, 0, 2**33 - 300_000, 2**33), (7, 10**10, 100, 0, 10**12 - 200_000, 10**12),
    (9, 50, 40, 41, 0, 820 + 9 * 40)])
def test_histogram_equals_oracle_edge_for_edge(ba, seed, n, d, n0, a, b):
    np.testing.assert_array_equal(_hist(ba, seed, n, d, n0, a, b),
                                  _want(oracle.chain_lengths(seed, n, d, n0, a, b)))


def test_clamped_last_bin_and_accumulate(ba):
    lens = oracle.chain_lengths(11, 10**5, 3, 0, 0, 3 * 10**5)
    np.testing.assert_array_equal(_hist(ba, 11, 10**5, 3, 0, 0, 3 * 10**5, bins=3), _want(lens, 3))
    h = torch.zeros(BINS, dtype=torch.int64, device="cuda")
    ba.ba_chain_lengths(11, 10**5, 3, 0, 0, 10**5, BINS, h)
    ba.ba_chain_lengths(11, 10**5, 3, 0, 10**5, 3 * 10**5, BINS, h, accumulate=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(h.cpu().numpy().astype(np.uint64), _want(lens))


def _exact_mean(m):
    # A_j = E[draws | r = 2j+1] = 1 + S_j / (2j+1), S_{j+1} = S_j + A_j, S_0 = 0
    s, total = 0.0, 0.0
    for j in range(m):
        a = 1.0 + s / (2 * j + 1)
        total += a
        s += a
    return total / m


@pytest.mark.parametrize("m,seeds", [(10**5, 60), (10**6, 24)])
def test_device_mean_within_five_sigma_of_exact(ba, m, seeds):
    ks = np.arange(BINS, dtype=np.float64)
    means = [float((_hist(ba, 2000 + s, m, 1, 0, 0, m) * ks).sum() / m) for s in range(seeds)]
    means = np.array(means)
    se = means.std(ddof=1) / np.sqrt(seeds)
    assert abs(means.mean() - _exact_mean(m)) <= 5 * se, (means.mean(), _exact_mean(m), se)


def test_large_workload_mean_near_two(ba):
    # 2^31 edges of the large workload: the mean sits near the bound 2 (one graph's mean
    # spreads by a few 10^-3 across seeds, far more than sqrt(Var/m): chains share suffixes)
    g = W.PLAIN_LARGE
    h = _hist(ba, g.seed, g.n, g.d, 0, 0, g.m).astype(np.float64)
    assert h.sum() == g.m and h[-1] == 0
    mean = (h * np.arange(BINS)).sum() / g.m
    assert 1.97 < mean < 2.03, mean
