"""Pins for the oracle's hash h(r) (section 2: a hash of position r into 0..r-1).

The mixed bits are pinned to published SplitMix64 outputs, the range reduction to its
closed form at powers of two, and the reduced value to its range and to uniformity.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_vectors.txt")
G = 0x9E3779B97F4A7C15
M64 = 1 << 64
G_INV = pow(G, -1, M64)


def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            s0, k, out = line.split()
            rows.append((int(s0, 0), int(k), int(out, 0)))
    return rows


def test_mixed_bits_match_published_splitmix64_outputs():
    # With seed 0 the mixed input is r*G; the k-th SplitMix64 state from s0 is s0 + k*G,
    # which is r*G for r = (s0 + k*G) * G^-1 (G is odd, so it is invertible mod 2^64).
    rows = _golden_rows()
    assert len(rows) >= 9
    for s0, k, expected in rows:
        r = ((s0 + k * G) * G_INV) % M64
        assert oracle.hash_bits(0, r) == expected, (s0, k)


def test_seed_enters_as_xor_of_r_times_gamma():
    rng = np.random.default_rng(11)
    for _ in range(200):
        seed = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        r = int(rng.integers(1, 2**62))
        r_equiv = ((seed ^ (r * G % M64)) * G_INV) % M64
        assert oracle.hash_bits(seed, r) == oracle.hash_bits(0, r_equiv)


def test_power_of_two_range_keeps_the_top_bits():
    # floor(z * 2^k / 2^64) = z >> (64 - k): multiply-shift, not a modulo.
    for seed in (0, 1, 42, 2**63 + 5):
        for k in range(0, 64):
            r = 1 << k
            z = oracle.hash_bits(seed, r)
            assert oracle.h(seed, r) == z >> (64 - k)


@pytest.mark.parametrize("r", [1, 2, 3, 5, 2**32 - 1, 2**32, 2**32 + 1, 2**41 + 1,
                               2**62 + 1, 2**63 - 1, 2**64 - 1])
def test_range_at_edge_values(r):
    for seed in range(64):
        v = oracle.h(seed, r)
        assert 0 <= v < r
    assert oracle.h(7, 1) == 0


def test_range_random_values():
    rng = np.random.default_rng(5)
    rs = rng.integers(1, 2**63, size=20000, dtype=np.int64)
    for i, r in enumerate(rs):
        r = int(r)
        assert 0 <= oracle.h(i, r) < r


@pytest.mark.parametrize("r", [3, 7, 64, 1001])
def test_uniform_over_seeds(r):
    # For a fixed position, the value over many seeds is uniform on 0..r-1 (chi^2, fixed
    # seeds so the outcome is deterministic; threshold at p = 1e-6).
    S = 200_000 if r < 100 else 500_000
    vals = np.fromiter((oracle.h(s, r) for s in range(S)), dtype=np.int64, count=S)
    counts = np.bincount(vals, minlength=r)
    expected = S / r
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < stats.chi2.ppf(1 - 1e-6, r - 1)


def test_uniform_over_positions():
    # For a fixed seed, x = h(2i+1) / (2i+1) over many i is uniform on [0, 1).
    i = np.arange(1, 200_001, dtype=np.int64)
    frac = np.array([oracle.h(3, 2 * int(k) + 1) / (2 * int(k) + 1) for k in i])
    assert stats.kstest(frac, "uniform").pvalue > 1e-6


def test_hash_equals_a_big_integer_statement():
    # a third statement of h in Python integers (the C oracle and the CUDA library are the
    # other two): SplitMix64 finaliser of seed ^ (r*G mod 2^64), then floor(z*r / 2^64)
    M = (1 << 64) - 1

    def h_big(seed, r):
        z = seed ^ ((r * G) & M)
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z ^= z >> 31
        return (z * r) >> 64

    rng = np.random.default_rng(11)
    pairs = [(int(s), int(r)) for s, r in zip(rng.integers(0, 2**63, 10_000, dtype=np.int64),
                                               rng.integers(1, 2**63, 10_000, dtype=np.int64))]
    pairs += [(s, r) for s in (0, 1, 2**64 - 1) for r in (1, 2**32 - 1, 2**32 + 1, 2**41 + 1,
                                                         2**63 - 1)]
    for s, r in pairs:
        assert oracle.h(s, r) == h_big(s, r), (s, r)
