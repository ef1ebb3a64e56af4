"""Pins for the oracle's variants: hash_crc of Fig. 3 and the self-loop-free graph of
section 4.

hash_crc is CRC-32C of the position, twice, with two initial values (Fig. 3 uses 0 and
1), the first result in the high half, reduced by the remainder.  The CRC is pinned to
published check values and to a third statement of it as polynomial division over GF(2)
written here; the self-loop-free rule (section 4: r starts at the first edge of the
current node) is pinned by its structure and by brute force over tiny graphs, where the
attachment process is enumerated on degrees rather than array positions.
"""
import itertools
import os
import random
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "crc32c_vectors.txt")
M32 = (1 << 32) - 1
M64 = (1 << 64) - 1
CASTAGNOLI = 0x11EDC6F41     # x^32 + x^28 + x^27 + x^26 + x^25 + x^23 + x^22 + x^20 + ...


def _golden():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            spec, value = line.split()
            kind, arg = spec.split(":")
            if kind == "ascii":
                data = arg.encode()
            elif kind == "zeros":
                data = bytes(int(arg))
            elif kind == "ones":
                data = b"\xff" * int(arg)
            elif kind == "inc":
                data = bytes(range(int(arg)))
            elif kind == "dec":
                data = bytes(range(int(arg) - 1, -1, -1))
            else:
                raise ValueError(spec)
            out.append((data, int(value, 0)))
    return out


def _reflect(v, bits):
    return int(format(v, f"0{bits}b")[::-1], 2)


def crc32c_by_division(init, data):
    """CRC register after `data` from `init`, as GF(2) polynomial division.

    The reflected CRC reads every byte least significant bit first; with the message bits
    in that order as the coefficients of M(x) (first bit highest) and the initial register
    I(x) (reflected), the register is (I(x) x^N + M(x) x^32) mod P(x), reflected back.
    """
    nbits = 8 * len(data)
    msg = 0
    for byte in data:
        for j in range(8):
            msg = (msg << 1) | ((byte >> j) & 1)
    a = (_reflect(init, 32) << nbits) ^ (msg << 32)
    while a.bit_length() > 32:
        a ^= CASTAGNOLI << (a.bit_length() - 33)
    return _reflect(a, 32)


def test_crc32c_matches_published_values():
    rows = _golden()
    assert len(rows) == 5
    for data, value in rows:
        assert oracle.crc32c_update(0xFFFFFFFF, data) ^ 0xFFFFFFFF == value, data[:4]
        assert crc32c_by_division(0xFFFFFFFF, data) ^ 0xFFFFFFFF == value, data[:4]


def test_crc32c_u64_takes_the_bytes_in_little_endian_order():
    for data, value in _golden():
        if len(data) != 32:
            continue
        crc = 0xFFFFFFFF
        for k in range(4):
            crc = oracle.crc32c_u64(crc, int.from_bytes(data[8 * k:8 * k + 8], "little"))
        assert crc ^ 0xFFFFFFFF == value


def test_crc32c_equals_polynomial_division():
    rnd = random.Random(11)
    for _ in range(300):
        init = rnd.getrandbits(32)
        v = rnd.getrandbits(64) >> rnd.randrange(64)
        assert oracle.crc32c_u64(init, v) == crc32c_by_division(init, v.to_bytes(8, "little"))
    for init in (0, 1, M32):
        for v in (0, 1, 2 ** 32 - 1, 2 ** 32 + 1, M64):
            assert oracle.crc32c_u64(init, v) == crc32c_by_division(init,
                                                                     v.to_bytes(8, "little"))
    assert oracle.crc32c_u64(0, 0) == 0          # linear map of zero data from zero


def test_crc32c_is_affine_in_initial_value_and_data():
    rnd = random.Random(12)
    for _ in range(200):
        a, b = rnd.getrandbits(32), rnd.getrandbits(32)
        x, y = rnd.getrandbits(64), rnd.getrandbits(64)
        assert (oracle.crc32c_u64(a ^ b, x ^ y) ^ oracle.crc32c_u64(0, 0)
                == oracle.crc32c_u64(a, x) ^ oracle.crc32c_u64(b, y))


def test_hash_crc_bits_is_fig3_for_seed_zero_and_splits_the_seed():
    rnd = random.Random(13)
    for _ in range(200):
        r = rnd.getrandbits(rnd.choice([20, 33, 41, 63])) | 1
        b = r.to_bytes(8, "little")
        fig3 = (crc32c_by_division(0, b) << 32) + crc32c_by_division(1, b)
        assert oracle.hash_crc_bits(0, r) == fig3
        seed = rnd.getrandbits(64)
        lo, hi = seed & M32, (seed >> 32) ^ 1
        assert oracle.hash_crc_bits(seed, r) == ((crc32c_by_division(lo, b) << 32)
                                                 + crc32c_by_division(hi, b))


def _splitmix_bits(seed, key):
    z = seed ^ ((key * 0x9E3779B97F4A7C15) & M64)
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_draw_reductions():
    rnd = random.Random(14)
    for _ in range(300):
        seed = rnd.getrandbits(64)
        key = rnd.getrandbits(rnd.choice([8, 31, 40, 62])) | 1
        rng = rnd.randrange(1, key + 1)
        x = oracle.draw(oracle.HASH_SPLITMIX, seed, key, rng)
        assert x == (_splitmix_bits(seed, key) * rng) >> 64 and 0 <= x < rng
        y = oracle.draw(oracle.HASH_CRC, seed, key, rng)
        assert y == oracle.hash_crc_bits(seed, key) % rng and 0 <= y < rng
        assert oracle.draw(oracle.HASH_SPLITMIX, seed, key, key) == oracle.h(seed, key)


@pytest.mark.parametrize("seed,n,d,n0", [(1, 300, 3, 0), (2, 200, 1, 4), (3, 150, 5, 6)])
def test_plain_variant_is_the_plain_array(seed, n, d, n0):
    E = oracle.bb_array_variant(seed, n, d, n0, oracle.HASH_SPLITMIX, False)
    assert np.array_equal(E, oracle.bb_array(seed, n, d, n0))


CASES = [(1, 400, 3, 2), (5, 300, 1, 3), (9, 200, 7, 8), (4, 250, 2, 5)]


@pytest.mark.parametrize("family", [oracle.HASH_SPLITMIX, oracle.HASH_CRC])
@pytest.mark.parametrize("no_loops", [False, True])
@pytest.mark.parametrize("seed,n,d,n0", CASES)
def test_variant_recomputation_equals_array_and_structure(family, no_loops, seed, n, d, n0):
    E = oracle.bb_array_variant(seed, n, d, n0, family, no_loops)
    m = oracle.num_edges(n, d, n0)
    m0 = oracle.seed_edges(n0)
    pairs = E.reshape(-1, 2)
    got = oracle.edges_range_variant(seed, n, d, n0, family, no_loops, 0, m)
    assert np.array_equal(got, pairs)
    mid = m // 3
    assert np.array_equal(oracle.edges_range_variant(seed, n, d, n0, family, no_loops, mid,
                                                     m - 1), pairs[mid:m - 1])
    i = np.arange(m0, m)
    assert np.array_equal(pairs[m0:, 0], n0 + (i - m0) // d)
    assert np.array_equal(pairs[:m0], oracle.bb_array(0, n0, 1, n0).reshape(-1, 2)[:m0])
    if no_loops:
        assert (pairs[m0:, 1] < pairs[m0:, 0]).all()
    else:
        assert (pairs[m0:, 1] <= pairs[m0:, 0]).all()
    counts = oracle.degree_count_range_variant(seed, n, d, n0, family, no_loops, 0, m, n)
    assert np.array_equal(counts, oracle.degrees_of_array(E, n))
    assert int(counts.sum()) == 2 * m
    part = oracle.degree_count_range_variant(seed, n, d, n0, family, no_loops, 0, mid, n)
    oracle.degree_count_range_variant(seed, n, d, n0, family, no_loops, mid, m, n, part)
    assert np.array_equal(part, counts)


def test_self_loops_do_occur_without_the_rule_and_the_rule_needs_a_seed_edge():
    E = oracle.bb_array_variant(3, 2000, 2, 2, oracle.HASH_CRC, False).reshape(-1, 2)
    assert (E[1:, 0] == E[1:, 1]).any()
    for n0 in (0, 1):
        with pytest.raises(ValueError):
            oracle.bb_array_variant(1, 10, 2, n0, oracle.HASH_SPLITMIX, True)
        with pytest.raises(ValueError):
            oracle.edges_range_variant(1, 10, 2, n0, oracle.HASH_CRC, True, 0, 3)
    with pytest.raises(ValueError):
        oracle.bb_array_variant(1, 10, 2, 3, 7, False)


def exact_distribution_no_loops(n, d, n0):
    """{tuple of new-edge targets: probability} of the self-loop-free process.

    Every edge of node s picks node j with probability deg(j) / (sum of degrees), the
    degrees taken over the edges that exist when s arrives (the seed clique and the
    edges of nodes < s): the draw starts at the first edge of the current node, so none
    of the node's own edges is a candidate and its d picks are independent.
    """
    deg = Counter()
    for v in range(1, n0):
        for u in range(v):
            deg[v] += 1
            deg[u] += 1
    dist = {}

    def walk(s, deg, prefix, prob):
        if s == n:
            dist[prefix] = dist.get(prefix, 0) + prob
            return
        total = sum(deg.values())
        cands = sorted((j, Fraction(w, total)) for j, w in deg.items() if w)
        for picks in itertools.product(cands, repeat=d):
            nd = Counter(deg)
            nd[s] += d
            q = Fraction(1)
            for j, pj in picks:
                nd[j] += 1
                q *= pj
            walk(s + 1, nd, prefix + tuple(j for j, _ in picks), prob * q)

    walk(n0, deg, (), Fraction(1))
    return dist


def test_exact_no_loop_distribution_by_hand():
    # n0=2: the clique is the edge (1, 0).  Node 2's single edge picks 0 or 1 with 1/2
    # each; node 3 then sees degrees {0: 1+a, 1: 1+b, 2: 1}, total 4.
    dist = exact_distribution_no_loops(4, 1, 2)
    assert dist[(0, 0)] == Fraction(1, 2) * Fraction(2, 4)
    assert dist[(0, 2)] == Fraction(1, 2) * Fraction(1, 4)
    assert dist[(1, 0)] == Fraction(1, 2) * Fraction(1, 4)
    assert sum(dist.values()) == 1 and len(dist) == 6


@pytest.mark.parametrize("n,d,n0,S", [(4, 2, 2, 60_000), (5, 1, 2, 60_000),
                                      (5, 2, 3, 100_000)])
def test_no_loop_oracle_matches_exact_distribution(n, d, n0, S):
    dist = exact_distribution_no_loops(n, d, n0)
    assert sum(dist.values()) == 1
    m0 = n0 * (n0 - 1) // 2
    seen = Counter()
    for seed in range(S):
        E = oracle.bb_array_variant(seed, n, d, n0, oracle.HASH_SPLITMIX, True)
        seen[tuple(int(x) for x in E[2 * m0 + 1::2])] += 1
    assert set(seen) <= set(dist), "oracle produced an edge list the model forbids"
    keys = sorted(dist)
    obs = np.array([seen.get(k, 0) for k in keys], dtype=float)
    exp = np.array([float(dist[k]) * S for k in keys])
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < stats.chi2.ppf(1 - 1e-6, len(keys) - 1), chi2
