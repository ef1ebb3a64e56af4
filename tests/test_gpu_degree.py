"""GPU parity of the streaming degree count (section 3) against the oracle; bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from oracle import parallel as opar
from paper_1602_07106_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _counts(ba, seed, n, d, n0, a, b, limit, accumulate=None):
    c = torch.zeros(limit, dtype=torch.int64, device="cuda") if accumulate is None else accumulate
    ba.ba_degree_count_range(seed, n, d, n0, a, b, limit, c, 0 if accumulate is None else 1)
    torch.cuda.synchronize()
    return c


def test_small_workload_degrees_bit_exact(ba):
    g = W.PLAIN_SMALL
    E = oracle.bb_array(g.seed, g.n, g.d, 0)
    for limit in (1, 1000, W.DEGREE_NODE_LIMIT, g.n, g.n + 7):
        c = torch.empty(limit, dtype=torch.int64, device="cuda")
        ba.ba_degree_count(g.seed, g.n, g.d, limit, c)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(c.cpu().numpy().astype(np.uint64),
                                      oracle.degrees_of_array(E, limit))


CASES = [(3, 5000, 3, 0), (5, 20_000, 1, 0), (7, 3000, 4, 5), (9, 500, 32, 33), (11, 200, 5, 1),
         (13, 40, 3, 40), (15, 100_000, 7, 9)]


@pytest.mark.parametrize("seed,n,d,n0", CASES)
def test_ranges_and_accumulation_match_oracle(ba, seed, n, d, n0):
    m = oracle.num_edges(n, d, n0)
    m0 = n0 * (n0 - 1) // 2
    cuts = sorted({c for c in (0, 1, m0 // 2, m0, m0 + 1, m // 3, m // 2 + 7, m - 1, m) if c <= m})
    for limit in (1, 17, n, n + 3):
        acc = torch.zeros(limit, dtype=torch.int64, device="cuda")
        for a, b in zip(cuts[:-1], cuts[1:]):
            part = _counts(ba, seed, n, d, n0, a, b, limit)
            np.testing.assert_array_equal(part.cpu().numpy().astype(np.uint64),
                                          oracle.degree_count_range(seed, n, d, n0, a, b, limit))
            _counts(ba, seed, n, d, n0, a, b, limit, accumulate=acc)
        np.testing.assert_array_equal(acc.cpu().numpy().astype(np.uint64),
                                      oracle.degree_count_range(seed, n, d, n0, 0, m, limit))


SHAPES = [
    {"refill": 0, "block": 256, "ctas_per_sm": 8},
    {"refill": 1, "block": 256, "ctas_per_sm": 2, "tile": 64, "hist_bins": 0},
    {"refill": 1, "block": 512, "ctas_per_sm": 2, "tile": 512, "hist_bins": 1000},
    {"refill": 1, "block": 512, "ctas_per_sm": 2, "tile": 512, "hist_bins": 24576, "hist_agg": 1},
    {"refill": 1, "block": 128, "ctas_per_sm": 8, "tile": 256, "hist_bins": 64, "hist_agg": 1},
    {"refill": 1, "block": 1024, "ctas_per_sm": 1, "tile": 1024, "hist_bins": 20480},
    {"refill": 1, "block": 32, "ctas_per_sm": 4, "tile": 4096, "hist_bins": 7},
    {"refill": 1, "block": 256, "ctas_per_sm": 2, "tile": 512, "hist_bins": 4096, "chains": 2},
    {"refill": 1, "block": 512, "ctas_per_sm": 1, "tile": 16384, "hist_bins": 8192, "hist_agg": 1,
     "chains": 2},
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()))
def test_counts_do_not_depend_on_launch_shape(ba, shape):
    seed, n, d = 41, 400_000, 5
    want = opar.degree_count_range(seed, n, d, 0, 0, n * d, 60_000)
    try:
        ba.ba_set_tuning(ba.BA_KIND_DEGREE, shape)
        got = _counts(ba, seed, n, d, 0, 0, n * d, 60_000)
    finally:
        ba.ba_set_tuning(ba.BA_KIND_DEGREE, None)
    np.testing.assert_array_equal(got.cpu().numpy().astype(np.uint64), want)


SCHEDULERS = [None, {"refill": 1, "chains": 1},
              {"refill": 1, "chains": 2, "block": 128, "tile": 256, "hist_bins": 300}]


@pytest.mark.parametrize("shape", SCHEDULERS, ids=str)
def test_64_bit_positions(ba, shape):
    n, d = 2**29, 16
    m = n * d
    a, b = m - 400_000, m
    try:
        if shape is not None:
            ba.ba_set_tuning(ba.BA_KIND_DEGREE, shape)
        np.testing.assert_array_equal(
            _counts(ba, 77, n, d, 0, a, b, 5000).cpu().numpy().astype(np.uint64),
            opar.degree_count_range(77, n, d, 0, a, b, 5000))
    finally:
        ba.ba_set_tuning(ba.BA_KIND_DEGREE, None)


@pytest.mark.parametrize("shape", SCHEDULERS, ids=str)
@pytest.mark.parametrize("seed,n,d,n0,a,b,limit", [
    (43, 300_000, 7, 8, 0, 28 + 299_992 * 7, 5000),           # seed clique, whole graph
    (45, 200_000, 3, 40, 500, 780 + 199_960 * 3, 70),         # clique of 40, range inside
    (47, 2**28, 24, 25, 2**31 - 300, 2**31 + 90_000, 3000),   # 64-bit positions + clique
])
def test_seed_cliques_and_ranges_across_schedulers(ba, shape, seed, n, d, n0, a, b, limit):
    try:
        if shape is not None:
            ba.ba_set_tuning(ba.BA_KIND_DEGREE, shape)
        got = _counts(ba, seed, n, d, n0, a, b, limit)
    finally:
        ba.ba_set_tuning(ba.BA_KIND_DEGREE, None)
    np.testing.assert_array_equal(got.cpu().numpy().astype(np.uint64),
                                  opar.degree_count_range(seed, n, d, n0, a, b, limit))


@pytest.mark.parametrize("shape", SCHEDULERS, ids=str)
def test_positions_near_2_to_the_61(ba, shape):
    seed, n, d = 97, 2**40, 2**20
    m = n * d
    a, b = m - 30_000, m
    try:
        if shape is not None:
            ba.ba_set_tuning(ba.BA_KIND_DEGREE, shape)
        got = _counts(ba, seed, n, d, 0, a, b, 1000)
    finally:
        ba.ba_set_tuning(ba.BA_KIND_DEGREE, None)
    np.testing.assert_array_equal(got.cpu().numpy().astype(np.uint64),
                                  oracle.degree_count_range(seed, n, d, 0, a, b, 1000))


def test_large_workload_prefix_partition_and_degree_sum(ba):
    g = W.PLAIN_LARGE
    L = W.DEGREE_NODE_LIMIT
    full = torch.empty(L, dtype=torch.int64, device="cuda")
    ba.ba_degree_count(g.seed, g.n, g.d, L, full)
    a = 10**7
    np.testing.assert_array_equal(_counts(ba, g.seed, g.n, g.d, 0, 0, a, L).cpu().numpy().astype(np.uint64),
                                  opar.degree_count_range(g.seed, g.n, g.d, 0, 0, a, L))
    split = _counts(ba, g.seed, g.n, g.d, 0, 0, 2**30 + 12345, L)
    _counts(ba, g.seed, g.n, g.d, 0, 2**30 + 12345, g.m, L, accumulate=split)
    assert torch.equal(split, full)
    allc = torch.empty(g.n, dtype=torch.int64, device="cuda")
    ba.ba_degree_count(g.seed, g.n, g.d, g.n, allc)
    torch.cuda.synchronize()
    assert int(allc.sum()) == 2 * g.m
    assert torch.equal(allc[:L], full)


def test_streaming_workload_prefix_and_partition(ba):
    # n = 10^10, d = 100: the section 3 experiment scaled 1000x down.  The oracle checks the
    # 10^9-edge prefix and the last 10^8 edges (64-bit positions); the full 10^12-edge count
    # is checked for split invariance.
    g = W.STREAM_HUGE
    L = W.DEGREE_NODE_LIMIT
    for a, b in [(0, 10**9), (g.m - 10**8, g.m)]:
        np.testing.assert_array_equal(
            _counts(ba, g.seed, g.n, g.d, 0, a, b, L).cpu().numpy().astype(np.uint64),
            opar.degree_count_range(g.seed, g.n, g.d, 0, a, b, L))
    full = torch.empty(L, dtype=torch.int64, device="cuda")
    ba.ba_degree_count(g.seed, g.n, g.d, L, full)
    cut = 5 * 10**11 + 3
    split = _counts(ba, g.seed, g.n, g.d, 0, 0, cut, L)
    _counts(ba, g.seed, g.n, g.d, 0, cut, g.m, L, accumulate=split)
    assert torch.equal(split, full)
    c = full.cpu().numpy().astype(float)
    j = np.arange(L)
    cuts = np.unique(np.logspace(2, 5, 25).astype(int))
    xs = [np.log(j[x:y].mean()) for x, y in zip(cuts[:-1], cuts[1:])]
    ys = [np.log(c[x:y].mean()) for x, y in zip(cuts[:-1], cuts[1:])]
    slope = np.polyfit(xs, ys, 1)[0]
    assert -0.55 <= slope <= -0.45      # Fig. 2: degree ~ d sqrt(n/j)


@pytest.mark.parametrize("seed,n,d,n0", [(5, 100_500, 3, 100_000), (6, 2**20 + 13, 2, 2**20 + 3)])
def test_huge_seed_cliques(ba, seed, n, d, n0):
    # closed-form clique end points (k_degree_init) and chains that stop in a clique whose
    # positions exceed 2^32 (and 2^40)
    m0 = n0 * (n0 - 1) // 2
    m = ba.ba_num_edges(n, d, n0)
    for a, b, limit in [(m0 - 700, m, n), (m0 - 700, m, 5000), (0, 500, 40)]:
        np.testing.assert_array_equal(_counts(ba, seed, n, d, n0, a, b, limit).cpu().numpy().astype(np.uint64),
                                      oracle.degree_count_range(seed, n, d, n0, a, b, limit))
