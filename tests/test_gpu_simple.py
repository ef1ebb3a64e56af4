"""GPU parity of the graph without parallel edges (BA_VARIANT_NO_PARALLEL_EDGES, section 4:
a node's duplicate targets are rejected and redrawn) against the oracle, bit-exact: whole
graphs, ranges that start or end inside a node, both position paths, with and without
self-loops and seed cliques, d up to 32 (a warp item of whole nodes) and 33..1024 (a warp
per node), the 2^31-edge graph at full size on sampled
ranges plus the no-parallel-edge property over every node, and the streaming degree count
of the same graph."""
import numpy as np
import pytest
import torch

import oracle
from oracle import parallel as opar
from paper_1602_07106_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NOLOOP, SIMPLE = 2, 4


def _gpu(ba, seed, n, d, n0, a, b, v):
    out = torch.full((b - a, 2), -1, dtype=torch.int64, device="cuda")
    ba.ba_generate_edges_variant(seed, n, d, n0, a, b, v, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [(21, 20_000, 4, 0, False, 0, None), (22, 5_000, 16, 0, False, 37, -11),
         (23, 3_000, 32, 33, True, 0, None), (24, 4_000, 5, 6, False, 100, 15_000),
         (25, 100_000, 3, 1, False, 0, None), (26, 2_000, 32, 0, False, 0, None),
         (27, 30_000, 7, 8, True, 1_234, -77), (28, 50_000, 2, 2, True, 0, None),
         (29, 3_000, 31, 0, False, 5, -3), (2**64 - 1, 9_000, 9, 0, False, 0, None),
         (32, 20_000, 16, 5, False, 3, -5), (33, 10_000, 8, 3, True, 0, None)]


@pytest.mark.parametrize("seed,n,d,n0,no_loops,a,b", CASES)
def test_bit_exact_against_oracle(ba, seed, n, d, n0, no_loops, a, b):
    m = oracle.num_edges(n, d, n0)
    b = m if b is None else (m + b if b < 0 else b)
    v = SIMPLE | (NOLOOP if no_loops else 0)
    got = _gpu(ba, seed, n, d, n0, a, b, v)
    np.testing.assert_array_equal(got, oracle.edges_range_simple(seed, n, d, n0, no_loops, a, b))


# d > 32: one warp per node (the paper's m = 100n shape among them)
WIDE_CASES = [(41, 3_000, 100, 0, False, 0, None), (42, 4_000, 33, 0, False, 17, -5),
              (43, 2_500, 64, 65, True, 0, None), (44, 6_000, 100, 3, False, 1_234, 431_777),
              (45, 1_200, 257, 1, False, 0, None), (46, 1_100, 1024, 0, False, 5_000, -700),
              (47, 2_000, 100, 101, True, 99, -1), (2**63 + 9, 5_000, 48, 0, False, 0, None)]


@pytest.mark.parametrize("seed,n,d,n0,no_loops,a,b", WIDE_CASES)
def test_wide_nodes_bit_exact_against_oracle(ba, seed, n, d, n0, no_loops, a, b):
    m = oracle.num_edges(n, d, n0)
    b = m if b is None else (m + b if b < 0 else b)
    v = SIMPLE | (NOLOOP if no_loops else 0)
    got = _gpu(ba, seed, n, d, n0, a, b, v)
    want = oracle.edges_range_simple(seed, n, d, n0, no_loops, a, b)
    np.testing.assert_array_equal(got, want)
    # the rejections happened: the plain graph differs from this one on the same range
    plain = _gpu(ba, seed, n, d, n0, a, b, v & ~SIMPLE)
    assert (plain[:, 1] != got[:, 1]).any()


@pytest.mark.parametrize("a_off,b_off", [(0, 1), (40, 41), (7, 99), (99, 101), (1, 350)])
def test_wide_ranges_inside_and_across_nodes(ba, a_off, b_off):
    # d = 100: ranges that start and end inside nodes, down to a single edge
    seed, n, d = 48, 3_000, 100
    base = 100 * 57
    got = _gpu(ba, seed, n, d, 0, base + a_off, base + b_off, SIMPLE)
    np.testing.assert_array_equal(got, oracle.edges_range_simple(seed, n, d, 0, False,
                                                                 base + a_off, base + b_off))


@pytest.mark.parametrize("no_loops,n0", [(False, 0), (True, 101)])
def test_wide_64bit_positions_and_property(ba, no_loops, n0):
    seed, n, d = 49, 2**26, 100
    m = oracle.num_edges(n, d, n0)
    v = SIMPLE | (NOLOOP if no_loops else 0)
    a, b = m - 100_037, m - 13
    np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b, v),
                                  oracle.edges_range_simple(seed, n, d, n0, no_loops, a, b))
    # a 2^24-edge prefix block: every node whose reach covers d has d distinct targets
    lo = (n0 * (n0 - 1)) // 2 + 200 * d
    hi = lo + 2**24 // d * d
    out = torch.from_numpy(_gpu(ba, seed, n, d, n0, lo, hi, v)).cuda()
    t = out[:, 1].view(-1, d)
    s_, _ = torch.sort(t, dim=1)
    assert bool((s_[:, 1:] > s_[:, :-1]).all())


@pytest.mark.parametrize("seed,n,d,n0,no_loops,a,b", WIDE_CASES[:5])
def test_wide_degree_count_against_oracle(ba, seed, n, d, n0, no_loops, a, b):
    m = oracle.num_edges(n, d, n0)
    b = m if b is None else (m + b if b < 0 else b)
    v = SIMPLE | (NOLOOP if no_loops else 0)
    limit = min(n, 5_000) + 3
    want = oracle.degree_count_range_simple(seed, n, d, n0, no_loops, a, b, limit)
    counts = torch.full((limit,), 7, dtype=torch.int64, device="cuda")
    ba.ba_degree_count_variant(seed, n, d, n0, a, b, limit, v, counts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.uint64), want)


@pytest.mark.parametrize("a_off,b_off", [(0, 1), (3, 5), (5, 37), (1, 64), (15, 33)])
def test_ranges_inside_and_across_nodes(ba, a_off, b_off):
    # d = 16: ranges that start and end inside nodes, down to a single edge
    seed, n, d = 31, 4_000, 16
    base = 16 * 40
    got = _gpu(ba, seed, n, d, 0, base + a_off, base + b_off, SIMPLE)
    np.testing.assert_array_equal(got, oracle.edges_range_simple(seed, n, d, 0, False,
                                                                 base + a_off, base + b_off))


@pytest.mark.parametrize("no_loops,n0", [(False, 0), (True, 17)])
def test_64bit_positions(ba, no_loops, n0):
    seed, n, d = 77, 2**29, 16
    m = oracle.num_edges(n, d, n0)
    a, b = 2**33 - 100_003 - (m - n * d), m - 17
    v = SIMPLE | (NOLOOP if no_loops else 0)
    np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b, v),
                                  oracle.edges_range_simple(seed, n, d, n0, no_loops, a, b))


@pytest.mark.parametrize("shape", [{"refill": 0, "block": 256, "ctas_per_sm": 8},
                                   {"refill": 1, "block": 64, "ctas_per_sm": 8, "tile": 64},
                                   {"refill": 1, "block": 128, "ctas_per_sm": 2, "tile": 256,
                                    "chains": 2}])
def test_output_does_not_depend_on_shape(ba, shape):
    want = oracle.edges_range_simple(5, 50_000, 8, 0, False, 11, 399_990)
    try:
        ba.ba_set_tuning(ba.BA_KIND_GENERATE, shape)
        np.testing.assert_array_equal(_gpu(ba, 5, 50_000, 8, 0, 11, 399_990, SIMPLE), want)
    finally:
        ba.ba_set_tuning(ba.BA_KIND_GENERATE, None)


@pytest.mark.parametrize("no_loops,n0", [(False, 0), (True, 17)])
def test_full_size_graph(ba, no_loops, n0):
    g = W.PLAIN_LARGE
    m = oracle.num_edges(g.n, g.d, n0)
    m0 = n0 * (n0 - 1) // 2
    v = SIMPLE | (NOLOOP if no_loops else 0)
    out = torch.empty((m, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges_variant(g.seed, g.n, g.d, n0, 0, m, v, out)
    torch.cuda.synchronize()
    for a, b in [(0, 1_000_000), (2**30 - 500_000, 2**30 + 500_003), (m - 1_000_000, m)]:
        np.testing.assert_array_equal(out[a:b].cpu().numpy(),
                                      opar.edges_range_simple(g.seed, g.n, g.d, n0, no_loops, a, b))
    # no node with 16 reachable nodes has two equal targets: sorted targets strictly increase
    first = 16                                               # reach(u) >= 16 from node 16 on
    t = out[m0:, 1].view(g.n - n0, g.d)[max(first - n0, 0):]
    s, _ = torch.sort(t, dim=1)
    assert bool((s[:, 1:] > s[:, :-1]).all())
    src = out[m0:, 0].view(g.n - n0, g.d)
    if no_loops:
        assert bool((out[m0:, 1] < out[m0:, 0]).all())
    else:
        assert bool((out[:, 1] <= out[:, 0]).all())
    assert bool((src == torch.arange(n0, g.n, device="cuda").view(-1, 1)).all())
    # the array's own targets are kept wherever the node had no duplicate
    plain = torch.empty_like(out)
    ba.ba_generate_edges_variant(g.seed, g.n, g.d, n0, 0, m, v & ~SIMPLE, plain)
    changed = int((plain[:, 1] != out[:, 1]).sum())
    assert 0 < changed < m // 1000


@pytest.mark.parametrize("seed,n,d,n0,no_loops,a,b", CASES + [(30, 40_000, 1, 0, False, 0, None),
                                                               (31, 9_000, 1, 2, True, 3, -4)])
def test_degree_count_bit_exact_against_oracle(ba, seed, n, d, n0, no_loops, a, b):
    m = oracle.num_edges(n, d, n0)
    b = m if b is None else (m + b if b < 0 else b)
    v = SIMPLE | (NOLOOP if no_loops else 0)
    limit = min(n, 5_000) + 3
    want = oracle.degree_count_range_simple(seed, n, d, n0, no_loops, a, b, limit)
    counts = torch.full((limit,), 7, dtype=torch.int64, device="cuda")
    ba.ba_degree_count_variant(seed, n, d, n0, a, b, limit, v, counts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.uint64), want)
    # a split of the range accumulates to the same counts
    mid = (a + b) // 2 + 3
    ba.ba_degree_count_variant(seed, n, d, n0, a, mid, limit, v, counts)
    ba.ba_degree_count_variant(seed, n, d, n0, mid, b, limit, v, counts, accumulate=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.uint64), want)


def test_degree_count_64bit_positions(ba):
    seed, n, d = 78, 2**29, 16
    a, b = 2**33 - 200_000, 2**33
    want = oracle.degree_count_range_simple(seed, n, d, 0, False, a, b, 100_000)
    counts = torch.empty(100_000, dtype=torch.int64, device="cuda")
    ba.ba_degree_count_variant(seed, n, d, 0, a, b, 100_000, SIMPLE, counts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.uint64), want)


@pytest.mark.parametrize("no_loops,n0", [(False, 0), (True, 3)])
def test_fold_launch_boundary(ba, no_loops, n0):
    # d = 2: the fold generates 2^25 nodes' edges (2^26 edges) per launch, so this range is
    # two launches, the second starting inside a node; the edges around the boundary and a
    # degree count over the whole range match the oracle
    seed, n, d = 41, 2**27, 2
    a = 1_000_001
    b = a + 2**26 + 20_000
    v = SIMPLE | (NOLOOP if no_loops else 0)
    out = torch.empty((b - a, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges_variant(seed, n, d, n0, a, b, v, out)
    torch.cuda.synchronize()
    cut = a + 2**26
    for lo, hi in [(a, a + 3_000), (cut - 5_000, cut + 5_001), (b - 3_000, b)]:
        np.testing.assert_array_equal(out[lo - a:hi - a].cpu().numpy(),
                                      opar.edges_range_simple(seed, n, d, n0, no_loops, lo, hi))
    limit = 50_000
    want = opar.degree_count_range_simple(seed, n, d, n0, no_loops, a, b, limit)
    counts = torch.empty(limit, dtype=torch.int64, device="cuda")
    ba.ba_degree_count_variant(seed, n, d, n0, a, b, limit, v, counts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.uint64), want)


@pytest.mark.parametrize("d,n0,no_loops", [(32, 40, False), (32, 40, True), (8, 6, True),
                                          (4, 0, False)])
def test_fold_64bit_positions_seeded(ba, d, n0, no_loops):
    # the fold on 64-bit positions, with seed cliques whose edge count is not a multiple
    # of d (m0 = 780 for n0 = 40: every chunk cuts a node), ranges that start and end
    # inside nodes; edges and a degree count against the oracle
    seed, n = 91, 2**30 // d * 4
    m = oracle.num_edges(n, d, n0)
    a, b = m - 150_001 - 2**32 // 3, m - 2**32 // 3 - 7
    assert b > 2**31
    v = SIMPLE | (NOLOOP if no_loops else 0)
    np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b, v),
                                  oracle.edges_range_simple(seed, n, d, n0, no_loops, a, b))
    limit = 100_000
    want = oracle.degree_count_range_simple(seed, n, d, n0, no_loops, a, b, limit)
    counts = torch.empty(limit, dtype=torch.int64, device="cuda")
    ba.ba_degree_count_variant(seed, n, d, n0, a, b, limit, v, counts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.uint64), want)
