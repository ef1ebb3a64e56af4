"""GPU parity of the variant graphs (BA_VARIANT_* flags) against the oracle.

hash_crc of Fig. 3 in place of h, the self-loop-free rule of section 4, and both
together, through ba_generate_edges_variant and ba_degree_count_variant.  Integer work:
every comparison is bit-exact.  Sizes span many tiles with ragged tails, both position
paths (positions below and above 2^32), and the 2^31-edge graph at full size on sampled
ranges plus properties that hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import parallel as opar

pytestmark = pytest.mark.gpu

CRC, NOLOOP = 1, 2
VARIANTS = [CRC, NOLOOP, CRC | NOLOOP]


def _family(v):
    return oracle.HASH_CRC if v & CRC else oracle.HASH_SPLITMIX


def _gpu(ba, seed, n, d, n0, a, b, v):
    out = torch.empty((b - a, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges_variant(seed, n, d, n0, a, b, v, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _oracle(seed, n, d, n0, a, b, v):
    return opar.edges_range_variant(seed, n, d, n0, _family(v), bool(v & NOLOOP), a, b)


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("seed,n,d,n0", [(1, 20_000, 4, 2), (2, 5_000, 7, 8), (3, 3_000, 1, 3),
                                         (4, 700, 33, 40), (2**64 - 1, 9_000, 2, 5)])
def test_full_graph_bit_exact(ba, v, seed, n, d, n0):
    E = oracle.bb_array_variant(seed, n, d, n0, _family(v), bool(v & NOLOOP)).reshape(-1, 2)
    m = E.shape[0]
    np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, 0, m, v), E)


@pytest.mark.parametrize("seed,n,d", [(5, 30_000, 3), (6, 1, 1), (7, 2, 5)])
def test_crc_hash_without_a_seed_graph(ba, seed, n, d):
    E = oracle.bb_array_variant(seed, n, d, 0, oracle.HASH_CRC, False).reshape(-1, 2)
    np.testing.assert_array_equal(_gpu(ba, seed, n, d, 0, 0, E.shape[0], CRC), E)


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("seed,n,d,n0,a,b", [
    (11, 400_000, 5, 6, 17, 1_500_003), (12, 100_000, 16, 17, 1_000_001, 1_599_864),
    (13, 2**27, 16, 17, 2**31 - 700_136, 2**31 - 136),        # end of the 32-bit path
    (14, 10**10, 100, 101, 10**12 - 505_050, 10**12 - 5_050),  # 64-bit positions
    (15, 2**28, 16, 2, 2**31 - 300_000, 2**31 + 300_001),      # across 2^32 positions
])
def test_ranges_match_oracle(ba, v, seed, n, d, n0, a, b):
    np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b, v),
                                  _oracle(seed, n, d, n0, a, b, v))


def test_variant_zero_is_the_plain_graph(ba):
    a, b = 1_000, 899_994
    plain = torch.empty((b - a, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges(21, 300_000, 3, 4, a, b, plain)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_gpu(ba, 21, 300_000, 3, 4, a, b, 0), plain.cpu().numpy())


@pytest.mark.parametrize("shape", [
    {"refill": 1, "block": 32, "ctas_per_sm": 1, "tile": 64},
    {"refill": 1, "block": 1024, "ctas_per_sm": 1, "tile": 2048},
    {"refill": 0, "block": 256, "ctas_per_sm": 4},            # variants still use refill
    {"refill": 1, "block": 256, "ctas_per_sm": 2, "tile": 1024, "chains": 2},
], ids=["b32-t64", "b1024-t2048", "simple", "b256-t1024-c2"])
def test_output_does_not_depend_on_launch_shape(ba, shape):
    seed, n, d, n0, a, b = 31, 200_000, 3, 4, 5, 599_994
    want = {v: _oracle(seed, n, d, n0, a, b, v) for v in VARIANTS}
    try:
        ba.ba_set_tuning(ba.BA_KIND_GENERATE, shape)
        for v in VARIANTS:
            np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b, v), want[v])
    finally:
        ba.ba_set_tuning(ba.BA_KIND_GENERATE, None)


def test_full_size_graph_sampled_and_loop_free(ba):
    # n = 2^27, d = 16 with a 17-clique: 2^31 - 136 edges (34 GB of pairs) in one call
    seed, n, d, n0 = 42, 2**27, 16, 17
    m = ba.ba_num_edges(n, d, n0)
    v = CRC | NOLOOP
    out = torch.empty((m, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges_variant(seed, n, d, n0, 0, m, v, out)
    torch.cuda.synchronize()
    for a, b in [(0, 400_000), (m // 2 - 200_000, m // 2 + 200_000), (m - 400_000, m)]:
        np.testing.assert_array_equal(out[a:b].cpu().numpy(), _oracle(seed, n, d, n0, a, b, v))
    src, tgt = out[136:, 0], out[136:, 1]
    assert bool((tgt < src).all()) and bool((tgt >= 0).all())
    idx = torch.arange(136, m, device="cuda", dtype=torch.int64)
    assert bool((src == n0 + (idx - 136) // d).all())
    del out, src, tgt, idx
    torch.cuda.empty_cache()


def _deg_gpu(ba, seed, n, d, n0, a, b, limit, v, counts=None, acc=0):
    if counts is None:
        counts = torch.empty(limit, dtype=torch.int64, device="cuda")
    ba.ba_degree_count_variant(seed, n, d, n0, a, b, limit, v, counts, acc)
    torch.cuda.synchronize()
    return counts


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("seed,n,d,n0,limit", [(41, 50_000, 4, 5, 50_000), (42, 9_000, 7, 2, 20_000),
                                               (43, 3_000, 1, 3, 100)])
def test_degree_count_full_graph(ba, v, seed, n, d, n0, limit):
    E = oracle.bb_array_variant(seed, n, d, n0, _family(v), bool(v & NOLOOP))
    want = oracle.degrees_of_array(E, limit)
    got = _deg_gpu(ba, seed, n, d, n0, 0, E.size // 2, limit, v).cpu().numpy().astype(np.uint64)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("v", VARIANTS)
def test_degree_count_ranges_add_up_and_match_oracle(ba, v):
    seed, n, d, n0, limit = 44, 10**10, 100, 101, 100_000
    m = ba.ba_num_edges(n, d, n0)
    a, mid, b = m - 3_000_000, m - 1_400_001, m                # 64-bit positions
    counts = _deg_gpu(ba, seed, n, d, n0, a, mid, limit, v)
    _deg_gpu(ba, seed, n, d, n0, mid, b, limit, v, counts, 1)
    want = opar.degree_count_range_variant(seed, n, d, n0, _family(v), bool(v & NOLOOP), a, b,
                                           limit)
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.uint64), want)


def test_crc_degree_count_of_the_paper_experiment_shape(ba):
    # section 3's analysis with the hash of its experiment, on a prefix of a 2^40-node
    # graph: the degrees of the first 10^5 nodes over the first 2 * 10^6 edges
    seed, n, d, limit, b = 0, 2**40, 100, 100_000, 2_000_000
    got = _deg_gpu(ba, seed, n, d, 0, 0, b, limit, CRC).cpu().numpy().astype(np.uint64)
    want = opar.degree_count_range_variant(seed, n, d, 0, oracle.HASH_CRC, False, 0, b, limit)
    np.testing.assert_array_equal(got, want)
    assert int(got.sum()) == 2 * b


def test_degree_shape_with_full_shared_bins_still_runs_the_table_draws(ba):
    # A degree shape whose bins fill the shared memory with the plain draw (the 64-bit
    # path's hit buffers at 1024 threads, 24576 bins): the table-driven hash_crc count gets
    # fewer bins, not an error, and the same counts.
    seed, n, d, n0, limit = 44, 10**10, 100, 101, 100_000
    m = ba.ba_num_edges(n, d, n0)
    a, b = m - 1_000_000, m                                    # 64-bit positions
    want = opar.degree_count_range_variant(seed, n, d, n0, oracle.HASH_CRC, True, a, b, limit)
    big = {"refill": 1, "block": 1024, "ctas_per_sm": 1, "tile": 65536, "hist_bins": 24576,
           "chains": 2}
    try:
        ba.ba_set_tuning(ba.BA_KIND_DEGREE, big)
        got = _deg_gpu(ba, seed, n, d, n0, a, b, limit, CRC | NOLOOP)
    finally:
        ba.ba_set_tuning(ba.BA_KIND_DEGREE, None)
    np.testing.assert_array_equal(got.cpu().numpy().astype(np.uint64), want)
