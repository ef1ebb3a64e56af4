"""GPU parity of ba_generate_edges (Fig. 1 over edge ranges) against the oracle.

Integer work: every comparison is bit-exact.  Sizes span many warp tiles with ragged
tails; the full 2^31-edge graph is generated in the launch shape the benchmark uses and
checked on oracle-computed ranges at its start, middle and end, plus properties that hold
at any size (the source column is n0 + floor((i-m0)/d); targets never exceed sources).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import parallel as opar
from paper_1602_07106_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu(ba, seed, n, d, n0, a, b):
    out = torch.empty((b - a, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges(seed, n, d, n0, a, b, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_small_workload_full_edge_list_bit_exact(ba):
    g = W.PLAIN_SMALL
    E = oracle.bb_array(g.seed, g.n, g.d, g.n0).reshape(-1, 2)
    got = ba.generate_edges(g.seed, g.n, g.d).cpu().numpy()
    np.testing.assert_array_equal(got, E)


CASES = [
    (1, 1, 1, 0, 0, 1), (1, 2, 1, 0, 0, 2), (3, 1000, 1, 0, 0, 1000),
    (5, 777, 7, 0, 0, 777 * 7), (9, 5000, 3, 0, 17, 14_983), (11, 40_000, 2, 0, 1, 79_999),
    (13, 1000, 4, 5, 0, 10 + 995 * 4), (15, 3000, 2, 3, 2, 5000), (17, 500, 32, 33, 0, 528 + 467 * 32),
    (19, 200, 5, 1, 0, 995), (21, 64, 1, 2, 0, 63), (23, 40, 3, 40, 0, 780), (25, 40, 3, 40, 100, 700),
    (27, 100_000, 13, 0, 123_457, 987_654), (2**63 + 5, 10_000, 16, 17, 0, 136 + 9983 * 16),
    (29, 4, 2**31 + 3, 0, 0, 4 * (2**31 + 3)),       # d above 2^31 (all four nodes)
]


@pytest.mark.parametrize("seed,n,d,n0,a,b", CASES)
def test_ranges_match_oracle(ba, seed, n, d, n0, a, b):
    if b - a > 3_000_000:
        a = b - 3_000_000
    np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b),
                                  opar.edges_range(seed, n, d, n0, a, b))


def test_empty_range_and_single_edges(ba):
    out = torch.full((4, 2), -7, dtype=torch.int64, device="cuda")
    ba.ba_generate_edges(1, 100, 2, 0, 50, 50, out)
    torch.cuda.synchronize()
    assert (out == -7).all()
    for i in (0, 1, 63, 64, 65, 199):
        np.testing.assert_array_equal(_gpu(ba, 4, 100, 2, 0, i, i + 1),
                                      oracle.edges_range(4, 100, 2, 0, i, i + 1))


SHAPES = [
    {"refill": 0, "block": 256, "ctas_per_sm": 8},
    {"refill": 0, "block": 32, "ctas_per_sm": 1},
    {"refill": 1, "block": 32, "ctas_per_sm": 1, "tile": 64},
    {"refill": 1, "block": 128, "ctas_per_sm": 2, "tile": 256},
    {"refill": 1, "block": 256, "ctas_per_sm": 4, "tile": 512},
    {"refill": 1, "block": 512, "ctas_per_sm": 2, "tile": 1024},
    {"refill": 1, "block": 1024, "ctas_per_sm": 1, "tile": 512},
    {"refill": 1, "block": 64, "ctas_per_sm": 16, "tile": 4096},
    {"refill": 1, "block": 32, "ctas_per_sm": 1, "tile": 64, "chains": 2},
    {"refill": 1, "block": 128, "ctas_per_sm": 2, "tile": 128, "chains": 2},
    {"refill": 1, "block": 256, "ctas_per_sm": 4, "tile": 16384, "chains": 2},
    {"refill": 1, "block": 1024, "ctas_per_sm": 1, "tile": 2048, "chains": 2},
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()))
def test_output_does_not_depend_on_launch_shape(ba, shape):
    # section 2: the graph depends only on the hash, not on how the work is split
    cases = [(31, 300_000, 3, 0, 5, 899_999), (37, 50_000, 6, 7, 0, 21 + 49_993 * 6)]
    try:
        ba.ba_set_tuning(ba.BA_KIND_GENERATE, shape)
        for seed, n, d, n0, a, b in cases:
            np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b),
                                          opar.edges_range(seed, n, d, n0, a, b))
    finally:
        ba.ba_set_tuning(ba.BA_KIND_GENERATE, None)


SCHEDULERS = [None, {"refill": 1, "chains": 1},
              {"refill": 1, "chains": 2, "block": 128, "tile": 256}]


def _with_shape(ba, shape, fn):
    try:
        if shape is not None:
            ba.ba_set_tuning(ba.BA_KIND_GENERATE, shape)
        fn()
    finally:
        ba.ba_set_tuning(ba.BA_KIND_GENERATE, None)


@pytest.mark.parametrize("shape", SCHEDULERS, ids=str)
def test_64_bit_positions_far_into_a_large_graph(ba, shape):
    # m = 2^33: positions above 2^32 take the 64-bit path
    n, d = 2**29, 16
    m = n * d

    def run():
        for a, b in [(m - 300_000, m), (2**31 - 1000, 2**31 + 150_000), (2**32 - 777, 2**32 + 777)]:
            np.testing.assert_array_equal(_gpu(ba, 77, n, d, 0, a, b),
                                          opar.edges_range(77, n, d, 0, a, b))
    _with_shape(ba, shape, run)


@pytest.mark.parametrize("shape", SCHEDULERS, ids=str)
@pytest.mark.parametrize("seed,n,d,n0", [(81, 2**29, 13, 0), (83, 2**28, 24, 25), (85, 2**29, 8, 9)])
def test_64_bit_positions_other_d_and_seed_cliques(ba, seed, n, d, n0, shape):
    # the 64-bit flush's general path (d not a power of two, or a seed clique)
    m = ba.ba_num_edges(n, d, n0)

    def run():
        for a, b in [(m - 200_000, m), (2**31 - 500, 2**31 + 60_000)]:
            np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b),
                                          opar.edges_range(seed, n, d, n0, a, b))
    _with_shape(ba, shape, run)


@pytest.mark.parametrize("seed,n,d", [(91, 2**40, 2**20), (93, 2**41 + 7, 2**21 - 3),
                                      (95, 3 * 2**60 // 2**20, 2**20 - 1)])
def test_positions_up_to_2_to_the_62(ba, seed, n, d):
    # every 32-bit partial product of the 64-bit-position hash is non-trivial here (the
    # high half of r reaches 2^29 and beyond)
    m = n * d
    for a, b in [(m - 20_000, m), (m // 2 - 5_000, m // 2 + 5_000), (2**33, 2**33 + 5_000)]:
        np.testing.assert_array_equal(_gpu(ba, seed, n, d, 0, a, b),
                                      oracle.edges_range(seed, n, d, 0, a, b))


def test_host_output_matches_device_output(ba):
    g = W.PLAIN_SMALL
    host = torch.empty((g.m, 2), dtype=torch.int64).pin_memory()
    ba.ba_generate_edges_host(g.seed, g.n, g.d, 0, 0, g.m, host)
    dev = ba.generate_edges(g.seed, g.n, g.d).cpu()
    assert torch.equal(host, dev)
    # several chunks and a ragged tail
    n, d = 2**26, 1
    a, b = 3, 2**26 - 5
    host2 = torch.empty((b - a, 2), dtype=torch.int64)
    ba.ba_generate_edges_host(99, n, d, 0, a, b, host2)
    for lo, hi in [(0, 100_000), (2**25 - 50_000, 2**25 + 50_000), (b - a - 100_000, b - a)]:
        np.testing.assert_array_equal(host2[lo:hi].numpy(),
                                      oracle.edges_range(99, n, d, 0, a + lo, a + hi))


def test_large_workload_full_size_spot_ranges_and_properties(ba):
    g = W.PLAIN_LARGE
    out = torch.empty((g.m, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges(g.seed, g.n, g.d, 0, 0, g.m, out)
    torch.cuda.synchronize()
    for a, b in W.PLAIN_LARGE_SPOT_RANGES:
        np.testing.assert_array_equal(out[a:b].cpu().numpy(),
                                      opar.edges_range(g.seed, g.n, g.d, 0, a, b))
    step = 2**27
    for a in range(0, g.m, step):
        blk = out[a:a + step]
        i = torch.arange(a, a + blk.shape[0], device="cuda", dtype=torch.int64)
        assert torch.equal(blk[:, 0], i // g.d)
        assert bool((blk[:, 1] <= blk[:, 0]).all()) and bool((blk[:, 1] >= 0).all())
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("seed,n,d,n0", [(5, 100_500, 3, 100_000),        # m0 ~ 5e9: 64-bit positions
                                         (6, 2**20 + 13, 2, 2**20 + 3)])  # 2 m0 > 2^40
def test_huge_seed_cliques(ba, seed, n, d, n0):
    # the clique lookup's float estimate (and, above 2^40, double) on positions beyond 2^32
    m0 = n0 * (n0 - 1) // 2
    m = ba.ba_num_edges(n, d, n0)
    for a, b in [(m0 - 700, min(m, m0 + 700)), (max(m0 - 300, m - 700), m), (0, 300)]:
        np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b),
                                      oracle.edges_range(seed, n, d, n0, a, b))


@pytest.mark.parametrize("seed,n,d,n0", [(8, 2**16 + 1, 2**15, 2**16),      # n0 d = 2^31, m = 2^31
                                         (9, 2**15 + 10_001, 2**16, 2**15 + 1)])  # n0 d > 2^31
def test_seeded_power_of_two_d_with_n0_d_at_2_31(ba, seed, n, d, n0):
    # Seed cliques whose n0 d reaches 2^31 on 32-bit positions (m <= 2^31): node IDs near
    # 2^16 with d = 2^15 and 2^16, chains that stop inside a clique of ~2^31 positions, and
    # the last edge of a graph with exactly 2^31 edges; int64 and int32 pairs
    m0 = n0 * (n0 - 1) // 2
    m = ba.ba_num_edges(n, d, n0)
    assert m <= 2**31
    for a, b in [(m0 - 500, m0 + 700), (m - 700, m), ((m0 + m) // 2, (m0 + m) // 2 + 700)]:
        want = oracle.edges_range(seed, n, d, n0, a, b)
        np.testing.assert_array_equal(_gpu(ba, seed, n, d, n0, a, b), want)
        out32 = torch.empty((b - a, 2), dtype=torch.int32, device="cuda")
        ba.ba_generate_edges32(seed, n, d, n0, a, b, out32)
        np.testing.assert_array_equal(out32.cpu().numpy().astype(np.int64), want)


def test_concurrent_calls_from_host_threads(ba):
    # the library is called from several host threads at once, each on its own stream
    # (ctypes releases the GIL): every result is the one a lone call gives
    import threading
    cases = [(101 + k, 50_000 + 1000 * k, 1 + k % 5, (k % 3) * 4) for k in range(8)]
    want = {c: oracle.bb_array(*c).reshape(-1, 2) for c in cases}
    got, errors = {}, []

    def worker(c):
        try:
            s = torch.cuda.Stream()
            m = want[c].shape[0]
            out = torch.empty((m, 2), dtype=torch.int64, device="cuda")
            for _ in range(3):
                ba.ba_generate_edges(*c, 0, m, out, s)
            s.synchronize()
            got[c] = out.cpu().numpy()
        except Exception as e:  # noqa: BLE001 -- reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(c,)) for c in cases]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for c in cases:
        np.testing.assert_array_equal(got[c], want[c])
