"""GPU parity of the batched launch: every graph of a batch, bit-exact against the oracle
and against the plain per-graph call."""
import numpy as np
import pytest
import torch

import oracle
from oracle import parallel as opar
from paper_1602_07106_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _plain(ba, seed, n, d, n0, a, b):
    out = torch.empty((b - a, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges(seed, n, d, n0, a, b, out)
    return out


def _check_against_oracle(host, graphs, offsets, full_limit=2_000_000):
    for k, g in enumerate(graphs):
        seed, n, d, n0, a, b = g
        got = host[offsets[k]:offsets[k] + (b - a)]
        if b - a <= full_limit:
            np.testing.assert_array_equal(got, oracle.edges_range(seed, n, d, n0, a, b))
        else:   # sampled ranges of large graphs
            for lo in (0, (b - a) // 2, b - a - 100_000):
                np.testing.assert_array_equal(got[lo:lo + 100_000],
                                              oracle.edges_range(seed, n, d, n0, a + lo, a + lo + 100_000))


def test_small_batch_table_every_graph_exact(ba):
    table = W.batch_table(G=256, n_lo=1e2, n_hi=1e5)
    graphs = [(g.seed, g.n, g.d, g.n0, 0, g.m) for g in table]
    plan = ba.ba_batch_plan_create(graphs)
    try:
        total = ba.ba_batch_plan_total_edges(plan)
        offsets = ba.ba_batch_plan_offsets(plan, len(graphs))
        assert total == sum(g.m for g in table) == offsets[-1]
        out = torch.full((total, 2), -1, dtype=torch.int64, device="cuda")
        ba.ba_batch_plan_launch(plan, out)
        torch.cuda.synchronize()
        host = out.cpu().numpy()
        _check_against_oracle(host, graphs, offsets)
        # replay into a second buffer: same bits
        out2 = torch.empty_like(out)
        ba.ba_batch_plan_launch(plan, out2)
        ba.ba_batch_plan_launch(plan, out2)
        torch.cuda.synchronize()
        assert torch.equal(out, out2)
    finally:
        ba.ba_batch_plan_destroy(plan)


def test_batch_ranges_gaps_and_64_bit_graphs_equal_plain_calls(ba):
    graphs = [(1, 1000, 3, 0, 10, 2000), (2, 50, 4, 5, 0, 10), (3, 2**29, 16, 0, 2**33 - 70_000, 2**33),
              (4, 10, 1, 0, 5, 5), (5, 2000, 32, 33, 100, 9000), (6, 2**27, 16, 0, 2**31 - 5000, 2**31),
              (7, 3, 2**31 + 3, 0, 0, 3 * (2**31 + 3) - 2**31)]
    offsets = [0]
    for g in graphs:
        offsets.append(offsets[-1] + (g[5] - g[4]) + 3)    # gaps between graphs
    out = torch.full((offsets[-1], 2), -9, dtype=torch.int64, device="cuda")
    ba.ba_generate_batch(graphs, out, offsets=offsets)
    torch.cuda.synchronize()
    for k, (seed, n, d, n0, a, b) in enumerate(graphs):
        if b - a > 1_000_000:
            a = b - 1_000_000
            sl = out[offsets[k + 1] - 3 - (b - a):offsets[k + 1] - 3]
        else:
            sl = out[offsets[k]:offsets[k] + (b - a)]
        assert torch.equal(sl, _plain(ba, seed, n, d, n0, a, b))
        np.testing.assert_array_equal(sl.cpu().numpy(), opar.edges_range(seed, n, d, n0, a, b))
        assert bool((out[offsets[k + 1] - 3:offsets[k + 1]] == -9).all())   # gaps untouched


@pytest.mark.parametrize("shape", [{"refill": 1, "block": 64, "ctas_per_sm": 2, "tile": 64},
                                   {"refill": 1, "block": 512, "ctas_per_sm": 2, "tile": 1024},
                                   {"refill": 1, "block": 256, "ctas_per_sm": 4, "tile": 256,
                                    "chains": 2}])
def test_batch_output_does_not_depend_on_shape(ba, shape):
    table = W.batch_table(G=64, n_lo=1e2, n_hi=1e4, table_seed=3)
    graphs = [(g.seed, g.n, g.d, g.n0, 0, g.m) for g in table]
    total = sum(g.m for g in table)
    a = torch.empty((total, 2), dtype=torch.int64, device="cuda")
    b = torch.empty((total, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_batch(graphs, a)
    ba.ba_generate_batch(graphs, b, tune=shape)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_batch_workload_first_wave_exact(ba):
    # The 4096-graph table is 1.2 TB of output, so it runs in waves; the first wave of
    # graphs that fits in 8 GB is checked here, every graph against the oracle.
    table = W.batch_table()
    graphs, total = [], 0
    for g in table:
        if total + g.m > 8 * 2**30 // 16 or len(graphs) == 96:
            continue
        graphs.append((g.seed, g.n, g.d, g.n0, 0, g.m))
        total += g.m
    assert len(graphs) >= 16
    plan = ba.ba_batch_plan_create(graphs)
    try:
        offsets = ba.ba_batch_plan_offsets(plan, len(graphs))
        out = torch.empty((total, 2), dtype=torch.int64, device="cuda")
        ba.ba_batch_plan_launch(plan, out)
        torch.cuda.synchronize()
        host = out.cpu().numpy()
        _check_against_oracle(host, graphs, offsets)
    finally:
        ba.ba_batch_plan_destroy(plan)


def test_batch_workload_whole_table_every_graph_exact(ba):
    # All 4096 graphs of the batched workload (7.6e10 edges, 1.2 TB of pairs) in waves of at
    # most 2^32 edges, one persistent launch per wave; every graph of every wave is checked
    # against the oracle: in full up to 2e6 edges, else on its first, middle and last 10^5.
    import multiprocessing as mp
    table = W.batch_table()
    budget = 2**32
    waves, cur, tot = [], [], 0
    for g in table:
        if cur and tot + g.m > budget:
            waves.append(cur)
            cur, tot = [], 0
        cur.append(g)
        tot += g.m
    waves.append(cur)
    assert sum(len(w) for w in waves) == 4096
    out = torch.empty((max(sum(g.m for g in w) for w in waves), 2), dtype=torch.int64,
                      device="cuda")
    checked = 0
    oracle.build()
    with mp.get_context("spawn").Pool(opar.default_workers()) as pool:
        for w in waves:
            graphs = [(g.seed, g.n, g.d, g.n0, 0, g.m) for g in w]
            plan = ba.ba_batch_plan_create(graphs)
            try:
                offsets = ba.ba_batch_plan_offsets(plan, len(graphs))
                ba.ba_batch_plan_launch(plan, out)
                torch.cuda.synchronize()
            finally:
                ba.ba_batch_plan_destroy(plan)
            jobs, slices = [], []
            for k, (seed, n, d, n0, a, b) in enumerate(graphs):
                spans = [(0, b - a)] if b - a <= 2_000_000 else \
                    [(0, 100_000), ((b - a) // 2, (b - a) // 2 + 100_000), (b - a - 100_000, b - a)]
                for lo, hi in spans:
                    jobs.append((seed, n, d, n0, a + lo, a + hi))
                    slices.append((offsets[k] + lo, offsets[k] + hi))
            for (x, y), want in zip(slices, pool.imap(opar._edges_piece, jobs, chunksize=8)):
                np.testing.assert_array_equal(out[x:y].cpu().numpy(), want)
            checked += len(graphs)
    assert checked == 4096
