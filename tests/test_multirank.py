"""The N > 1 path on CPU: two gloo ranks shard a graph by edge ranges (no exchange), sum their
degree counters with one all-reduce, and together reproduce the unsharded oracle bit for bit
(paper section 2: the result does not depend on the number of processors) -- for the plain
graph and for the simple graph of section 4 (no self-loops, duplicate targets rejected),
whose shards cut through a node's edges."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1602_07106_gb300 import shard

GRAPH = (11, 30_000, 5, 6)   # seed, n, d, n0 (clique seed graph)
LIMIT = 500


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _edges(simple, a, b):
    seed, n, d, n0 = GRAPH
    if simple:
        return oracle.edges_range_simple(seed, n, d, n0, True, a, b)
    return oracle.edges_range(seed, n, d, n0, a, b)


def _counts(simple, a, b):
    seed, n, d, n0 = GRAPH
    if simple:
        return oracle.degree_count_range_simple(seed, n, d, n0, True, a, b, LIMIT)
    return oracle.degree_count_range(seed, n, d, n0, a, b, LIMIT)


def _rank_main(rank, world, port, result_dir, weak, simple):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed, n, d, n0 = GRAPH
    if weak:
        per = oracle.num_edges(n, d, n0) // world
        a, b = shard.weak_shard(per, rank)
    else:
        a, b = shard.strong_shard(oracle.num_edges(n, d, n0), rank, world)
    edges = torch.from_numpy(_edges(simple, a, b))
    counts = torch.from_numpy(_counts(simple, a, b).astype(np.int64))
    shard.sum_degree_counts(counts)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([edges.shape[0]]))
    top = max(int(s) for s in sizes)     # gloo gathers equal shapes: pad, then trim
    padded = torch.zeros((top, 2), dtype=torch.int64)
    padded[:edges.shape[0]] = edges
    gathered = [torch.zeros((top, 2), dtype=torch.int64) for _ in sizes]
    dist.all_gather(gathered, padded)
    if rank == 0:
        parts = [t[:int(s)] for t, s in zip(gathered, sizes)]
        torch.save({"edges": torch.cat(parts), "counts": counts, "end": sum(int(s) for s in sizes)},
                   os.path.join(result_dir, "out.pt"))
    dist.destroy_process_group()


@pytest.mark.parametrize("weak,simple", [(False, False), (True, False), (False, True)])
def test_two_gloo_ranks_reproduce_the_unsharded_graph(tmp_path, weak, simple):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), weak, simple),
                       nprocs=world, join=True, start_method="spawn")
    res = torch.load(tmp_path / "out.pt")
    total = res["end"]
    np.testing.assert_array_equal(res["edges"].numpy(), _edges(simple, 0, total))
    np.testing.assert_array_equal(res["counts"].numpy().astype(np.uint64),
                                  _counts(simple, 0, total))
    if simple:  # the cut falls inside a node
        seed, n, d, n0 = GRAPH
        assert (total // 2 - n0 * (n0 - 1) // 2) % d != 0


def test_shard_bounds():
    m = 10**6 + 7
    cuts = [shard.strong_shard(m, r, 3) for r in range(3)]
    assert cuts[0][0] == 0 and cuts[-1][1] == m
    assert all(cuts[k][1] == cuts[k + 1][0] for k in range(2))
    assert shard.weak_shard(100, 2) == (200, 300)
    with pytest.raises(ValueError):
        shard.strong_shard(m, 3, 3)
