"""GPU test of ba_generate_batch_noalloc, the batched launch that allocates nothing.

It is meant for callers that cannot allocate device memory at the point of the call (for
example while another framework's caching allocator owns the device memory, or under a
fixed device memory budget).  Its scratch lives in a static device table shared by all
calls, so the test calls it twice in a row with different batches, through the C ABI,
and compares each result with the allocating entry point ba_generate_batch: the work is
integer hashing, so the comparison is bit-exact.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import pytest
import torch

from paper_1602_07106_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(table_seed, G):
    table = W.batch_table(G=G, n_lo=1e2, n_hi=2e5, table_seed=table_seed)
    graphs = [(g.seed, g.n, g.d, g.n0, g.m // 7, g.m) for g in table]
    total = sum(b - a for *_, a, b in graphs)
    return graphs, total


def test_noalloc_batch_matches_allocating_batch_on_two_calls_in_a_row(ba):
    first, total1 = _batch(101, 700)
    second, total2 = _batch(202, 1024)       # the largest batch the static table holds
    out1 = torch.full((total1, 2), -1, dtype=torch.int64, device="cuda")
    out2 = torch.full((total2, 2), -1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    allocs = ba.ba_device_allocations()
    ba.ba_generate_batch_noalloc(first, out1)
    ba.ba_generate_batch_noalloc(second, out2)
    torch.cuda.synchronize()
    assert ba.ba_device_allocations() == allocs      # the two calls allocated nothing
    want1 = torch.empty_like(out1)
    want2 = torch.empty_like(out2)
    ba.ba_generate_batch(first, want1)
    ba.ba_generate_batch(second, want2)
    torch.cuda.synchronize()
    assert torch.equal(out1, want1)
    assert torch.equal(out2, want2)
    # the scratch keeps the previous call's contents: a smaller batch after a larger one
    # must not see stale graphs or a stale tile counter
    out3 = torch.full((total1, 2), -1, dtype=torch.int64, device="cuda")
    allocs = ba.ba_device_allocations()
    ba.ba_generate_batch_noalloc(first, out3)
    torch.cuda.synchronize()
    assert ba.ba_device_allocations() == allocs
    assert torch.equal(out3, want1)
    # the allocating entry point is counted, so the counter does see allocations
    ba.ba_generate_batch(first, want1)
    torch.cuda.synchronize()
    assert ba.ba_device_allocations() > allocs


def test_noalloc_batch_with_offsets_and_rejections(ba):
    graphs = [(1, 1000, 3, 0, 10, 2000), (2, 50, 4, 5, 0, 10), (3, 2**29, 16, 0, 2**33 - 70_000, 2**33)]
    offsets = [0]
    for g in graphs:
        offsets.append(offsets[-1] + (g[5] - g[4]) + 5)
    got = torch.full((offsets[-1], 2), -3, dtype=torch.int64, device="cuda")
    want = torch.full((offsets[-1], 2), -3, dtype=torch.int64, device="cuda")
    ba.ba_generate_batch_noalloc(graphs, got, offsets=offsets)
    ba.ba_generate_batch(graphs, want, offsets=offsets)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    too_many = [(k, 100, 1, 0, 0, 100) for k in range(ba.BA_NOALLOC_MAX_GRAPHS + 1)]
    with pytest.raises(ba.BAError) as e:
        ba.ba_generate_batch_noalloc(too_many, got)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    assert "1024" in str(e.value)
