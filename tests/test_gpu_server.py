"""GPU tests of the serving loop: each served result is bit-identical to the plain call
(and to the oracle), alone and in a mix of concurrent requests; admission respects the
memory budget without hanging."""
import numpy as np
import pytest
import torch

import oracle
from paper_1602_07106_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _plain(ba, seed, n, d, n0, a, b):
    out = torch.empty((b - a, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges(seed, n, d, n0, a, b, out)
    torch.cuda.synchronize()
    return out


def _requests():
    trace = W.serving_trace(rate=2000.0, duration=0.02, trace_seed=11, len_hi=3e6)
    reqs = [(r.graph.seed, r.graph.n, r.graph.d, 0, r.edge_begin, r.edge_end) for r in trace]
    reqs += [(5, 1000, 3, 4, 0, 2994), (6, 2**29, 16, 0, 2**33 - 100_000, 2**33), (7, 10, 1, 0, 3, 3)]
    return reqs


def test_served_results_equal_plain_alone_and_in_mix(ba):
    reqs = _requests()
    assert len(reqs) >= 20
    srv = ba.ba_server_create(memory_budget_bytes=4 << 30, chunk_edges=1 << 20, max_active=64)
    try:
        alone = []
        for r in reqs:
            t = ba.ba_server_submit(srv, *r)
            ba.ba_server_wait(srv, t, 60_000)
            alone.append(ba.server_result_tensor(srv, t))
            ba.ba_server_release(srv, t)
        tickets = [ba.ba_server_submit(srv, *r) for r in reqs]
        mixed = []
        for t in tickets:
            ba.ba_server_wait(srv, t, 60_000)
            state, lat = ba.ba_server_poll(srv, t)
            assert state == ba.BA_REQ_DONE and lat >= 0
            mixed.append(ba.server_result_tensor(srv, t))
        torch.cuda.synchronize()
        for t in tickets:
            ba.ba_server_release(srv, t)
        stats = ba.ba_server_stats_get(srv)
        assert stats["completed"] == 2 * len(reqs) and stats["bytes_in_use"] == 0
    finally:
        ba.ba_server_destroy(srv)
    for k, r in enumerate(reqs):
        want = _plain(ba, *r)
        assert torch.equal(alone[k], want), k
        assert torch.equal(mixed[k], want), k
        if k % 7 == 0 and r[5] > r[4]:
            a = r[4]
            b = min(r[5], a + 200_000)
            np.testing.assert_array_equal(mixed[k][:b - a].cpu().numpy(), oracle.edges_range(r[0], r[1], r[2], r[3], a, b))


def test_admission_waits_for_memory_and_never_hangs(ba):
    # budget for two 1M-edge requests: the third stays queued until one is released
    srv = ba.ba_server_create(memory_budget_bytes=2 * 16 * 2**20, chunk_edges=1 << 18, max_active=8)
    try:
        ts = [ba.ba_server_submit(srv, 100 + k, 2**22, 4, 0, 0, 2**20) for k in range(3)]
        ba.ba_server_wait(srv, ts[0], 60_000)
        ba.ba_server_wait(srv, ts[1], 60_000)
        with pytest.raises(ba.BAError) as e:
            ba.ba_server_wait(srv, ts[2], 300)
        assert e.value.status == ba.BA_ERR_TIMEOUT
        assert ba.ba_server_poll(srv, ts[2])[0] == ba.BA_REQ_QUEUED
        with pytest.raises(ba.BAError) as e:
            ba.ba_server_release(srv, ts[2])                 # not done yet
        assert e.value.status == ba.BA_ERR_BUSY
        ba.ba_server_release(srv, ts[0])
        ba.ba_server_wait(srv, ts[2], 60_000)
        got = ba.server_result_tensor(srv, ts[2])
        assert torch.equal(got, _plain(ba, 102, 2**22, 4, 0, 0, 2**20))
        with pytest.raises(ba.BAError) as e:
            ba.ba_server_submit(srv, 1, 2**22, 4, 0, 0, 2**21 + 1)   # larger than the budget
        assert e.value.status == ba.BA_ERR_NOMEM
        with pytest.raises(ba.BAError) as e:
            ba.ba_server_poll(srv, 10**9)
        assert e.value.status == ba.BA_ERR_NOT_FOUND
    finally:
        ba.ba_server_destroy(srv)


def test_full_admission_queue_answers_busy(ba):
    # budget for one 1M-edge request and room for one waiting request: A runs (and holds the
    # budget until released), B waits, C is turned away until the queue has room again
    srv = ba.ba_server_create(memory_budget_bytes=16 * 2**20, chunk_edges=1 << 18, max_active=4,
                              max_queued=1)
    try:
        a = ba.ba_server_submit(srv, 200, 2**22, 4, 0, 0, 2**20)
        ba.ba_server_wait(srv, a, 60_000)
        b = ba.ba_server_submit(srv, 201, 2**22, 4, 0, 2**20, 2**21)
        with pytest.raises(ba.BAError) as e:
            ba.ba_server_submit(srv, 202, 2**22, 4, 0, 0, 2**20)
        assert e.value.status == ba.BA_ERR_BUSY
        empty = ba.ba_server_submit(srv, 203, 2**22, 4, 0, 5, 5)   # nothing to queue: done at once
        assert ba.ba_server_poll(srv, empty)[0] == ba.BA_REQ_DONE
        assert ba.ba_server_stats_get(srv)["rejected_busy"] == 1
        ba.ba_server_release(srv, a)
        ba.ba_server_wait(srv, b, 60_000)
        assert torch.equal(ba.server_result_tensor(srv, b), _plain(ba, 201, 2**22, 4, 0, 2**20, 2**21))
        ba.ba_server_release(srv, b)
        c = ba.ba_server_submit(srv, 202, 2**22, 4, 0, 0, 2**20)
        ba.ba_server_wait(srv, c, 60_000)
        assert torch.equal(ba.server_result_tensor(srv, c), _plain(ba, 202, 2**22, 4, 0, 0, 2**20))
    finally:
        ba.ba_server_destroy(srv)


def test_autotuner_picks_a_valid_shape_and_output_is_unchanged(ba):
    n, d = 2**20, 8
    m = n * d
    scratch = torch.empty((m, 2), dtype=torch.int64, device="cuda")
    before = _plain(ba, 3, n, d, 0, 0, m).clone()
    shape = ba.ba_tune(ba.BA_KIND_GENERATE, 3, n, d, 0, 0, m, scratch)
    assert shape["block"] % 32 == 0
    assert ba.ba_get_tuning(ba.BA_KIND_GENERATE, m) == shape
    assert torch.equal(_plain(ba, 3, n, d, 0, 0, m), before)
    dshape = ba.ba_tune(ba.BA_KIND_DEGREE, 3, n, d, 0, m // 2, m)
    assert dshape["block"] % 32 == 0
    bshape = ba.ba_tune(ba.BA_KIND_BATCH, 3, n, d, 0, 0, m, scratch)
    assert bshape["block"] % 32 == 0
    assert torch.equal(_plain(ba, 3, n, d, 0, 0, m), before)


def test_poisson_trace_sampled_one_percent_exact_against_oracle(ba):
    # The serving workload's shape (Poisson 2000 req/s, n log-uniform 1e4..1e9, d in
    # {2,..,32}, 1e4..1e8 edges) for 3 s of arrivals in real time; a seeded 1 % of the
    # requests is copied out of the server before release and checked against the oracle
    # (in full up to 2e6 edges, else on its first, middle and last 10^5 edges).
    import threading
    import time
    from oracle import parallel as opar
    trace = W.serving_trace(rate=2000.0, duration=3.0, trace_seed=17)
    pick = set(int(k) for k in np.random.Generator(np.random.PCG64(19)).choice(
        len(trace), size=len(trace) // 100, replace=False))
    srv = ba.ba_server_create(memory_budget_bytes=64 << 30, chunk_edges=1 << 24, max_active=256)
    tickets = [None] * len(trace)
    kept = {}
    try:
        def submit():
            t0 = time.perf_counter()
            for k, r in enumerate(trace):
                delay = r.t_arrival - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                tickets[k] = ba.ba_server_submit(srv, r.graph.seed, r.graph.n, r.graph.d, 0,
                                                 r.edge_begin, r.edge_end)
        th = threading.Thread(target=submit)
        th.start()
        for k, r in enumerate(trace):
            while tickets[k] is None:
                time.sleep(0.0005)
            ba.ba_server_wait(srv, tickets[k], 600_000)
            if k in pick:
                res = ba.server_result_tensor(srv, tickets[k])
                ln = r.edge_end - r.edge_begin
                spans = [(0, ln)] if ln <= 2_000_000 else \
                    [(0, 100_000), (ln // 2, ln // 2 + 100_000), (ln - 100_000, ln)]
                kept[k] = [(lo, hi, res[lo:hi].cpu().numpy()) for lo, hi in spans]
            ba.ba_server_release(srv, tickets[k])
        th.join()
        assert ba.ba_server_stats_get(srv)["bytes_in_use"] == 0
    finally:
        ba.ba_server_destroy(srv)
    assert len(kept) == len(pick) >= 50
    for k, spans in kept.items():
        r = trace[k]
        for lo, hi, got in spans:
            np.testing.assert_array_equal(
                got, opar.edges_range(r.graph.seed, r.graph.n, r.graph.d, 0,
                                      r.edge_begin + lo, r.edge_begin + hi))


def test_cancel_withdraws_only_queued_requests(ba):
    # a budget of one request's output: the second and third requests queue behind the first
    n, d = 2**22, 4
    big = (1, n, d, 0, 0, 4 * 2**20)
    srv = ba.ba_server_create(memory_budget_bytes=16 * 4 * 2**20, chunk_edges=1 << 18,
                              max_active=8)
    try:
        t1 = ba.ba_server_submit(srv, *big)
        ba.ba_server_wait(srv, t1, 60_000)           # done, its buffer still held
        t2 = ba.ba_server_submit(srv, 2, n, d, 0, 100, 100 + 2**20)
        t3 = ba.ba_server_submit(srv, 3, n, d, 0, 7, 7 + 2**20)
        state2, _ = ba.ba_server_poll(srv, t2)
        assert state2 == ba.BA_REQ_QUEUED            # no room until t1 is released
        ba.ba_server_cancel(srv, t2)
        with pytest.raises(ba.BAError) as e:
            ba.ba_server_poll(srv, t2)
        assert e.value.status == ba.BA_ERR_NOT_FOUND
        with pytest.raises(ba.BAError) as e:         # finished: released, not withdrawn
            ba.ba_server_cancel(srv, t1)
        assert e.value.status == ba.BA_ERR_BUSY
        with pytest.raises(ba.BAError) as e:
            ba.ba_server_cancel(srv, 10**9)
        assert e.value.status == ba.BA_ERR_NOT_FOUND
        r1 = ba.server_result_tensor(srv, t1)
        ba.ba_server_release(srv, t1)                # frees room: t3 runs now
        ba.ba_server_wait(srv, t3, 60_000)
        r3 = ba.server_result_tensor(srv, t3)
        ba.ba_server_release(srv, t3)
        st = ba.ba_server_stats_get(srv)
        assert st["cancelled"] == 1 and st["completed"] == 2 and st["bytes_in_use"] == 0
    finally:
        ba.ba_server_destroy(srv)
    assert torch.equal(r1, _plain(ba, *big))
    assert torch.equal(r3, _plain(ba, 3, n, d, 0, 7, 7 + 2**20))
