"""Seeded synthetic workloads (parameters only; none of the method's arithmetic).

The paper's workloads are defined by their parameters alone (n, d, n0 and the hash seed;
section 3 uses n = 10^13, m = 100 n), so these generators stand in for them completely.
Both the CUDA path's tests/benchmark and the oracle take their inputs from here.

* ``PLAIN_SMALL``   n = 10^6,  d = 4,   seed 1   (4e6 edges, full edge list)
* ``PLAIN_LARGE``   n = 2^27,  d = 16,  seed 42  (2^31 edges, 34.4 GB of int64 pairs)
* ``STREAM_HUGE``   n = 10^10, d = 100, seed 7   (10^12 edges, degree count only; the
                    section 3 experiment, n = 10^13, scaled down 1000x)
* ``batch_table``   4096 graphs, seed 1000+g, n log-uniform on [10^3, 10^7],
                    d uniform on 1..32, even g: clique seed graph of n0 = d+1 nodes
* ``serving_trace`` Poisson arrivals of edge-range requests
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Graph:
    seed: int
    n: int
    d: int
    n0: int = 0

    @property
    def m0(self) -> int:
        return self.n0 * (self.n0 - 1) // 2 if self.n0 > 0 else 0

    @property
    def m(self) -> int:
        return self.m0 + (self.n - self.n0) * self.d


PLAIN_SMALL = Graph(seed=1, n=10**6, d=4)
PLAIN_LARGE = Graph(seed=42, n=2**27, d=16)
STREAM_HUGE = Graph(seed=7, n=10**10, d=100)
DEGREE_NODE_LIMIT = 100_000

# Edge ranges of 10^7 edges at the start, middle and end of PLAIN_LARGE.
PLAIN_LARGE_SPOT_RANGES = [(0, 10**7), (2**30 - 5 * 10**6, 2**30 + 5 * 10**6),
                           (2**31 - 10**7, 2**31)]


def batch_table(G: int = 4096, table_seed: int = 20160223, n_lo: float = 1e3,
                n_hi: float = 1e7, d_max: int = 32) -> list[Graph]:
    """G graphs: seed 1000+g, n = floor(10^(log10 n_lo + u log10(n_hi/n_lo))), d uniform on
    1..d_max; even g gets the clique seed graph on n0 = d+1 nodes, odd g none."""
    rng = np.random.Generator(np.random.PCG64(table_seed))
    u = rng.random(G)
    d = rng.integers(1, d_max + 1, size=G)
    lo, hi = np.log10(n_lo), np.log10(n_hi)
    graphs = []
    for g in range(G):
        n = int(np.floor(10 ** (lo + (hi - lo) * u[g])))
        dg = int(d[g])
        n0 = dg + 1 if g % 2 == 0 else 0
        n = max(n, n0)
        graphs.append(Graph(seed=1000 + g, n=n, d=dg, n0=n0))
    return graphs


@dataclass(frozen=True)
class Request:
    t_arrival: float      # seconds since the start of the trace
    graph: Graph
    edge_begin: int
    edge_end: int


def serving_trace(rate: float = 2000.0, duration: float = 60.0, trace_seed: int = 5,
                  n_lo: float = 1e4, n_hi: float = 1e9, len_lo: float = 1e4,
                  len_hi: float = 1e8, degrees=(2, 4, 8, 16, 32)) -> list[Request]:
    """Poisson arrivals at ``rate``/s for ``duration`` s of edge-range requests: a drawn
    hash seed, n log-uniform on [n_lo, n_hi], d from ``degrees``, n0 = 0, a range length
    log-uniform on [len_lo, len_hi] clipped to m, and a start uniform on 0..m-len."""
    rng = np.random.Generator(np.random.PCG64(trace_seed))
    reqs = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        seed = int(rng.integers(0, 2**63))
        n = int(10 ** rng.uniform(np.log10(n_lo), np.log10(n_hi)))
        d = int(rng.choice(degrees))
        m = n * d
        length = min(int(10 ** rng.uniform(np.log10(len_lo), np.log10(len_hi))), m)
        a = int(rng.integers(0, m - length + 1))
        reqs.append(Request(t, Graph(seed, n, d, 0), a, a + length))
    return reqs
