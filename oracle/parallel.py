"""Runs the oracle over large edge ranges on several host cores -- TEST INFRASTRUCTURE.

The range is cut into contiguous pieces, each evaluated by the single-threaded oracle in
its own process (``spawn`` start method, so it is safe after CUDA has been initialised in
the parent), and the pieces are concatenated or summed.  This is only a harness around
the oracle: the arithmetic stays in ``ba_oracle.c``.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

import oracle


def _edges_piece(args):
    seed, n, d, n0, a, b = args
    return oracle.edges_range(seed, n, d, n0, a, b)


def _degrees_piece(args):
    seed, n, d, n0, a, b, limit = args
    return oracle.degree_count_range(seed, n, d, n0, a, b, limit)


def _variant_edges_piece(args):
    seed, n, d, n0, family, no_loops, a, b = args
    return oracle.edges_range_variant(seed, n, d, n0, family, no_loops, a, b)


def _variant_degrees_piece(args):
    seed, n, d, n0, family, no_loops, a, b, limit = args
    return oracle.degree_count_range_variant(seed, n, d, n0, family, no_loops, a, b, limit)


def default_workers() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def _cuts(a: int, b: int, pieces: int) -> list[tuple[int, int]]:
    pieces = max(1, min(pieces, b - a)) if b > a else 1
    bounds = [a + (b - a) * k // pieces for k in range(pieces + 1)]
    return list(zip(bounds[:-1], bounds[1:]))


def edges_range(seed, n, d, n0, a, b, workers: int | None = None) -> np.ndarray:
    """oracle.edges_range over [a, b), split across processes."""
    workers = workers or default_workers()
    if workers == 1 or b - a < 20_000_000:
        return oracle.edges_range(seed, n, d, n0, a, b)
    oracle.build()
    jobs = [(seed, n, d, n0, x, y) for x, y in _cuts(a, b, 4 * workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_edges_piece, jobs)
    return np.concatenate(parts, axis=0)


def degree_count_range(seed, n, d, n0, a, b, limit, workers: int | None = None) -> np.ndarray:
    """oracle.degree_count_range over [a, b), split across processes and summed."""
    workers = workers or default_workers()
    if workers == 1 or b - a < 20_000_000:
        return oracle.degree_count_range(seed, n, d, n0, a, b, limit)
    oracle.build()
    jobs = [(seed, n, d, n0, x, y, limit) for x, y in _cuts(a, b, 4 * workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_degrees_piece, jobs)
    return np.sum(parts, axis=0, dtype=np.uint64)


def edges_range_variant(seed, n, d, n0, family, no_loops, a, b,
                        workers: int | None = None) -> np.ndarray:
    """oracle.edges_range_variant over [a, b), split across processes."""
    workers = workers or default_workers()
    if workers == 1 or b - a < 4_000_000:
        return oracle.edges_range_variant(seed, n, d, n0, family, no_loops, a, b)
    oracle.build()
    jobs = [(seed, n, d, n0, family, no_loops, x, y) for x, y in _cuts(a, b, 4 * workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_variant_edges_piece, jobs)
    return np.concatenate(parts, axis=0)


def degree_count_range_variant(seed, n, d, n0, family, no_loops, a, b, limit,
                               workers: int | None = None) -> np.ndarray:
    """oracle.degree_count_range_variant over [a, b), split across processes and summed."""
    workers = workers or default_workers()
    if workers == 1 or b - a < 4_000_000:
        return oracle.degree_count_range_variant(seed, n, d, n0, family, no_loops, a, b, limit)
    oracle.build()
    jobs = [(seed, n, d, n0, family, no_loops, x, y, limit)
            for x, y in _cuts(a, b, 4 * workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_variant_degrees_piece, jobs)
    return np.sum(parts, axis=0, dtype=np.uint64)


def _simple_edges_piece(args):
    seed, n, d, n0, no_loops, a, b = args
    return oracle.edges_range_simple(seed, n, d, n0, no_loops, a, b)


def edges_range_simple(seed, n, d, n0, no_loops, a, b, workers: int | None = None) -> np.ndarray:
    """oracle.edges_range_simple (no parallel edges) over [a, b), split across processes;
    each piece recomputes the node it starts inside, so any cut gives the same edges."""
    workers = workers or default_workers()
    if workers == 1 or b - a < 4_000_000:
        return oracle.edges_range_simple(seed, n, d, n0, no_loops, a, b)
    oracle.build()
    jobs = [(seed, n, d, n0, no_loops, x, y) for x, y in _cuts(a, b, 4 * workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_simple_edges_piece, jobs)
    return np.concatenate(parts, axis=0)


def _simple_degrees_piece(args):
    seed, n, d, n0, no_loops, a, b, limit = args
    return oracle.degree_count_range_simple(seed, n, d, n0, no_loops, a, b, limit)


def degree_count_range_simple(seed, n, d, n0, no_loops, a, b, limit,
                              workers: int | None = None) -> np.ndarray:
    """oracle.degree_count_range_simple over [a, b), split across processes and summed."""
    workers = workers or default_workers()
    if workers == 1 or b - a < 4_000_000:
        return oracle.degree_count_range_simple(seed, n, d, n0, no_loops, a, b, limit)
    oracle.build()
    jobs = [(seed, n, d, n0, no_loops, x, y, limit) for x, y in _cuts(a, b, 4 * workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_simple_degrees_piece, jobs)
    return np.sum(parts, axis=0, dtype=np.uint64)
