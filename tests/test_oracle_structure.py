"""Pins for the oracle's edge array: closed forms the paper fixes (sections 1, 2 and 4).

* E[2i] is the owner of edge i: floor(i/d) for an empty seed graph, so every node gets
  exactly d edges (section 2); with a seed clique the new nodes start at n0 (section 4).
* E[2i+1] copies an earlier position, so the target is never larger than the source.
* The degree sum is 2m; the seed clique gives every seed node n0-1 seed edges.
* The recomputation form (Fig. 1) and the stored array agree on every range, and the
  result does not depend on how the edge range is split (section 2, reproducibility).
"""
import itertools

import numpy as np
import pytest

import oracle

CASES = [(1, 1000, 1, 0), (2, 1000, 4, 0), (3, 5000, 3, 0), (4, 777, 7, 0),
         (5, 1000, 4, 5), (6, 3000, 2, 3), (7, 500, 32, 33), (8, 200, 5, 1),
         (9, 64, 1, 2), (10, 40, 3, 40)]


def test_num_edges_closed_form_and_invalid_parameters():
    assert oracle.num_edges(10**6, 4, 0) == 4 * 10**6
    assert oracle.num_edges(2**27, 16, 0) == 2**31
    assert oracle.num_edges(10**10, 100, 0) == 10**12
    assert oracle.num_edges(10, 3, 4) == 6 + 6 * 3
    assert oracle.num_edges(5, 2, 5) == 10
    assert oracle.num_edges(0, 1, 0) == 0
    assert oracle.num_edges(10, 0, 0) == 0
    assert oracle.num_edges(10, 1, 11) == 0
    assert oracle.num_edges(2**62, 1, 0) == 2**62
    assert oracle.num_edges(2**62 + 1, 1, 0) == 0
    with pytest.raises(ValueError):
        oracle.edges_range(1, 10, 1, 0, 5, 11)


@pytest.mark.parametrize("seed,n,d,n0", CASES)
def test_source_column_and_d_edges_per_node(seed, n, d, n0):
    E = oracle.bb_array(seed, n, d, n0)
    m0 = n0 * (n0 - 1) // 2
    m = m0 + (n - n0) * d
    assert E.size == 2 * m
    i = np.arange(m0, m)
    np.testing.assert_array_equal(E[2 * i], n0 + (i - m0) // d)
    owners = np.bincount(E[2 * m0::2], minlength=n)
    assert (owners[n0:] == d).all() and (owners[:n0] == 0).all()


@pytest.mark.parametrize("seed,n,d,n0", CASES)
def test_target_never_exceeds_source_and_ids_in_range(seed, n, d, n0):
    E = oracle.bb_array(seed, n, d, n0).reshape(-1, 2)
    assert (E[:, 1] <= E[:, 0]).all()
    assert E.min() >= 0 and E.max() < n


@pytest.mark.parametrize("seed,n,d,n0", CASES)
def test_degree_sum_is_twice_the_edge_count(seed, n, d, n0):
    E = oracle.bb_array(seed, n, d, n0)
    deg = oracle.degrees_of_array(E, n)
    assert int(deg.sum()) == E.size
    # isolated node 0 when the seed graph is a single node (no seed edges to attach to)
    if n0 == 1:
        assert deg[0] == 0


def test_first_d_edges_of_an_empty_seed_graph_are_loops_at_node_0():
    for d in (1, 4, 16):
        E = oracle.bb_array(123, 100, d, 0).reshape(-1, 2)
        np.testing.assert_array_equal(E[:d], 0)


@pytest.mark.parametrize("n0", [2, 3, 5, 9])
def test_seed_prefix_is_the_clique_in_v_major_order(n0):
    d = 3
    E = oracle.bb_array(17, n0 + 20, d, n0).reshape(-1, 2)
    m0 = n0 * (n0 - 1) // 2
    expected = [(v, u) for v in range(1, n0) for u in range(v)]
    np.testing.assert_array_equal(E[:m0], np.array(expected).reshape(-1, 2))
    # a graph that is only the seed clique: every node has degree n0-1
    C = oracle.bb_array(17, n0, d, n0)
    assert (oracle.degrees_of_array(C, n0) == n0 - 1).all()


@pytest.mark.parametrize("seed,n,d,n0", CASES)
def test_recomputation_equals_stored_array(seed, n, d, n0):
    E = oracle.bb_array(seed, n, d, n0).reshape(-1, 2)
    m = E.shape[0]
    np.testing.assert_array_equal(oracle.edges_range(seed, n, d, n0, 0, m), E)
    rng = np.random.default_rng(seed)
    for _ in range(5):
        a, b = sorted(int(x) for x in rng.integers(0, m + 1, size=2))
        np.testing.assert_array_equal(oracle.edges_range(seed, n, d, n0, a, b), E[a:b])


@pytest.mark.parametrize("seed,n,d,n0", CASES[:6])
def test_degree_count_range_equals_array_degrees_and_splits_add_up(seed, n, d, n0):
    E = oracle.bb_array(seed, n, d, n0)
    m = E.size // 2
    for limit in (1, 10, n, n + 7):
        full = oracle.degree_count_range(seed, n, d, n0, 0, m, limit)
        np.testing.assert_array_equal(full, oracle.degrees_of_array(E, limit))
        cuts = sorted({0, m, m // 3, m // 2, (2 * m) // 3})
        acc = np.zeros(limit, dtype=np.uint64)
        for a, b in itertools.pairwise(cuts):
            oracle.degree_count_range(seed, n, d, n0, a, b, limit, acc)
        np.testing.assert_array_equal(acc, full)


def test_same_seed_same_graph_other_seed_other_graph():
    a = oracle.bb_array(5, 2000, 3, 0)
    b = oracle.bb_array(5, 2000, 3, 0)
    c = oracle.bb_array(6, 2000, 3, 0)
    np.testing.assert_array_equal(a, b)
    assert (a != c).any()


def test_graph_prefix_does_not_depend_on_n():
    # n only says where the generation stops: the first edges are the same for any n.
    small = oracle.bb_array(9, 300, 4, 0)
    large = oracle.bb_array(9, 5000, 4, 0)
    np.testing.assert_array_equal(small, large[:small.size])


def test_self_loops_occur():
    # x is drawn from 0..2i including 2i, the edge's own first end point (section 2).
    E = oracle.bb_array(1, 10**5, 1, 0).reshape(-1, 2)
    loops = int((E[:, 0] == E[:, 1]).sum())
    assert loops > 5
