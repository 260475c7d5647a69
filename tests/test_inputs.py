"""The seeded input generators (host only): every graph is a valid
undirected CSR (rows sorted, no duplicates, no self loops, symmetric), the
same seed gives the same graph, the link split holds out edges and draws
non-edges, and the multi-graph mix does not depend on how many worker
processes build it."""
import numpy as np
import pytest

from paper_2606_22180_b300 import inputs


def _check_csr(g):
    off, cols = g.offsets.astype(np.int64), g.cols.astype(np.int64)
    assert off[0] == 0 and off[-1] == cols.shape[0] and np.all(np.diff(off) >= 0)
    assert cols.shape[0] == 0 or (cols.min() >= 0 and cols.max() < g.n)
    rows = np.repeat(np.arange(g.n), np.diff(off))
    assert np.all(rows != cols)  # loop-free
    for v in range(g.n):
        r = cols[off[v]:off[v + 1]]
        assert np.all(np.diff(r) > 0)  # sorted, no duplicates
    fwd = np.sort(rows * g.n + cols)
    bwd = np.sort(cols * g.n + rows)
    assert np.array_equal(fwd, bwd)  # symmetric


@pytest.mark.parametrize("make", [
    lambda: inputs.sbm(600, 6, 0.05, 0.004, seed=3)[0],
    lambda: inputs.rmat(10, 8, seed=4),
    lambda: inputs.rmat_nodes(700, 12.0, seed=5),
    lambda: inputs.sbm_degree(800, 4, 10.0, seed=6),
])
def test_generators_give_valid_undirected_csr_and_are_seeded(make):
    g1, g2 = make(), make()
    _check_csr(g1)
    assert np.array_equal(g1.offsets, g2.offsets) and np.array_equal(g1.cols, g2.cols)


def test_rmat_nodes_keeps_the_requested_size():
    g = inputs.rmat_nodes(700, 12.0, seed=5)
    assert g.n == 700
    assert 4.0 < g.nnz / g.n < 30.0


def test_link_split_holds_out_edges_and_draws_non_edges():
    g, _ = inputs.sbm(800, 8, 0.05, 0.003, seed=9)
    sp = inputs.link_split(g, 0.1, seed=2)
    _check_csr(sp.train)
    m = g.nnz // 2
    assert sp.pos.shape == (int(round(0.1 * m)), 2) and sp.neg.shape == sp.pos.shape
    full = set(zip(*np.nonzero(_dense(g))))
    train = set(zip(*np.nonzero(_dense(sp.train))))
    for u, v in sp.pos:
        assert (u, v) in full and (u, v) not in train
    for u, v in sp.neg:
        assert u != v and (u, v) not in full
    assert sp.train.nnz == g.nnz - 2 * sp.pos.shape[0]


def _dense(g):
    a = np.zeros((g.n, g.n), dtype=bool)
    rows = np.repeat(np.arange(g.n), g.degrees())
    a[rows, g.cols] = True
    return a


def test_graph_mix_is_the_same_for_any_worker_count():
    a = inputs.graph_mix(6, 11, 500, 3000)
    b = inputs.graph_mix(6, 11, 500, 3000, workers=2)
    assert [d for _, d in a] == [d for _, d in b]
    for (ga, _), (gb, _) in zip(a, b):
        assert np.array_equal(ga.offsets, gb.offsets) and np.array_equal(ga.cols, gb.cols)
        _check_csr(ga)
        assert 500 <= ga.n <= 3000
