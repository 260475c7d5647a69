"""Pins for the oracle's uniform truncated walks (Section 2; Algorithm 1, Sampling).

Brute force: every length-L path from a start has probability prod 1/deg; the
sampled walk frequencies must match it.  Stationarity: on a connected
non-bipartite undirected graph the position of a long walk tends to
deg(v) / 2|E|.
"""
import itertools

import numpy as np
import pytest
from scipy import stats

from conftest import tiny_graph


def _path_probs(g, s, L):
    deg = g.degrees()
    probs = {}

    def rec(path, p):
        if len(path) == L:
            probs[tuple(path)] = p
            return
        v = path[-1]
        for u in g.cols[g.offsets[v]:g.offsets[v + 1]]:
            rec(path + [int(u)], p / deg[v])

    rec([s], 1.0)
    return probs


@pytest.mark.parametrize("name", ["path4", "star4", "triangle_tail", "k4", "cycle6"])
def test_path_probabilities_brute_force(orc, name):
    g = tiny_graph(name)
    L = 4
    for s in range(g.n):
        probs = _path_probs(g, s, L)
        assert abs(sum(probs.values()) - 1.0) < 1e-12
        n_walks = 40000
        W = orc.walk(g.offsets, g.cols, np.array([s]), L, n_walks, seed=7 + s, round_=0)
        keys = list(probs)
        index = {k: i for i, k in enumerate(keys)}
        hist = np.zeros(len(keys))
        for row in map(tuple, W.tolist()):
            hist[index[row]] += 1  # KeyError = an impossible path
        expect = np.array([probs[k] for k in keys]) * n_walks
        if len(keys) > 1:
            assert stats.chisquare(hist, expect).pvalue > 1e-4


def test_stationary_distribution(orc):
    for name in ["triangle_tail", "k4"]:
        g = tiny_graph(name)
        deg = g.degrees()
        pi = deg / deg.sum()
        n_walks, L = 30000, 25
        W = orc.walk(g.offsets, g.cols, np.array([0]), L, n_walks, seed=3, round_=1)
        freq = np.bincount(W[:, -1], minlength=g.n) / n_walks
        sigma = np.sqrt(pi * (1 - pi) / n_walks)
        assert np.all(np.abs(freq - pi) < 5 * sigma + 1e-3 * 0), (freq, pi)


def test_walks_follow_edges_and_order(orc):
    from paper_2606_22180_b300 import inputs

    g, _ = inputs.workload_sbm1000(0)
    starts = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
    W = orc.walk(g.offsets, g.cols, starts, 12, 2, seed=5, round_=3)
    assert W.shape == (2 * starts.shape[0], 12)
    # row j * n_starts + i starts at starts[i]
    assert np.array_equal(W[: starts.shape[0], 0], starts)
    assert np.array_equal(W[starts.shape[0]:, 0], starts)
    edges = set(zip(np.repeat(np.arange(g.n), g.degrees()).tolist(), g.cols.tolist()))
    for a, b in zip(W[:, :-1].ravel().tolist(), W[:, 1:].ravel().tolist()):
        assert (a, b) in edges
    # the two reps of a start differ (independent counters)
    assert not np.array_equal(W[: starts.shape[0]], W[starts.shape[0]:])


def test_isolated_start_pads(orc):
    g = tiny_graph("with_isolated")
    W = orc.walk(g.offsets, g.cols, np.array([3, 0]), 5, 1, seed=1, round_=0)
    assert W[0].tolist() == [3, -1, -1, -1, -1]
    assert (W[1] >= 0).all()


def test_step_keying(orc):
    """Step t of walk (round r, rep j, start s) uses Philox(x0=t, x1=s, x2=r*wpr+j, 0)."""
    g = tiny_graph("k4")
    W = orc.walk(g.offsets, g.cols, np.array([2]), 6, 3, seed=99, round_=4)
    for j in range(3):
        v = 2
        for t in range(1, 6):
            w = orc.philox(99, (t, 2, 4 * 3 + j, 0))
            u = int(w[0]) | (int(w[1]) << 32)
            deg = int(g.offsets[v + 1] - g.offsets[v])
            idx = (u * deg) >> 64
            v = int(g.cols[g.offsets[v] + idx])
            assert W[j, t] == v
