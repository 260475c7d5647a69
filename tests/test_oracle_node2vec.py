"""Pins for the oracle's node2vec walks (the rule of Grover and Leskovec,
KDD 2016, a Sample variant the paper names in Section 5.4).

Pinned by: the second-order transition law, checked by chi-square on every
(previous, current) pair of small graphs against weights written from the
definition (1/p back to the previous node, 1 to its neighbours, 1/q
further out); the p = q = 1 case, where every step is uniform; every step
an edge; a dead end padded with -1; a degree-1 node, where the only move
is back even when returning is unlikely; and the 64-attempt cap, which
with acceptance ratios near 1e-6 makes the step the 64th proposal,
uniform, instead of the rule's 2:1.
"""
import numpy as np
import pytest
from scipy import stats

from conftest import tiny_graph


def _graph():
    """Two triangles sharing node 2, plus a tail 4-5 and a pendant 6 on 0."""
    from paper_2606_22180_b300.inputs import csr_from_edges

    e = np.array([(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (2, 4), (4, 5), (0, 6)], np.int64)
    return csr_from_edges(7, e[:, 0], e[:, 1])


def _nbrs(g, v):
    return list(g.cols[g.offsets[v]:g.offsets[v + 1]])


def _expected(g, t, v, p, q):
    xs = _nbrs(g, v)
    w = np.array([1 / p if x == t else (1.0 if x in _nbrs(g, t) else 1 / q) for x in xs])
    return xs, w / w.sum()


@pytest.mark.parametrize("p,q", [(0.5, 2.0), (4.0, 0.25), (1.0, 1.0), (0.3, 0.3)])
def test_second_order_transition_law(orc, p, q):
    g = _graph()
    starts = np.arange(7, dtype=np.int32)
    W = np.concatenate([orc.walk_node2vec(g.offsets, g.cols, starts, 6, 600, p, q, 11, r) for r in range(4)])
    trans = {}
    for row in W:
        for i in range(2, row.size):
            if row[i] < 0:
                break
            trans.setdefault((row[i - 2], row[i - 1]), []).append(row[i])
    checked = 0
    for (t, v), nxt in trans.items():
        xs, pr = _expected(g, t, v, p, q)
        assert set(nxt) <= set(xs)  # every step an edge
        if len(xs) < 2 or len(nxt) < 400:
            continue
        obs = np.array([nxt.count(x) for x in xs])
        chi2 = stats.chisquare(obs, pr * obs.sum())
        assert chi2.pvalue > 1e-4, (t, v, obs, pr)
        checked += 1
    assert checked >= 10


def test_p_q_one_is_uniform(orc):
    g = tiny_graph("k4")
    W = orc.walk_node2vec(g.offsets, g.cols, np.arange(4, dtype=np.int32), 40, 50, 1.0, 1.0, 5, 0)
    nxt = W[:, 2:].ravel()
    cur = W[:, 1:-1].ravel()
    for v in range(4):
        obs = np.bincount(nxt[cur == v], minlength=4)
        assert obs[v] == 0
        obs = np.delete(obs, v)
        assert stats.chisquare(obs).pvalue > 1e-4


def test_dead_end_and_forced_return(orc):
    g = tiny_graph("with_isolated")  # 0-1-2 path, 3 and 4 isolated
    W = orc.walk_node2vec(g.offsets, g.cols, np.array([3, 0], np.int32), 6, 1, 1000.0, 1.0, 2, 0)
    assert list(W[0]) == [3, -1, -1, -1, -1, -1]
    # 0 has one neighbour: every step from 0 or 2 must go back to 1
    assert list(W[1]) == [0, 1, W[1, 2], 1, W[1, 4], 1]
    assert set(W[1, [2, 4]]) <= {0, 2}


def test_attempt_cap_takes_the_64th_proposal(orc):
    """Path 0-1-2 with p = 1e6, q = 2e6: at node 1 every proposal is accepted
    with probability 1e-6 (back) or 5e-7 (further out), so nearly every step
    exhausts the 64 attempts and takes the last proposal, uniform over {0, 2}.
    The uncapped rule would give 2:1 towards the previous node."""
    from paper_2606_22180_b300.inputs import csr_from_edges

    e = np.array([(0, 1), (1, 2)], np.int64)
    g = csr_from_edges(3, e[:, 0], e[:, 1])
    W = orc.walk_node2vec(g.offsets, g.cols, np.array([0], np.int32), 40, 2000, 1e6, 2e6, 17, 0)
    back = fwd = 0
    for row in W:
        for i in range(2, row.size):
            if row[i - 1] == 1:
                if row[i] == row[i - 2]:
                    back += 1
                else:
                    fwd += 1
    n = back + fwd
    assert n > 30000
    assert stats.chisquare([back, fwd], [n / 2, n / 2]).pvalue > 1e-4
    assert stats.chisquare([back, fwd], [2 * n / 3, n / 3]).pvalue < 1e-12
