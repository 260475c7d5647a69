"""Pins for the oracle's skip-gram negative-sampling trainer (Eq. 1, Eq. 2)."""
import math

import numpy as np
import pytest

from conftest import tiny_graph


def _pair_loss(orc, in_x, outs):
    a = in_x.copy()
    o = [x.copy() for x in outs]
    return orc.pair_update(a, o, 0.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pair_gradient_matches_finite_differences(orc, seed):
    """The pair update equals eta times the gradient of the Eq. 2 log-likelihood."""
    rng = np.random.default_rng(seed)
    d, K = 4, 3
    in_x = rng.normal(size=d)
    outs = [rng.normal(size=d) for _ in range(K + 1)]
    eta = 1e-3
    a = in_x.copy()
    o = [x.copy() for x in outs]
    orc.pair_update(a, o, eta)
    g_in = -(a - in_x) / eta  # gradient of the loss (= -log-likelihood)
    g_out = [-(o[t] - outs[t]) / eta for t in range(K + 1)]
    h = 1e-6
    for i in range(d):
        e = np.zeros(d)
        e[i] = h
        fd = (_pair_loss(orc, in_x + e, outs) - _pair_loss(orc, in_x - e, outs)) / (2 * h)
        assert abs(fd - g_in[i]) <= 1e-6 * max(1.0, abs(fd))
    for t in range(K + 1):
        for i in range(d):
            e = np.zeros(d)
            e[i] = h
            op = [x.copy() for x in outs]
            om = [x.copy() for x in outs]
            op[t] = op[t] + e
            om[t] = om[t] - e
            fd = (_pair_loss(orc, in_x, op) - _pair_loss(orc, in_x, om)) / (2 * h)
            assert abs(fd - g_out[t][i]) <= 1e-6 * max(1.0, abs(fd))


def test_pair_loss_definition_points(orc):
    """-log sigma(s+) - sum log sigma(-s_k) at a few exact points."""
    d = 3
    x = np.array([1.0, 0.0, 0.0])
    c = np.array([2.0, 5.0, -1.0])  # s+ = 2
    n1 = np.array([-3.0, 1.0, 1.0])  # s1 = -3
    loss = _pair_loss(orc, x, [c, n1])
    expect = math.log1p(math.exp(-2.0)) + math.log1p(math.exp(-3.0))
    assert abs(loss - expect) < 1e-15
    # zero out-vectors: every score 0, loss (1 + K) log 2
    loss0 = _pair_loss(orc, x, [np.zeros(d)] * 4)
    assert abs(loss0 - 4 * math.log(2)) < 1e-15


def test_first_step_closed_form(orc):
    """phi_out = 0: the context row is unchanged, phi_out[c] += eta/2 phi_in[x],
    each negative row gets -eta/2 phi_in[x] (direction of Eq. 2)."""
    rng = np.random.default_rng(4)
    d = 8
    x = rng.normal(size=d)
    outs = [np.zeros(d) for _ in range(4)]
    eta = 0.025
    a = x.copy()
    orc.pair_update(a, outs, eta)
    assert np.array_equal(a, x)
    assert np.allclose(outs[0], eta / 2 * x, rtol=0, atol=1e-17)
    for t in range(1, 4):
        assert np.allclose(outs[t], -eta / 2 * x, rtol=0, atol=1e-17)


def test_learning_rate_schedule(orc):
    assert orc.learning_rate(0.025, 0, 1000) == 0.025
    assert abs(orc.learning_rate(0.025, 500, 1000) - 0.0125) < 1e-18
    assert orc.learning_rate(0.025, 1000, 1000) == 0.025 * 1e-4
    assert orc.learning_rate(0.025, 5000, 1000) == 0.025 * 1e-4


def test_init_tables(orc):
    n, d = 300, 64
    pi, po = orc.init_tables(n, d, seed=3)
    assert (po == 0).all()
    assert pi.min() >= -0.5 / d and pi.max() < 0.5 / d
    q = (pi * d + 0.5) * 2 ** 24  # integer 24-bit draws
    assert np.array_equal(q, np.round(q))
    assert abs(pi.mean()) < 0.01 / d


def _noise(orc, walks, n):
    return orc.noise_table(orc.counts(walks, n))


def _walks(orc, name="k4", L=6, wpr=3, seed=1):
    g = tiny_graph(name)
    starts = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
    return g, orc.walk(g.offsets, g.cols, starts, L, wpr, seed, 0)


def test_minibatch_from_zero_loss_closed_form(orc):
    """One batch covering the corpus with phi_out = 0: every pair reads scores
    of 0, so the loss is log 2 times the number of (pair, kept target)."""
    from paper_2606_22180_b300 import inputs

    g, _ = inputs.workload_sbm1000(0)
    starts = np.nonzero(g.degrees() > 0)[0][:60].astype(np.int32)
    L, w, K, seed = 10, 3, 4, 8
    W = orc.walk(g.offsets, g.cols, starts, L, 1, seed, 0)
    _, thr, alias, S = _noise(orc, W, g.n)
    pi, po = orc.init_tables(g.n, 16, seed)
    loss = orc.sgns_minibatch(W, g.n, 16, w, K, 0.025, 10 ** 6, W.size, thr, alias, S, seed, 0, 0,
                              pi, po)
    kept = 0
    for wi in range(W.shape[0]):
        for p in range(L):
            for o in list(range(-w, 0)) + list(range(1, w + 1)):
                if 0 <= p + o < L:
                    q = o + w if o < 0 else o + w - 1
                    kept += 1
                    for k in range(K):
                        kept += orc.draw_negative(thr, alias, S, seed, 0, wi, p, q, k) != W[wi, p]
    assert abs(loss - kept * math.log(2)) < 1e-9 * loss


def test_minibatch_single_pair_equals_serial(orc):
    """A batch holding one pair with distinct targets is the serial update."""
    g = tiny_graph("k4")
    W = np.array([[0, 1]], np.int32)  # two centers, one context each
    _, thr, alias, S = _noise(orc, np.array([[0, 1, 2, 3]], np.int32), g.n)
    rng = np.random.default_rng(2)
    pi = rng.normal(size=(4, 5))
    po = rng.normal(size=(4, 5))
    # negatives per pair: K = 1 keeps the target rows distinct
    a_in, a_out = pi.copy(), po.copy()
    b_in, b_out = pi.copy(), po.copy()
    ls = orc.sgns_serial(W, 4, 5, 1, 1, 0.05, 100, thr, alias, S, 9, 0, 0, a_in, a_out)
    lm = orc.sgns_minibatch(W, 4, 5, 1, 1, 0.05, 100, 1, thr, alias, S, 9, 0, 0, b_in, b_out)
    assert ls == lm
    assert np.array_equal(a_in, b_in) and np.array_equal(a_out, b_out)


def test_serial_training_reduces_loss_and_separates_communities(orc):
    """Plain Algorithm 1 (feedback off) on the 1,000-node planted partition:
    the per-round loss falls and held-out links score above non-links."""
    from paper_2606_22180_b300 import inputs

    g, _ = inputs.workload_sbm1000(0)
    sp = inputs.link_split(g, 0.1, 0)
    pi, po, st = orc.embed(sp.train.offsets, sp.train.cols, 40, 1, 32, 5, 5, 0.025, False, 0.65,
                           8, 4, False, 0)
    assert st.shape[0] == 4
    assert st[-1, 2] < 0.7 * st[0, 2]
    assert orc.link_auc(pi, sp.pos, sp.neg) > 0.65


def test_minibatch_tracks_serial(orc):
    """Small batches approach the serial trajectory (same pairs, same eta)."""
    from paper_2606_22180_b300 import inputs

    g, _ = inputs.workload_sbm1000(0)
    sp = inputs.link_split(g, 0.1, 0)
    args = (sp.train.offsets, sp.train.cols, 20, 1, 16, 3, 3, 0.025, False, 0.65, 8, 2, False, 1)
    s_in, _, s_st = orc.embed(*args, mode="serial")
    m_in, _, m_st = orc.embed(*args, mode="minibatch", B=8)
    assert abs(s_st[:, 2].sum() - m_st[:, 2].sum()) < 0.02 * s_st[:, 2].sum()
    cos = (s_in * m_in).sum(1) / np.linalg.norm(s_in, axis=1) / np.linalg.norm(m_in, axis=1)
    assert np.median(cos) > 0.9
