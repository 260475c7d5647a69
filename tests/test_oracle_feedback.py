"""Pins for the oracle's Psi (Eq. 4), next active set (Eq. 5) and Algorithm 1."""
import numpy as np
import pytest
from scipy import stats

from conftest import tiny_graph


def test_psi_identical_and_orthogonal_rows(orc):
    g = tiny_graph("star4")  # 0 - {1, 2, 3}
    phi = np.zeros((4, 4))
    phi[0] = [1, 2, 3, 4]
    phi[1] = phi[2] = phi[3] = phi[0] * 3.5
    assert abs(orc.psi_node(g.offsets, g.cols, phi, 8, 0, 0, 0) - 1.0) < 1e-15
    phi[1:] = [[-4, 3, -2, 1.0 / 1]] * 3  # orthogonal: -4 + 6 - 6 + 4 = 0
    assert orc.psi_node(g.offsets, g.cols, phi, 8, 0, 0, 0) == 0.0
    phi[1] = 0  # zero norm contributes cos 0
    phi[2] = phi[3] = phi[0]
    assert abs(orc.psi_node(g.offsets, g.cols, phi, 8, 0, 0, 0) - 2.0 / 3.0) < 1e-15


def _cos_mean(phi, v, nbrs):
    a = phi[v]
    cs = []
    for u in nbrs:
        b = phi[u]
        na, nb = np.linalg.norm(a), np.linalg.norm(b)
        cs.append(0.0 if na == 0 or nb == 0 else float(a @ b) / (na * nb))
    return float(np.mean(cs))


def test_psi_full_neighbourhood_when_degree_small(orc):
    from paper_2606_22180_b300 import inputs

    g, _ = inputs.workload_sbm1000(0)
    rng = np.random.default_rng(0)
    phi = rng.normal(size=(g.n, 48))
    deg = g.degrees()
    for v in np.nonzero((deg > 0) & (deg <= 8))[0][:50]:
        nb = g.cols[g.offsets[v]:g.offsets[v + 1]]
        assert abs(orc.psi_node(g.offsets, g.cols, phi, 8, 3, 1, v) - _cos_mean(phi, v, nb)) < 1e-12


def test_psi_subset_is_uniform_without_replacement(orc):
    deg, ks = 13, 5
    hist = np.zeros(deg)
    trials = 8000
    pair_hist = {}
    for v in range(trials):
        s = orc.psi_subset(deg, ks, 21, v, 2)
        assert len(set(s.tolist())) == ks
        assert (np.diff(s) > 0).all() and s.min() >= 0 and s.max() < deg
        hist[s] += 1
        key = (int(s[0]), int(s[1]))
        pair_hist[key] = pair_hist.get(key, 0) + 1
    # each position included with probability ks/deg
    assert stats.chisquare(hist, np.full(deg, trials * ks / deg)).pvalue > 1e-4


def test_psi_sampled_subset_mean(orc):
    from paper_2606_22180_b300 import inputs

    g = inputs.rmat(10, 8, seed=3)
    rng = np.random.default_rng(1)
    phi = rng.normal(size=(g.n, 40))
    deg = g.degrees()
    for v in np.nonzero(deg > 8)[0][:40]:
        sub = orc.psi_subset(int(deg[v]), 8, 4, int(v), 6)
        nb = g.cols[g.offsets[v] + sub]
        assert abs(orc.psi_node(g.offsets, g.cols, phi, 8, 4, 6, v) - _cos_mean(phi, v, nb)) < 1e-12


def test_feedback_rules(orc):
    from paper_2606_22180_b300 import inputs

    g = inputs.rmat(9, 8, seed=5)
    rng = np.random.default_rng(2)
    phi = rng.normal(size=(g.n, 32)) + 0.8  # mean cosine around 0.5
    live = (g.degrees() > 0).astype(np.uint8)
    active = live * (rng.random(g.n) < 0.6).astype(np.uint8)
    psi, nxt, cnt = orc.feedback(g.offsets, g.cols, phi, active, True, 0.65, 8, False, 1, 3)
    assert cnt == nxt.sum()
    assert np.all(nxt <= active)  # V_a^{r+1} is a subset of V_a^r (Eq. 5)
    ev = active.astype(bool)
    assert np.all(np.isnan(psi[~ev]))
    assert np.array_equal(nxt[ev].astype(bool), psi[ev] < 0.65)
    # reactivation reading: every non-isolated node is evaluated
    psi_r, nxt_r, _ = orc.feedback(g.offsets, g.cols, phi, active, True, 0.65, 8, True, 1, 3)
    assert np.array_equal(~np.isnan(psi_r), live.astype(bool))
    assert np.array_equal(psi_r[ev], psi[ev])
    # feedback off (the plain method): every non-isolated node stays active
    _, nxt_off, cnt_off = orc.feedback(g.offsets, g.cols, phi, active, False, 0.65, 8, False, 1, 3)
    assert np.array_equal(nxt_off, live) and cnt_off == live.sum()
    # a threshold above every cosine keeps all evaluated nodes (mu = 1 vs w/o-FeeST)
    _, nxt_hi, _ = orc.feedback(g.offsets, g.cols, phi, live, True, 1.0 + 1e-9, 8, False, 1, 3)
    assert np.array_equal(nxt_hi, live)


def test_algorithm1_token_counter_and_termination(orc):
    from paper_2606_22180_b300 import inputs

    g, _ = inputs.workload_sbm1000(0)
    L = 20
    _, _, st = orc.embed(g.offsets, g.cols, L, 1, 16, 3, 3, 0.025, True, 0.995, 8, 6, False, 2)
    # tokens of round r = |V_a^r| * L; next round starts from the surviving set
    assert np.array_equal(st[:, 1], st[:, 0] * L)
    assert np.array_equal(st[1:, 0], st[:-1, 3])
    assert np.all(np.diff(st[:, 0]) <= 0)
    if st.shape[0] < 6:
        assert st[-1, 3] == 0  # stopped because the active set emptied


def test_lagged_feedback_option(orc):
    """feedback_lag = 1 (V_a^{r+1} decided on the table as round r's training
    starts): with feedback off it changes nothing; with feedback on, the first
    decision is Eq. 5 applied to Psi of the untrained (initial) table, and the
    active sets still shrink monotonically."""
    from paper_2606_22180_b300 import inputs

    g = inputs.rmat(10, 8, seed=3)
    args = (g.offsets, g.cols, 12, 1, 16, 3, 3, 0.025)
    a0 = orc.embed(*args, False, 0.9, 8, 4, False, 5, mode="minibatch", B=500, feedback_lag=0)
    a1 = orc.embed(*args, False, 0.9, 8, 4, False, 5, mode="minibatch", B=500, feedback_lag=1)
    for x, y in zip(a0, a1):
        assert np.array_equal(x, y)
    mu = 0.5
    _, _, st = orc.embed(*args, True, mu, 8, 5, False, 5, mode="minibatch", B=500, feedback_lag=1)
    _, _, st0 = orc.embed(*args, True, mu, 8, 5, False, 5, mode="minibatch", B=500, feedback_lag=0)
    live = (g.degrees() > 0).astype(np.uint8)
    ri, _ = orc.init_tables(g.n, 16, 5)
    psi, nxt, cnt = orc.feedback(g.offsets, g.cols, ri, live, True, mu, 8, False, 5, 0)
    assert st[0, 3] == cnt and st[1, 0] == cnt
    assert st0[0, 3] != cnt  # the trained table decides differently: the option is visible
    assert all(st[r + 1, 0] <= st[r, 0] for r in range(st.shape[0] - 1))
