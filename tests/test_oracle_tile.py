"""Pins for the oracle's shared-negatives tile form of Eq. 2.

The tile form draws Ns negatives once per tile of T consecutive centers and
gives each weight K / Ns; a node's summed tile increment is divided by the
node's rows in the tile.  It is pinned by: the loss at phi_out = 0 (every
score 0, so the loss counts kept targets with their weights); without the
averaging, equality with the per-pair minibatch form when the noise
distribution is a point mass (then every draw of either form is the same
node) and finite differences of the tile loss (one tile updates by exactly
-eta times its gradient); the averaging against row counts taken here from
the corpus; and the frequencies of the shared draws against the
unigram^0.75 distribution.
"""
import math

import numpy as np
import pytest

from conftest import tiny_graph


def _corpus(orc, n_starts=40, L=12, seed=5):
    from paper_2606_22180_b300 import inputs

    g, _ = inputs.workload_sbm1000(0)
    starts = np.nonzero(g.degrees() > 0)[0][:n_starts].astype(np.int32)
    W = orc.walk(g.offsets, g.cols, starts, L, 1, seed, 0)
    _, thr, alias, S = orc.noise_table(orc.counts(W, g.n))
    return g, W, thr, alias, S


def _pairs(W, w):
    """(walk, center position, context position) in corpus order."""
    out = []
    L = W.shape[1]
    for wi in range(W.shape[0]):
        for p in range(L):
            if W[wi, p] < 0:
                continue
            for o in list(range(-w, 0)) + list(range(1, w + 1)):
                if 0 <= p + o < L and W[wi, p + o] >= 0:
                    out.append((wi, p, p + o))
    return out


@pytest.mark.parametrize("T,Ns", [(7, 8), (12, 6), (480, 64)])
def test_tile_loss_at_zero_out_table(orc, T, Ns):
    """phi_out = 0 and lr0 = 0 (tables stay put): every score is 0 and each
    term is log 2, so the loss is log 2 * sum over pairs of
    (1 + K/Ns * #{shared negatives != center})."""
    g, W, thr, alias, S = _corpus(orc)
    d, w, K, seed = 8, 3, 5, 11
    pi, po = orc.init_tables(g.n, d, seed)
    loss = orc.sgns_tile(W, g.n, d, w, K, 0.0, 10 ** 6, T, Ns, thr, alias, S, seed, 0, 0, pi, po)
    L = W.shape[1]
    negs = {}
    expect = 0.0
    for wi, p, _ in _pairs(W, w):
        t = (wi * L + p) // T
        if t not in negs:
            negs[t] = orc.tile_negatives(thr, alias, g.n, S, seed, 0, t, Ns)
        kept = int((negs[t] != W[wi, p]).sum())
        expect += math.log(2) * (1.0 + K / Ns * kept)
    assert abs(loss - expect) <= 1e-10 * expect  # one misweighted term is ~7e-5


@pytest.mark.parametrize("T,Ns", [(5, 6), (13, 8), (40, 3)])
def test_tile_equals_minibatch_under_point_mass_noise(orc, T, Ns):
    """With every draw forced to one node u, Ns shared draws of weight K/Ns
    and K per-pair draws of weight 1 are the same update, so the tile form
    equals the minibatch form with B = T (up to summation order)."""
    g, W, _, _, _ = _corpus(orc, n_starts=30, L=10)
    counts = orc.counts(W, g.n)
    for u in (int(np.argmax(counts)), int(W[0, 0])):  # a hub, and a node that is also a center
        thr = np.zeros(g.n, np.uint64)
        alias = np.full(g.n, u, np.int32)
        S = 12345
        d, w, K = 6, 3, 4
        rng = np.random.default_rng(u)
        pi0 = rng.normal(scale=0.3, size=(g.n, d))
        po0 = rng.normal(scale=0.3, size=(g.n, d))
        a_in, a_out = pi0.copy(), po0.copy()
        b_in, b_out = pi0.copy(), po0.copy()
        lt, tl = orc.sgns_tile(W, g.n, d, w, K, 0.05, 5000, T, Ns, thr, alias, S, 3, 0, 7, a_in,
                               a_out, per_tile=True, normalize=False)
        lm, bl = orc.sgns_minibatch(W, g.n, d, w, K, 0.05, 5000, T, thr, alias, S, 3, 0, 7, b_in,
                                    b_out, per_batch=True)
        assert tl.shape == bl.shape
        assert np.allclose(tl, bl, rtol=1e-12, atol=1e-12)
        assert abs(lt - lm) <= 1e-12 * abs(lm)
        assert np.allclose(a_in, b_in, rtol=0, atol=1e-12)
        assert np.allclose(a_out, b_out, rtol=0, atol=1e-12)
        assert not np.array_equal(a_in, pi0)


def test_tile_update_is_minus_eta_gradient(orc):
    """One tile without averaging: the update equals -eta times the gradient
    of the tile loss, checked against central differences of the loss
    (lr0 = 0 evaluates the loss without updating)."""
    g = tiny_graph("triangle_tail")
    W = np.array([[0, 1, 2, 3, 2, 0], [3, 2, 1, 0, 2, 1]], np.int32)
    _, thr, alias, S = orc.noise_table(orc.counts(W, g.n))
    d, w, K, Ns, seed = 3, 2, 3, 5, 4
    rng = np.random.default_rng(9)
    pi0 = rng.normal(scale=0.5, size=(g.n, d))
    po0 = rng.normal(scale=0.5, size=(g.n, d))
    eta = 1e-3
    T = W.size  # a single tile

    def loss_at(pi, po):
        return orc.sgns_tile(W, g.n, d, w, K, 0.0, 10 ** 9, T, Ns, thr, alias, S, seed, 0, 0,
                             pi.copy(), po.copy(), normalize=False)

    a_in, a_out = pi0.copy(), po0.copy()
    orc.sgns_tile(W, g.n, d, w, K, eta, 10 ** 9, T, Ns, thr, alias, S, seed, 0, 0, a_in, a_out,
                  normalize=False)
    grad_in = -(a_in - pi0) / eta
    grad_out = -(a_out - po0) / eta
    h = 1e-6
    for v in range(g.n):
        for i in range(d):
            e = np.zeros_like(pi0)
            e[v, i] = h
            fd_in = (loss_at(pi0 + e, po0) - loss_at(pi0 - e, po0)) / (2 * h)
            fd_out = (loss_at(pi0, po0 + e) - loss_at(pi0, po0 - e)) / (2 * h)
            assert abs(fd_in - grad_in[v, i]) <= 1e-6 * max(1.0, abs(fd_in))
            assert abs(fd_out - grad_out[v, i]) <= 1e-6 * max(1.0, abs(fd_out))


def _tile_rows(W, w, T, negs, t):
    """Rows of tile t per node: distinct context positions in a pair (phi_in)
    and distinct center positions in a pair plus negative slots (phi_out)."""
    L = W.shape[1]
    ctx, ctr = set(), set()
    for wi, p, pp in _pairs(W, w):
        if (wi * L + p) // T == t:
            ctx.add((wi, pp))
            ctr.add((wi, p))
    r_in, r_out = {}, {}
    for wi, pp in ctx:
        r_in[W[wi, pp]] = r_in.get(W[wi, pp], 0) + 1
    for wi, p in ctr:
        r_out[W[wi, p]] = r_out.get(W[wi, p], 0) + 1
    for v in negs:
        r_out[int(v)] = r_out.get(int(v), 0) + 1
    return r_in, r_out


@pytest.mark.parametrize("seed", [1, 2])
def test_tile_average_divides_by_rows_per_node(orc, seed):
    """One tile: the averaged update of a node is the summed update divided by
    the node's rows in the tile, counted here from the corpus and the draws.
    Walks that revisit nodes make several counts exceed one."""
    g = tiny_graph("star4")  # walks alternate between the hub 0 and a leaf
    rng = np.random.default_rng(seed)
    W = np.array([[0, 1, 0, 2, 0, 3, 0, 1], [2, 0, 3, 0, 1, 0, 2, 0]], np.int32)
    _, thr, alias, S = orc.noise_table(orc.counts(W, g.n))
    d, w, K, Ns = 4, 2, 3, 6
    T = W.size
    pi0 = rng.normal(scale=0.3, size=(g.n, d))
    po0 = rng.normal(scale=0.3, size=(g.n, d))
    res = {}
    for norm in (False, True):
        a_in, a_out = pi0.copy(), po0.copy()
        orc.sgns_tile(W, g.n, d, w, K, 0.05, 10 ** 6, T, Ns, thr, alias, S, seed, 0, 0, a_in, a_out,
                      normalize=norm)
        res[norm] = (a_in - pi0, a_out - po0)
    negs = orc.tile_negatives(thr, alias, g.n, S, seed, 0, 0, Ns)
    r_in, r_out = _tile_rows(W, w, T, negs, 0)
    assert max(r_in.values()) > 1 and max(r_out.values()) > 1
    for v in range(g.n):
        np.testing.assert_allclose(res[True][0][v], res[False][0][v] / r_in.get(v, 1), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(res[True][1][v], res[False][1][v] / r_out.get(v, 1), rtol=1e-12, atol=1e-15)


def test_tile_negatives_follow_unigram_three_quarter(orc):
    """Shared draws over many tiles match Pn(u) ~ count^0.75 (Eq. 2's noise
    distribution) by a chi-square bound, and differ between tiles/rounds."""
    counts = np.array([1, 4, 9, 16, 100, 3, 0, 50], np.uint32)
    _, thr, alias, S = orc.noise_table(counts)
    n, Ns, tiles = counts.size, 64, 400
    draws = np.concatenate([orc.tile_negatives(thr, alias, n, S, 21, 2, t, Ns)
                            for t in range(tiles)])
    freq = np.bincount(draws, minlength=n).astype(float)
    p = counts.astype(float) ** 0.75
    p /= p.sum()
    exp = p * draws.size
    mask = exp > 0
    assert freq[~mask].sum() == 0
    chi2 = (((freq - exp) ** 2)[mask] / exp[mask]).sum()
    assert chi2 < 30.0  # 6 degrees of freedom; p ~ 4e-5
    a = orc.tile_negatives(thr, alias, n, S, 21, 2, 0, Ns)
    assert not np.array_equal(a, orc.tile_negatives(thr, alias, n, S, 21, 2, 1, Ns))
    assert not np.array_equal(a, orc.tile_negatives(thr, alias, n, S, 21, 3, 0, Ns))
