"""Pins for the oracle's noise distribution Pn(u) (Eq. 2) and its alias table."""
import numpy as np
import pytest


def _check_invariant(W, thr, alias, S):
    """thr[v] + sum_{b: alias[b] = v, b != v} (S - thr[b]) = n * W_v, exactly."""
    n = W.shape[0]
    got = [int(t) for t in thr]
    for b in range(n):
        if alias[b] != b:
            got[alias[b]] += S - int(thr[b])
    assert all(got[v] == n * int(W[v]) for v in range(n))
    assert all(0 <= int(t) <= S for t in thr)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_alias_invariant_random_counts(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 400))
    c = rng.zipf(1.7, size=n).astype(np.uint32)
    c[rng.random(n) < 0.3] = 0
    if c.sum() == 0:
        c[0] = 1
    W, thr, alias, S = orc.noise_table(c)
    assert S == int(W.astype(object).sum())
    _check_invariant(W, thr, alias, S)


def test_weights_are_three_quarter_power(orc):
    c = np.array([0, 1, 2, 3, 10, 100, 1000, 123456, 1, 0, 7], dtype=np.uint32)
    W, thr, alias, S = orc.noise_table(c)
    ref = np.where(c > 0, np.maximum(1, np.floor(c ** 0.75 / c.max() ** 0.75 * 2.0 ** 32)), 0)
    assert np.all(np.abs(W.astype(np.float64) - ref) <= 1)
    assert W[c.argmax()] == 2 ** 32
    assert W[0] == 0 and W[9] == 0


def test_degenerate_tables(orc):
    # all counts equal: every bucket is exactly full
    W, thr, alias, S = orc.noise_table(np.full(17, 5, np.uint32))
    assert (thr == S).all() and (alias == np.arange(17)).all()
    # one node holds all the mass
    c = np.zeros(9, np.uint32)
    c[4] = 3
    W, thr, alias, S = orc.noise_table(c)
    assert S == 2 ** 32
    for b in range(9):
        assert b == 4 or (thr[b] == 0 and alias[b] == 4)


def test_draw_frequencies(orc):
    rng = np.random.default_rng(11)
    n = 50
    c = rng.integers(0, 1000, size=n).astype(np.uint32)
    c[3] = 0
    W, thr, alias, S = orc.noise_table(c)
    draws = 60000
    hist = np.zeros(n)
    for i in range(draws):
        hist[orc.draw_negative(thr, alias, S, seed=5, round_=2, walk_idx=i, pos=i % 40, q=i % 10,
                               k=i % 5)] += 1
    p = W.astype(np.float64) / S
    sigma = np.sqrt(p * (1 - p) / draws)
    assert hist[3] == 0
    assert np.all(np.abs(hist / draws - p) < 5 * sigma + 1e-12)


def test_sequential_sweep_small_case(orc):
    # hand-checked: counts 16,1,1 -> weights 2^32, 2^32/8, 2^32/8
    W, thr, alias, S = orc.noise_table(np.array([16, 1, 1], np.uint32))
    assert list(W) == [2 ** 32, 2 ** 29, 2 ** 29]
    S_exp = 2 ** 32 + 2 ** 30
    assert S == S_exp
    # light items 1, 2 (mass 3 * 2^29 < S); heavy item 0 (mass 3 * 2^32)
    assert list(alias) == [0, 0, 0]
    assert list(thr) == [S_exp, 3 * 2 ** 29, 3 * 2 ** 29]
