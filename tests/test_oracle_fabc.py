"""Pins for the oracle's FaBC codec (Section 5.2.2, Eq. 7, Eq. 8).

Pinned by: exact round trips (encode then decode returns the corpus, padding
included); the encoded size against Eq. 7, with F_k counted here from the
corpus; the paper's worked example (top-2 nodes covering 60 % of the
positions: bitmaps plus tail come to 1.85 N L of 4 N L bytes, 0.4625); and the
selection rule of Eq. 8 on hand-computed frequency profiles.
"""
import numpy as np
import pytest


def _eq7(F, k, L):
    """Eq. 7: g(k) = 1 - F_k + k/L + k/32."""
    return 1.0 - F + k / L + k / 32.0


@pytest.mark.parametrize("seed,L,k", [(0, 80, 0), (1, 80, 2), (2, 40, 3), (3, 13, 1), (4, 7, 5), (5, 33, 2)])
def test_round_trip_is_exact(orc, seed, L, k):
    rng = np.random.default_rng(seed)
    N = 57
    W = rng.integers(0, 20, size=(N, L)).astype(np.int32)
    W[::5, L // 2:] = -1  # truncated walks
    ids = np.arange(k, dtype=np.int32) * 3  # nodes 0, 3, 6, ...
    buf = orc.fabc_encode(W, ids)
    assert np.array_equal(orc.fabc_decode(buf, N, L, k), W)


@pytest.mark.parametrize("L,k", [(80, 1), (80, 2), (40, 3), (16, 4)])
def test_size_matches_eq7(orc, L, k):
    """For L a multiple of 8 the encoded size is exactly g(k) * 4 N L."""
    rng = np.random.default_rng(L + k)
    N = 200
    p = np.array([0.3, 0.2, 0.1, 0.05] + [0.35 / 96] * 96)
    W = rng.choice(100, size=(N, L), p=p / p.sum()).astype(np.int32)
    ids = np.arange(k, dtype=np.int32)
    F = float(np.isin(W, ids).mean())  # covered fraction of positions
    size = orc.fabc_encode(W, ids).size
    assert size == pytest.approx(_eq7(F, k, L) * 4 * N * L, rel=0, abs=1e-6)


def test_worked_example_ratio(orc):
    """Section 5.2.2's example: the top-2 nodes cover 60 % of the positions;
    bitmaps (k N L / 8) plus the tail (4 N 0.4 L) are 1.85 N L bytes, 0.4625
    of the 4 N L raw bytes.  (The example leaves out the 4 N k id bytes.)"""
    N, L = 100, 80
    W = np.full((N, L), 7, np.int32)
    W[:, :24] = 1  # 30 % node 1
    W[:, 24:48] = 2  # 30 % node 2
    W[:, 48:] = np.arange(10, 42)  # the other 40 %
    ids, F = orc.fabc_select(np.bincount(W.ravel(), minlength=50).astype(np.uint32), L, 8)
    assert list(ids) == [1, 2] and F == pytest.approx(0.6)
    size = orc.fabc_encode(W, ids).size
    assert (size - 4 * N * len(ids)) / (4 * N * L) == pytest.approx(0.4625, abs=1e-12)


@pytest.mark.parametrize("probs,L,expect", [
    # the example's narrative: two nodes over 50 %, the third adds little
    ([0.3, 0.3, 0.05, 0.03], 80, 2),
    # one dominant node: g(1) = 0.14375, the second needs p >= 0.058
    ([0.9, 0.01, 0.01], 80, 1),
    # a flat profile: the first node needs p >= c + 0.1 = 0.14375
    ([0.01] * 10, 80, 0),
    # longer walks lower c = 1/L + 1/32
    ([0.2, 0.12, 0.1, 0.02], 1000, 2),
])
def test_selection_rule(orc, probs, L, expect):
    """Eq. 8, worked by hand: p(k+1) >= c + 0.1 g(k), c = 1/L + 1/32."""
    scale = 10 ** 6
    counts = np.zeros(64, np.uint32)
    rest = scale - int(round(sum(probs) * scale))
    for i, p in enumerate(probs):
        counts[10 + 3 * i] = int(round(p * scale))  # not in id order
    counts[40:] = rest // 24  # filler, each below any threshold
    counts[40] += rest - (rest // 24) * 24
    ids, F = orc.fabc_select(counts, L, 32)
    assert len(ids) == expect
    assert list(ids) == [10 + 3 * i for i in range(expect)]


def test_selection_ties_take_the_smaller_id(orc):
    counts = np.zeros(20, np.uint32)
    counts[[4, 9, 2]] = 1000
    counts[0] = 10
    ids, _ = orc.fabc_select(counts, 80, 2)
    assert list(ids) == [2, 4]
