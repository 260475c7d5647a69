"""Stochastic rounding of the bf16 tables, measured through felog_train.

A controlled corpus makes every update of Eq. 2 known in closed form: walks
of two distinct nodes (each node in exactly one walk), window 1, one
negative, phi_out = 0, every phi_in element equal to one bf16 value v, and a
constant learning rate.  All scores are then zero (minibatch form: the
snapshot is phi_out = 0) or far below 2^-24 (Hogwild), so sigma = 1/2 and
every pair adds exactly +delta0 (positive) or -delta0 (negative) to one
phi_out row, delta0 = eta/2 * v.  The negatives are the oracle's draws with
the same keys and table, so the exact sum each phi_out row receives is known.
delta0 is chosen 0.1875 ulp above a bf16 value, where rounding to nearest is
biased by 0.1875 ulp per store.

Checked: every stored element is one of the two bf16 neighbours of its exact
value; the fraction of elements rounded away from zero matches the exact
fractions within 5 sigma (E[SR(x)] = x); phi_in, whose increments are zero
in the minibatch form, stays exactly v (bf16 values are fixed points of the
stores at a non-zero learning rate).
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SEED = 77
N = 1 << 18           # nodes; N / 2 walks of length 2
LR0 = 2.0 ** -5 * (1 + 2.0 ** -10)  # eta / 2 = 2^-6 (1 + 2^-10), exact in float
T_HUGE = 1 << 62      # 1 - t / T rounds to 1: eta = lr0 for every position


@pytest.fixture(scope="module")
def fl():
    from paper_2606_22180_b300 import build, felog

    build.build()
    felog.load()
    return felog


@pytest.fixture(scope="module")
def corpus(orc):
    """Walks [a, b] pairing a random permutation of the nodes, the uniform
    noise table of their counts, and the per-row count of negative draws."""
    rng = np.random.default_rng(5)
    walks = rng.permutation(N).astype(np.int32).reshape(-1, 2)
    cnt = orc.counts(walks, N)
    assert (cnt == 1).all()
    _, thr, alias, S = orc.noise_table(cnt)
    lib = orc.lib()
    tp_ = thr.ctypes.data_as(ctypes.c_void_p)
    ap_ = alias.ctypes.data_as(ctypes.c_void_p)
    n_neg = np.zeros(N, np.int64)
    skipped = 0
    for wi in range(walks.shape[0]):
        for p, q in ((0, 1), (1, 0)):  # center 0: offset +1 (slot 1); center 1: offset -1 (slot 0)
            c = walks[wi, p]
            nk = lib.oracle_draw_negative(tp_, ap_, N, S, SEED, 0, wi, p, q, 0)
            if nk != c:
                n_neg[nk] += 1
            else:
                skipped += 1
    return walks, thr, alias, S, n_neg, skipped


def _bf16_bits(t: torch.Tensor) -> np.ndarray:
    return t.view(torch.int16).cpu().numpy().view(np.uint16).astype(np.uint32)


def _neighbours(exact: np.ndarray):
    """Truncation and next-away bf16 patterns of float64 values exactly
    representable in binary32, and the fraction of an ulp above truncation."""
    xb = exact.astype(np.float32).view(np.uint32)
    assert np.array_equal(xb.view(np.float32).astype(np.float64), exact)
    down = xb >> 16
    frac = (xb & 0xffff) / 65536.0
    return down, down + 1, frac


def _train(fl, corpus, mode, v_bits):
    walks, thr, alias, S = corpus[:4]
    dev = "cuda"
    phi_in = torch.full((N, 128), 0, dtype=torch.int16, device=dev)
    phi_in.fill_(np.int16(np.uint16(v_bits)))
    phi_in = phi_in.view(torch.bfloat16)
    phi_out = torch.zeros((N, 128), dtype=torch.bfloat16, device=dev)
    tp = fl.train_params(128, 1, 1, LR0, T_HUGE, mode, walks.size, fl.FELOG_BF16_SR)
    W = torch.from_numpy(walks).cuda()
    loss = fl.felog_train(W, N, tp, torch.from_numpy(thr.astype(np.int64)).cuda(), torch.from_numpy(alias).cuda(),
                          torch.tensor([S], dtype=torch.int64).cuda(), SEED, 0, 0, phi_in, phi_out)
    torch.cuda.synchronize()
    return phi_in, phi_out, float(loss.item())


def _z(dev_rows: np.ndarray) -> float:
    """Self-normalised z of per-row deviations (rows are independent; the
    elements of a row share rounding words and need not be)."""
    return float(dev_rows.sum() / np.sqrt((dev_rows ** 2).sum()))


def test_minibatch_bf16_stores_are_unbiased(fl, corpus):
    _, _, _, _, n_neg, skipped = corpus
    v = np.float32(1.5 * 2.0 ** -16)  # delta0 * 2^40 is an integer: fixed-point sums are exact
    v_bits = int(v.view(np.uint32)) >> 16
    phi_in, phi_out, loss = _train(fl, corpus, fl.FELOG_SGNS_MINIBATCH, v_bits)
    # phi_in: zero increments (every score reads phi_out = 0), so SR must return v exactly
    assert (_bf16_bits(phi_in) == v_bits).all()
    delta0 = float(np.float32(2.0 ** -6 * (1 + 2.0 ** -10)) * v)
    exact_row = (1 - n_neg) * delta0          # each node: one positive pair, n_neg negative slots
    got = _bf16_bits(phi_out)                 # [N, 128]
    zero = exact_row == 0
    assert (got[zero] == 0).all()             # SR(0) = 0
    rows = ~zero
    down, up, frac = _neighbours(np.abs(exact_row[rows]))
    mag = got[rows] & 0x7fff
    assert (np.sign(exact_row[rows])[:, None] * np.where(got[rows] & 0x8000, -1, 1) > 0).all()
    assert ((mag == down[:, None]) | (mag == up[:, None])).all()
    away = (mag == up[:, None]).sum(1).astype(np.float64)
    z = _z(away - 128 * frac)
    print(f"minibatch SR: {int(rows.sum())} rows, rounded away {away.sum() / (128 * rows.sum()):.5f}, "
          f"expected {frac.mean():.5f}, z = {z:.2f}")
    assert abs(z) < 5
    # rounding to nearest would round every element down here (all fractions < 1/2)
    assert frac.max() < 0.5 and away.sum() > 0
    # every score is 0: each pair term is log 2 (N pairs, N - skipped negatives)
    assert abs(loss - np.log(2) * (2 * N - skipped)) / loss < 1e-5


def test_hogwild_bf16_stores_are_unbiased(fl, corpus):
    n_neg = corpus[4]
    v = np.float32(1.5 * 2.0 ** -40)  # scores ~2^-79: sigma rounds to 1/2 exactly
    v_bits = int(v.view(np.uint32)) >> 16
    _, phi_out, loss = _train(fl, corpus, fl.FELOG_SGNS_HOGWILD, v_bits)
    assert np.isfinite(loss)
    delta0 = float(np.float32(2.0 ** -6 * (1 + 2.0 ** -10)) * v)
    got = _bf16_bits(phi_out)
    # rows with one update (the positive pair, no negative draw): a Bernoulli per element
    one = n_neg == 0
    down, up, frac = _neighbours(np.full(int(one.sum()), delta0))
    g1 = got[one]
    assert ((g1 == down[0]) | (g1 == up[0])).all()
    p_away = float((g1 == up[0]).mean())
    f = float(frac[0])
    z1 = _z((g1 == up[0]).sum(1) - 128 * f)
    print(f"hogwild SR, one-update rows: {g1.shape[0]}, rounded away {p_away:.5f}, expected {f:.5f}, "
          f"z = {z1:.2f}")
    assert abs(z1) < 5
    # every row, whatever its number of updates: the errors against the exact
    # sum (1 - n_neg) * delta0, in units of delta0, have mean zero
    exact_row = (1 - n_neg) * delta0
    vals = (got.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    err = ((vals - exact_row[:, None]) / delta0).sum(1)
    z = _z(err)
    print(f"hogwild SR, all {N} rows: z = {z:.2f}")
    assert abs(z) < 5


def test_sr_conversion_matches_oracle_bitwise(fl, orc):
    """felog_sr_bf16 rounds with the instruction the bf16 Hogwild trainers use
    for their stores.  Against the oracle's SR definition (add the 16 random
    bits below the kept bits, truncate), bit for bit, over an odd number of
    elements (a ragged last pair): random bit patterns across the whole
    binary32 range including subnormals, zeros of both signs, the largest
    finite values (whose carry gives infinity) and infinities.  A NaN must
    stay a NaN (its payload is not fixed)."""
    rng = np.random.default_rng(5)
    n = (1 << 20) + 3
    xb = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    special = np.array([0x00000000, 0x80000000, 0x00000001, 0x807fffff, 0x7f7fffff, 0xff7fffff,
                        0x7f800000, 0xff800000, 0x7fc00000, 0xffc00001, 0x3f800000, 0x3f80ffff], np.uint32)
    xb[: special.size] = special
    r = rng.integers(0, 1 << 16, size=n, dtype=np.uint64).astype(np.uint16)
    r[: special.size] = 0xffff
    x = torch.from_numpy(xb.view(np.float32)).cuda()
    rt = torch.from_numpy(r.view(np.int16)).cuda()
    got = fl.felog_sr_bf16(x, rt).cpu().numpy().view(np.uint16)
    want = orc.sr_bf16_array(xb, r)
    nan_in = ((xb & 0x7f800000) == 0x7f800000) & ((xb & 0x007fffff) != 0)
    assert np.array_equal(got[~nan_in], want[~nan_in])
    got_nan = ((got & 0x7f80) == 0x7f80) & ((got & 0x007f) != 0)
    assert np.all(got_nan[nan_in])
    assert got[6] == 0x7f80 and got[7] == 0x7f80 | 0x8000  # inf stays inf
    assert got[4] == 0x7f80  # largest finite + carry -> inf
    with pytest.raises(fl.FelogError):
        fl.felog_sr_bf16(x, rt[:-1])
