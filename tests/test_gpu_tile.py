"""TILE mode (shared negatives, tensor-core contractions) against the oracle's
tile routine.

Inputs are on the bf16 grid so that the gathered operands are exact; the
remaining differences come from the bf16 gradient matrix and f32
accumulation.  With lr0 = 0 the tables stay put and the loss alone checks
scores, the shared draws, the positive band, walk boundaries, padding and
the skip rule.
"""
import numpy as np
import pytest
import torch

from paper_2606_22180_b300 import inputs

pytestmark = pytest.mark.gpu

SEED = 13


@pytest.fixture(scope="module")
def fl():
    from paper_2606_22180_b300 import build, felog

    build.build()
    felog.load()
    return felog


@pytest.fixture(scope="module")
def sbm():
    g, _ = inputs.workload_sbm1000(0)
    return g


def _dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def _bf16_grid(a):
    return torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _corpus(orc, g, L, seed, rnd, n_starts=None, pad=False):
    starts = np.nonzero(g.degrees() > 0)[0][:n_starts].astype(np.int32)
    W = orc.walk(g.offsets, g.cols, starts, L, 1, seed, rnd)
    if pad:  # truncated walks: -1 padding inside the corpus
        W[::7, L // 2:] = -1
        W[3::11, 1:] = -1
    _, thr, alias, S = orc.noise_table(orc.counts(W, g.n))
    return W, thr, alias, S


def _tables(n, dim, seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return (_bf16_grid(rng.normal(scale=scale, size=(n, dim))),
            _bf16_grid(rng.normal(scale=scale, size=(n, dim))))


def _to_dev(fl, a, precision):
    t = torch.from_numpy(a.astype(np.float32)).cuda()
    return t if precision == fl.FELOG_FP32 else t.to(torch.bfloat16)


def _train(fl, W, thr, alias, S, n, tp, seed, rnd, clock, pi, po):
    loss = fl.felog_train(_dev(W), n, tp, _dev(thr.astype(np.int64)), _dev(alias),
                          _dev(np.array([S], np.int64)), seed, rnd, clock, pi, po)
    return float(loss.item())


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("dim,window,Ns,prec,pad,ctas", [(128, 10, 512, 0, False, 8), (64, 5, 128, 1, True, 0),
                                                         (32, 16, 256, 0, True, 8), (128, 3, 384, 1, False, 4),
                                                         (64, 10, 512, 1, True, 1)])
def test_tile_loss_matches_oracle_at_fixed_tables(fl, orc, sbm, dim, window, Ns, prec, pad, ctas):
    """Both the in-order form (one CTA) and the pipelined form (several)."""
    g = sbm
    L, K = 40, 5
    W, thr, alias, S = _corpus(orc, g, L, SEED, 1, n_starts=300, pad=pad)
    ri, ro = _tables(g.n, dim, 3)
    pi, po = _to_dev(fl, ri, prec), _to_dev(fl, ro, prec)
    tp = fl.train_params(dim, window, K, 0.0, 10 ** 9, fl.FELOG_SGNS_TILE, 1, prec,
                         tile_negatives=Ns, tile_ctas=ctas)
    lg = _train(fl, W, thr, alias, S, g.n, tp, SEED, 1, 0, pi, po)
    lo = orc.sgns_tile(W, g.n, dim, window, K, 0.0, 10 ** 9, 128 - 2 * window, Ns, thr, alias, S,
                       SEED, 1, 0, ri, ro)
    print(f"loss rel err {abs(lg - lo) / lo:.3e}")
    assert abs(lg - lo) / lo < 1e-4
    assert np.array_equal(pi.double().cpu().numpy(), ri)
    assert np.array_equal(po.double().cpu().numpy(), ro)


@pytest.mark.parametrize("dim,window,Ns", [(128, 10, 512), (64, 5, 128), (32, 8, 256)])
def test_tile_serial_fp32_tracks_oracle(fl, orc, sbm, dim, window, Ns):
    """Tiles one at a time (tile_ctas = 1) is the oracle's order: the loss
    and the table increments agree up to the bf16 gradient operand."""
    g = sbm
    L, K = 40, 5
    W, thr, alias, S = _corpus(orc, g, L, SEED, 0, n_starts=200, pad=True)
    ri0, ro0 = _tables(g.n, dim, 4)
    ri, ro = ri0.copy(), ro0.copy()
    pi, po = _to_dev(fl, ri0, 0), _to_dev(fl, ro0, 0)
    T = 20 * W.size
    tp = fl.train_params(dim, window, K, 0.025, T, fl.FELOG_SGNS_TILE, 1, fl.FELOG_FP32,
                         tile_negatives=Ns, tile_ctas=1)
    lg = _train(fl, W, thr, alias, S, g.n, tp, SEED, 0, 77, pi, po)
    lo = orc.sgns_tile(W, g.n, dim, window, K, 0.025, T, 128 - 2 * window, Ns, thr, alias, S, SEED,
                       0, 77, ri, ro)
    gi, go = pi.double().cpu().numpy(), po.double().cpu().numpy()
    e_loss = abs(lg - lo) / lo
    e_in, e_out = _rel(gi - ri0, ri - ri0), _rel(go - ro0, ro - ro0)
    print(f"loss {e_loss:.3e}  d_phi_in {e_in:.3e}  d_phi_out {e_out:.3e}")
    assert e_loss < 1e-3
    assert e_in < 2e-2 and e_out < 2e-2


def test_tile_serial_bf16_tracks_oracle(fl, orc, sbm):
    """bf16 tables with stochastic rounding: the loss tracks the oracle; the
    tables carry the rounding noise (zero mean, up to one bf16 ulp, about
    0.4 % of a value, per update; some 20 updates per element in this
    round), so they are held to 1.5 % in norm."""
    g = sbm
    dim, window, K, Ns = 128, 10, 5, 512
    W, thr, alias, S = _corpus(orc, g, 40, SEED, 2, n_starts=200)
    ri0, ro0 = _tables(g.n, dim, 5)
    ri, ro = ri0.copy(), ro0.copy()
    pi, po = _to_dev(fl, ri0, 1), _to_dev(fl, ro0, 1)
    T = 20 * W.size
    tp = fl.train_params(dim, window, K, 0.025, T, fl.FELOG_SGNS_TILE, 1, fl.FELOG_BF16_SR,
                         tile_negatives=Ns, tile_ctas=1)
    lg = _train(fl, W, thr, alias, S, g.n, tp, SEED, 2, 0, pi, po)
    lo = orc.sgns_tile(W, g.n, dim, window, K, 0.025, T, 128 - 2 * window, Ns, thr, alias, S, SEED,
                       2, 0, ri, ro)
    e_loss = abs(lg - lo) / lo
    e_in = _rel(pi.double().cpu().numpy(), ri)
    e_out = _rel(po.double().cpu().numpy(), ro)
    print(f"loss {e_loss:.3e}  phi_in {e_in:.3e}  phi_out {e_out:.3e}")
    assert e_loss < 1e-3
    assert e_in < 1.5e-2 and e_out < 1.5e-2


def test_tile_parallel_round_close_to_serial(fl, orc):
    """Many tiles at once (32 on R-MAT 16) race on shared rows, so the
    trajectory departs from the in-order oracle (the quality of this form is
    judged by link AUC); here the round must stay stable: loss within 10 %
    of the oracle's, increments of the same size."""
    g = inputs.rmat(16, 16, seed=3)
    dim, window, K, Ns = 64, 10, 5, 512
    W, thr, alias, S = _corpus(orc, g, 80, SEED, 0, n_starts=1000)
    ri0, ro0 = _tables(g.n, dim, 6, scale=0.05)
    ri, ro = ri0.copy(), ro0.copy()
    pi, po = _to_dev(fl, ri0, 0), _to_dev(fl, ro0, 0)
    T = 5 * W.size
    tp = fl.train_params(dim, window, K, 0.025, T, fl.FELOG_SGNS_TILE, 1, fl.FELOG_FP32,
                         tile_negatives=Ns, tile_ctas=32)
    lg = _train(fl, W, thr, alias, S, g.n, tp, SEED, 0, 0, pi, po)
    lo = orc.sgns_tile(W, g.n, dim, window, K, 0.025, T, 128 - 2 * window, Ns, thr, alias, S, SEED,
                       0, 0, ri, ro)
    e_in = _rel(pi.double().cpu().numpy() - ri0, ri - ri0)
    print(f"parallel loss rel diff {abs(lg - lo) / lo:.3e}  d_phi_in {e_in:.3e}")
    assert abs(lg - lo) / lo < 0.1
    assert e_in < 1.0


def test_tile_degenerate_inputs(fl, orc, sbm):
    g = sbm
    dim = 64
    ri, ro = _tables(g.n, dim, 7)
    pi, po = _to_dev(fl, ri, 0), _to_dev(fl, ro, 0)
    tp = fl.train_params(dim, 5, 5, 0.025, 1000, fl.FELOG_SGNS_TILE, 1, fl.FELOG_FP32)
    thr = np.zeros(g.n, np.uint64)
    alias = np.arange(g.n, dtype=np.int32)
    # walks of one node: no pairs
    W1 = np.arange(50, dtype=np.int32).reshape(50, 1)
    assert _train(fl, W1, thr, alias, 1, g.n, tp, 1, 0, 0, pi, po) == 0.0
    # all padding
    Wp = np.full((9, 30), -1, np.int32)
    assert _train(fl, Wp, thr, alias, 1, g.n, tp, 1, 0, 0, pi, po) == 0.0
    assert np.array_equal(pi.double().cpu().numpy(), ri)
    assert np.array_equal(po.double().cpu().numpy(), ro)
