"""Round-interleaved pipeline (Section 5.3) through felog_embed_pipelined.

feedback_lag = 0 is Algorithm 1 as printed: in the deterministic (minibatch)
form its tables and schedule are bit-identical to felog_embed's.
feedback_lag = 1 decides V_a^{r+1} on the snapshot taken as round r's
training starts: it must track the oracle's Algorithm 1 with the same option
(schedule and loss per round, tables within 1e-5), and its sample stream
must run while the train stream trains.
"""
import numpy as np
import pytest
import torch

from paper_2606_22180_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    from paper_2606_22180_b300 import build, felog

    build.build()
    felog.load()
    return felog


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("enabled,mu", [(True, 0.9), (False, 0.65)])
def test_lag0_equals_felog_embed_bitwise(fl, enabled, mu):
    g, _ = inputs.workload_sbm1000(0)
    dg = fl.DeviceGraph.from_host(g)
    tp = fl.train_params(32, 3, 3, 0.025, 0, fl.FELOG_SGNS_MINIBATCH, 1000, fl.FELOG_FP32)
    fp = fl.feedback_params(enabled, mu, 8, 6, False)
    pi, po, st = fl.felog_embed(dg, 20, 1, tp, fp, 2)
    qi, qo, qst, ps = fl.felog_embed_pipelined(dg, 20, 1, tp, fp, 2, feedback_lag=0)
    assert [s["n_active"] for s in qst] == [s["n_active"] for s in st]
    assert [s["loss"] for s in qst] == [s["loss"] for s in st]
    assert torch.equal(pi, qi) and torch.equal(po, qo)
    assert ps["rounds"] == len(st) and ps["feedback_lag"] == 0


def test_lag1_tracks_the_lagged_oracle(fl, orc):
    g, _ = inputs.workload_sbm1000(0)
    dim, L, R, w, K, B, mu, seed = 32, 20, 6, 3, 3, 1000, 0.9, 2
    dg = fl.DeviceGraph.from_host(g)
    tp = fl.train_params(dim, w, K, 0.025, 0, fl.FELOG_SGNS_MINIBATCH, B, fl.FELOG_FP32)
    fp = fl.feedback_params(True, mu, 8, R, False)
    qi, qo, qst, ps = fl.felog_embed_pipelined(dg, L, 1, tp, fp, seed, feedback_lag=1)
    ri, ro, rst = orc.embed(g.offsets, g.cols, L, 1, dim, w, K, 0.025, True, mu, 8, R, False, seed,
                            mode="minibatch", B=B, feedback_lag=1)
    print("lag-1 schedule:", [s["n_active"] for s in qst], "oracle:", [int(x) for x in rst[:, 0]])
    assert [s["n_active"] for s in qst] == [int(x) for x in rst[:, 0]]
    for s, r in zip(qst, rst):
        assert abs(s["loss"] - r[2]) / r[2] < 1e-5
    assert _rel(qi.double().cpu().numpy(), ri) < 1e-5 and _rel(qo.double().cpu().numpy(), ro) < 1e-5
    # the lag is visible: round 1 starts from the decision on the initial table
    _, _, st0 = fl.felog_embed(dg, L, 1, tp, fp, seed)
    assert [s["n_active"] for s in st0] != [s["n_active"] for s in qst]


def test_lag1_overlaps_sampling_with_training(fl):
    g = inputs.rmat(16, 16, seed=3)
    dg = fl.DeviceGraph.from_host(g)
    tp = fl.train_params(128, 10, 5, 0.025, 0, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_FP32)
    fp = fl.feedback_params(False, 0.65, 8, 4, False)
    _, _, st, ps = fl.felog_embed_pipelined(dg, 80, 1, tp, fp, 7, feedback_lag=1)
    print("pipeline stats:", ps)
    assert ps["rounds"] == 4 and len(st) == 4
    assert ps["overlap_ms"] > 0.5 * ps["sample_busy_ms"]
    assert all(np.isfinite(s["loss"]) for s in st)
