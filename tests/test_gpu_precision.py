"""Precision form: bf16 tables (float math, stochastic rounding on every
store) against the binary64 oracle, error stated per result.  Both sides
start from the same bf16-rounded initial table, so the measured error is
the rounding during training alone.  The deterministic form is used so the
comparison is pair for pair (same pairs, same negatives, same batches)."""
import json
import os

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


def _cos_rows(a, b):
    na = np.linalg.norm(a, axis=1)
    nb = np.linalg.norm(b, axis=1)
    ok = (na > 0) & (nb > 0)
    return (a[ok] * b[ok]).sum(1) / (na[ok] * nb[ok])


def test_bf16_error_against_oracle(fl, orc):
    g, _ = inputs.workload_sbm1000(0)
    starts = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
    L, dim, w, K, B = 40, 64, 5, 5, 4096
    report = {}
    pi0, _ = fl.felog_init_tables(g.n, dim, fl.FELOG_BF16_SR, 3)
    ri = pi0.double().cpu().numpy()  # the bf16-rounded start, exactly
    ro = np.zeros_like(ri)
    pi, po = pi0.clone(), torch.zeros_like(pi0)
    T = 3 * starts.shape[0] * L
    clock = 0
    for r in range(3):
        W = orc.walk(g.offsets, g.cols, starts, L, 1, 3, r)
        _, thr, alias, S = orc.noise_table(orc.counts(W, g.n))
        tp = fl.train_params(dim, w, K, 0.025, T, fl.FELOG_SGNS_MINIBATCH, B, fl.FELOG_BF16_SR)
        lg = float(fl.felog_train(torch.from_numpy(W).cuda(), g.n, tp, torch.from_numpy(thr.astype(np.int64)).cuda(),
                                  torch.from_numpy(alias).cuda(), torch.tensor([S], dtype=torch.int64).cuda(), 3, r,
                                  clock, pi, po).item())
        lo = orc.sgns_minibatch(W, g.n, dim, w, K, 0.025, T, B, thr, alias, S, 3, r, clock, ri, ro)
        clock += W.size
        cin = _cos_rows(pi.double().cpu().numpy(), ri)
        cout = _cos_rows(po.double().cpu().numpy(), ro)
        report[f"round{r}"] = {
            "loss_rel_err": abs(lg - lo) / lo,
            "phi_in_cos_mean": float(cin.mean()), "phi_in_cos_p1": float(np.percentile(cin, 1)),
            "phi_out_cos_mean": float(cout.mean()), "phi_out_cos_p1": float(np.percentile(cout, 1)),
            "phi_in_rel_frobenius": float(np.linalg.norm(pi.double().cpu().numpy() - ri) / np.linalg.norm(ri)),
        }
    print("bf16 vs binary64 oracle:", json.dumps(report))
    out = os.environ.get("FELOG_PRECISION_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump(report, f, indent=1)
    last = report["round2"]
    assert last["loss_rel_err"] < 2e-3
    assert last["phi_in_cos_mean"] > 0.999 and last["phi_in_cos_p1"] > 0.99
    assert last["phi_out_cos_mean"] > 0.999


def test_bf16_round_trip_is_exact_for_representable_values(fl):
    """Stochastic rounding leaves bf16-representable sums unchanged: a
    zero-learning-rate round must return the tables bit for bit."""
    g, _ = inputs.workload_sbm1000(1)
    starts = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
    dg = fl.DeviceGraph.from_host(g)
    pi, po = fl.felog_init_tables(g.n, 64, fl.FELOG_BF16_SR, 5)
    po.copy_(pi.flip(0))
    a, b = pi.clone(), po.clone()
    counts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    W = fl.felog_walk(dg, torch.from_numpy(starts).cuda(), starts.shape[0], 20, 1, 5, 0, counts=counts)
    thr, alias, S = fl.felog_noise_table(counts)
    for mode in (fl.FELOG_SGNS_HOGWILD, fl.FELOG_SGNS_MINIBATCH):
        tp = fl.train_params(64, 3, 3, 0.0, 10 ** 6, mode, 512, fl.FELOG_BF16_SR)
        fl.felog_train(W, g.n, tp, thr, alias, S, 5, 0, 0, pi, po)
        assert torch.equal(pi, a) and torch.equal(po, b)
