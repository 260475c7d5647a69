"""Serving form: requests that arrive while others are on the GPU are
admitted as memory frees up, their rounds run together with the others', and
each result is the same as the job trained alone (same tokens; link AUC
within 0.005)."""
import time

import numpy as np
import pytest

from paper_2606_22180_b300 import inputs

pytestmark = pytest.mark.gpu

L, W, K, R = 40, 5, 5, 6


@pytest.fixture(scope="module")
def fl():
    from paper_2606_22180_b300 import build, felog

    build.build()
    felog.load()
    return felog


def _jobs(count, base=1000, step=600):
    out = []
    for i in range(count):
        g, _ = inputs.sbm(base + step * i, 8, 0.04, 0.002, seed=400 + i)
        out.append(inputs.link_split(g, 0.1, i))
    return out


def _params(fl):
    tp = fl.train_params(64, W, K, 0.025, 0, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_FP32)
    fp = fl.feedback_params(False, 0.65, 8, R, False)
    return tp, fp


def test_served_results_equal_solo_and_overlap(fl):
    """Six graphs, each served twice (two seeds, 12 requests): the second
    half of the requests arrives while the first are on the GPU.  Every job
    trains the same tokens as alone, and each graph's link AUC (mean of its
    two seeds) is within 0.005 of the same jobs trained alone."""
    from paper_2606_22180_b300 import evaluate

    splits = _jobs(6)
    tp, fp = _params(fl)
    sv = fl.Server(4 << 30, L, 1, tp, fp)
    reqs = [(i, 50 + i + 100 * rep) for rep in range(2) for i in range(6)]
    ids = []
    for i, seed in reqs[:6]:
        ids.append(sv.submit(splits[i].train, 64, seed))
    # the next requests arrive while the first ones are on the GPU
    t0 = time.time()
    while sv.poll(ids[0])["state"] == fl.JOB_QUEUED and time.time() - t0 < 30:
        time.sleep(0.001)
    for i, seed in reqs[6:]:
        ids.append(sv.submit(splits[i].train, 64, seed))
    res = [sv.wait(r, 300) for r in ids]
    st = sv.stats()
    embs = [sv.fetch(r) for r in ids]
    sv.close()
    assert all(r["state"] == fl.JOB_DONE for r in res)
    assert st["completed"] == 12 and st["peak_resident_jobs"] >= 2
    # some job was admitted while an earlier one was still running
    assert any(res[j]["t_admit"] < res[i]["t_done"] and res[j]["t_submit"] > res[i]["t_admit"]
               for i in range(12) for j in range(12) if i != j)
    diffs = np.zeros((2, 6))
    for k, (i, seed) in enumerate(reqs):
        sp = splits[i]
        dg = fl.DeviceGraph.from_host(sp.train)
        solo, _, sst = fl.felog_embed(dg, L, 1, tp, fp, seed)
        assert res[k]["rounds"] == len(sst) and res[k]["tokens"] == sum(s["tokens"] for s in sst)
        diffs[k // 6, i] = evaluate.link_auc(embs[k], sp.pos, sp.neg) - evaluate.link_auc(solo, sp.pos, sp.neg)
    per_graph = diffs.mean(0)
    print("served - solo AUC per graph (mean of 2 seeds):", np.round(per_graph, 4))
    assert np.all(np.abs(per_graph) <= 0.005), per_graph


def test_budget_admission_and_rejection(fl):
    splits = _jobs(3, base=1500, step=0)
    tp, fp = _params(fl)
    probe = fl.Server(1 << 30, L, 1, tp, fp)
    need = probe.job_bytes(splits[0].train.n, splits[0].train.nnz, 64)
    probe.close()
    sv = fl.Server(int(need * 1.5), L, 1, tp, fp)  # room for one job at a time
    big, _ = inputs.sbm(6000, 8, 0.04, 0.002, seed=9)
    ids = [sv.submit(sp.train, 64, 7 + i) for i, sp in enumerate(splits)]
    rid_big = sv.submit(big, 64, 1)
    res = [sv.wait(r, 300) for r in ids]
    rb = sv.wait(rid_big, 300)
    st = sv.stats()
    sv.close()
    assert all(r["state"] == fl.JOB_DONE for r in res)
    assert rb["state"] == fl.JOB_REJECTED
    assert st["peak_resident_jobs"] == 1 and st["rejected"] == 1
    assert st["peak_resident_bytes"] <= int(need * 1.5)
    # first come first served, one at a time
    assert res[0]["t_done"] <= res[1]["t_admit"] + 1e-6 and res[1]["t_done"] <= res[2]["t_admit"] + 1e-6


def test_malformed_csr_rejected_on_host(fl):
    tp, fp = _params(fl)
    sv = fl.Server(1 << 30, L, 1, tp, fp)

    class Bad:
        offsets = np.array([0, 2, 1, 3], np.int32)  # not monotone
        cols = np.array([1, 2, 0], np.int32)

    with pytest.raises(fl.FelogError, match="malformed"):
        sv.submit(Bad, 64, 1)

    class OutOfRange:
        offsets = np.array([0, 1, 2], np.int32)
        cols = np.array([1, 5], np.int32)

    with pytest.raises(fl.FelogError, match="malformed"):
        sv.submit(OutOfRange, 64, 1)
    assert sv.stats()["submitted"] == 0
    sv.close()


def test_served_minibatch_results_equal_solo_bitwise(fl):
    """The deterministic form served: jobs admitted at different times and
    trained in the mix return exactly the embedding each gets alone."""
    splits = _jobs(4)
    tp = fl.train_params(64, W, K, 0.025, 0, fl.FELOG_SGNS_MINIBATCH, 1 << 30, fl.FELOG_FP32)
    fp = fl.feedback_params(True, 0.9, 8, R, False)
    sv = fl.Server(4 << 30, L, 1, tp, fp)
    ids = [sv.submit(sp.train, 64, 70 + i) for i, sp in enumerate(splits[:2])]
    t0 = time.time()
    while sv.poll(ids[0])["state"] == fl.JOB_QUEUED and time.time() - t0 < 30:
        time.sleep(0.001)
    ids += [sv.submit(sp.train, 64, 72 + i) for i, sp in enumerate(splits[2:])]
    res = [sv.wait(r, 300) for r in ids]
    embs = [sv.fetch(r) for r in ids]
    sv.close()
    assert all(r["state"] == fl.JOB_DONE for r in res)
    for i, sp in enumerate(splits):
        solo, _, st = fl.felog_embed(fl.DeviceGraph.from_host(sp.train), L, 1, tp, fp, 70 + i)
        assert res[i]["rounds"] == len(st) and res[i]["loss_last"] == st[-1]["loss"], i
        assert np.array_equal(np.asarray(embs[i]), solo.cpu().numpy()), i
