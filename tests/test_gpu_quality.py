"""Hogwild and BF16 forms against the serial oracle by link-prediction AUC
on the 1,000-node planted partition (10 % of edges held out)."""
import numpy as np
import pytest

from paper_2606_22180_b300 import inputs

pytestmark = pytest.mark.gpu

L, DIM, W, K, R = 40, 64, 5, 5, 10
SEEDS = 8
TILE_R, TILE_NS = 3, 128


@pytest.fixture(scope="module")
def fl():
    from paper_2606_22180_b300 import build, felog

    build.build()
    return felog


# (name, precision: 0 float / 1 bf16-SR, hogwild_form, dim).  Form 0 is the
# automatic choice: form 2 at dim 64, and for bf16 at dim 128 the prefetching
# form 4 (which covers rows of 128 to 512 bytes: float dim 32/64/128, bf16 dim
# 64/128); the forms at dim 128 are held to the dim-128 oracle.
FORMS = [("hogwild", 0, 0, DIM), ("bf16", 1, 0, DIM), ("staged", 0, 3, DIM), ("staged_bf16", 1, 3, DIM),
         ("prefetch", 0, 4, DIM), ("prefetch_128", 0, 4, 128), ("prefetch_bf16", 1, 0, 128),
         ("bf16_128", 1, 2, 128), ("bulk", 0, 5, DIM), ("bulk_128", 0, 5, 128), ("prefetch_bf16_64", 1, 4, DIM)]


@pytest.fixture(scope="module")
def runs(fl, orc):
    from paper_2606_22180_b300 import evaluate

    res = []
    # 8 seeds: one lock-free bf16 run's AUC on this 1,000-node graph moves by
    # about 0.005 from seed to seed, so a mean over 5 would sit within a few
    # standard errors of the 0.005 bound by chance alone
    for seed in range(SEEDS):
        g, _ = inputs.workload_sbm1000(seed)
        sp = inputs.link_split(g, 0.1, seed)
        tr = sp.train
        out = {}
        for d in (DIM, 128):
            ri, _, _ = orc.embed(tr.offsets, tr.cols, L, 1, d, W, K, 0.025, False, 0.65, 8, R, False, seed)
            out[f"oracle{d}"] = orc.link_auc(ri, sp.pos, sp.neg)
        out["oracle"] = out[f"oracle{DIM}"]
        dg = fl.DeviceGraph.from_host(tr)
        fp = fl.feedback_params(False, 0.65, 8, R, False)
        for name, prec, form, d in FORMS:
            tp = fl.train_params(d, W, K, 0.025, 0, fl.FELOG_SGNS_HOGWILD, 4096, prec, hogwild_form=form)
            pi, _, _ = fl.felog_embed(dg, L, 1, tp, fp, seed)
            out[name] = evaluate.link_auc(pi, sp.pos, sp.neg)
        # tile form: 3 rounds, 128 shared negatives on both sides (the serial
        # binary64 tile oracle is the slow one: about 20 s per seed here)
        fp3 = fl.feedback_params(False, 0.65, 8, TILE_R, False)
        T3 = TILE_R * int((tr.degrees() > 0).sum()) * L
        tp = fl.train_params(DIM, W, K, 0.025, T3, fl.FELOG_SGNS_TILE, 1, fl.FELOG_BF16_SR, tile_negatives=TILE_NS)
        pi, _, _ = fl.felog_embed(dg, L, 1, tp, fp3, seed)
        out["tile"] = evaluate.link_auc(pi, sp.pos, sp.neg)
        rt, _, _ = orc.embed(tr.offsets, tr.cols, L, 1, DIM, W, K, 0.025, False, 0.65, 8, TILE_R, False, seed,
                             mode="tile", B=TILE_NS, T=T3)
        out["oracle_tile"] = orc.link_auc(rt, sp.pos, sp.neg)
        res.append(out)
    return res


def test_hogwild_auc_within_tolerance_of_serial_oracle(runs):
    d = np.array([r["hogwild"] - r["oracle"] for r in runs])
    print("hogwild - oracle AUC per seed:", d.round(4))
    assert abs(d.mean()) <= 0.005


def test_bf16_auc_within_tolerance_of_serial_oracle(runs):
    d = np.array([r["bf16"] - r["oracle"] for r in runs])
    print("bf16 - oracle AUC per seed:", d.round(4))
    assert abs(d.mean()) <= 0.005


@pytest.mark.parametrize("form", ["staged", "staged_bf16", "prefetch", "prefetch_128", "prefetch_bf16",
                                  "bf16_128", "bulk", "bulk_128", "prefetch_bf16_64"])
def test_other_hogwild_forms_auc_within_tolerance_of_serial_oracle(runs, form):
    """The staged form (window phi_in increments summed in shared memory and
    added when a position leaves the window), the prefetching form (rows of
    the next step copied to shared memory during this one) and the bulk
    form (row increments added by the bulk-copy engine) keep the per-pair
    estimator.  Each is held to the oracle of its own dimension."""
    dim = next(f[3] for f in FORMS if f[0] == form)
    d = np.array([r[form] - r[f"oracle{dim}"] for r in runs])
    print(f"{form} - oracle AUC per seed:", d.round(4))
    assert abs(d.mean()) <= 0.005


def test_tile_auc_within_tolerance_of_serial_tile_oracle(runs):
    """The shared-negatives tile form changes the estimator (Ns draws per
    tile of weight K/Ns instead of K per pair), so it is held to the oracle of
    that estimator run serially (tiles in order, binary64): on this graph
    the GPU runs its tiles in order too.  Against the per-pair oracle it is
    only reported."""
    d = np.array([r["tile"] - r["oracle_tile"] for r in runs])
    print("tile (bf16, 3 rounds) - serial tile oracle AUC per seed:", d.round(4))
    assert abs(d.mean()) <= 0.005
