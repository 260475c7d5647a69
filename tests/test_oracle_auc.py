"""Pins for the oracle's link-prediction AUC (Section 6.4)."""
import numpy as np
from scipy import stats


def test_auc_special_cases(orc):
    assert orc.auc_pairs([3.0, 4.0], [1.0, 2.0]) == 1.0
    assert orc.auc_pairs([1.0, 2.0], [3.0, 4.0]) == 0.0
    assert orc.auc_pairs([1.0, 1.0], [1.0]) == 0.5
    # 3 of 4 pairs ordered, one tie: (1 + 1 + 0.5 + 0) / 4
    assert orc.auc_pairs([2.0, 1.0], [1.0, 3.0]) == 0.375


def test_auc_equals_mann_whitney(orc):
    rng = np.random.default_rng(0)
    pos = np.round(rng.normal(1.0, 1.0, 300), 1)  # rounding creates ties
    neg = np.round(rng.normal(0.0, 1.0, 250), 1)
    u = stats.mannwhitneyu(pos, neg, alternative="two-sided").statistic
    assert abs(orc.auc_pairs(pos, neg) - u / (300 * 250)) < 1e-12


def test_link_scores_are_dot_products(orc):
    rng = np.random.default_rng(1)
    phi = rng.normal(size=(20, 7))
    pairs = rng.integers(0, 20, size=(15, 2)).astype(np.int32)
    ref = (phi[pairs[:, 0]] * phi[pairs[:, 1]]).sum(1)
    assert np.allclose(orc.link_scores(phi, pairs), ref, rtol=1e-14, atol=1e-14)


def test_package_evaluator_matches_definition(orc):
    """The rank-based AUC the benchmark uses equals the oracle's pair count."""
    from paper_2606_22180_b300 import evaluate

    rng = np.random.default_rng(3)
    phi = rng.normal(size=(60, 8))
    pos = rng.integers(0, 60, size=(40, 2)).astype(np.int32)
    neg = rng.integers(0, 60, size=(45, 2)).astype(np.int32)
    assert abs(evaluate.link_auc(phi, pos, neg) - orc.link_auc(phi, pos, neg)) < 1e-12
    assert abs(evaluate.auc(np.array([1.0, 1.0]), np.array([1.0])) - 0.5) < 1e-15
