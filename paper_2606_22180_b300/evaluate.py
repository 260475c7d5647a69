"""Link-prediction AUC of an embedding (Section 6.4), outside the hot path.

Scores are dot products phi(u) . phi(v) of held-out edges and of non-edges;
the AUC is the Mann-Whitney statistic U / (P * N) computed from mid-ranks
(ties count one half).  Used to check that a run reached a given quality;
it is not part of the timed path.
"""
from __future__ import annotations

import numpy as np
import torch
from scipy.stats import rankdata


def link_scores(phi, pairs: np.ndarray) -> np.ndarray:
    if isinstance(phi, torch.Tensor):
        p = torch.as_tensor(pairs, dtype=torch.long, device=phi.device)
        a = phi[p[:, 0]].double()
        b = phi[p[:, 1]].double()
        return (a * b).sum(1).cpu().numpy()
    phi = np.asarray(phi, dtype=np.float64)
    return np.einsum("ij,ij->i", phi[pairs[:, 0]], phi[pairs[:, 1]])


def auc(pos_scores: np.ndarray, neg_scores: np.ndarray) -> float:
    P, N = pos_scores.shape[0], neg_scores.shape[0]
    ranks = rankdata(np.concatenate([pos_scores, neg_scores]))
    U = ranks[:P].sum() - P * (P + 1) / 2.0
    return float(U / (P * N))


def link_auc(phi, pos: np.ndarray, neg: np.ndarray) -> float:
    return auc(link_scores(phi, pos), link_scores(phi, neg))
