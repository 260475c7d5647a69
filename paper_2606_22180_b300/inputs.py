"""Seeded synthetic input generators: graphs, link-prediction splits.

This module holds none of the embedding method's arithmetic.  It builds the
graphs the method runs on and the held-out edge sets it is evaluated on, using
numpy's PCG64 generator; both the CUDA path and the CPU oracle receive its
outputs as plain arrays.

The paper's datasets (Table 3) are not available, so two synthetic families
stand in for them:

* a planted-partition stochastic block model (homophilic communities, the
  regime the neighbourhood-consistency feedback of Section 5.1 targets);
* R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004), the generator the paper
  itself uses for its scalability runs (Section 6.1, Section 6.3).

Every graph is returned as an undirected, unweighted CSR (the graph model of
Section 2, Table 1): int32 ``offsets[n+1]``, int32 ``cols[nnz]``, each row
sorted ascending, no self loops, no duplicate entries, and symmetric
(``u`` lists ``v`` iff ``v`` lists ``u``).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class CSR:
    """Undirected graph in compressed sparse row form (host arrays)."""

    offsets: np.ndarray  # int32 [n+1]
    cols: np.ndarray  # int32 [nnz]

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.cols.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))

    def n_isolated(self) -> int:
        return int((self.degrees() == 0).sum())


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray) -> CSR:
    """Symmetrise an edge list, drop self loops and duplicates, build CSR."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    a = np.concatenate([src, dst])
    b = np.concatenate([dst, src])
    key = a * np.int64(n) + b
    key.sort(kind="stable")  # radix sort on int64 keys: rows, then columns
    if key.shape[0]:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]  # drop duplicates
    rows = key // n
    cols = (key % n).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    if offsets[-1] >= 2**31:
        raise ValueError("graph too large for int32 CSR offsets")
    return CSR(offsets.astype(np.int32), cols)


def _upper_triangle_decode(idx: np.ndarray, na: int) -> tuple[np.ndarray, np.ndarray]:
    """Row-major index over the strict upper triangle of an na x na matrix -> (i, j)."""
    i = np.floor((2 * na - 1 - np.sqrt((2.0 * na - 1) ** 2 - 8.0 * idx)) / 2).astype(np.int64)
    i = np.clip(i, 0, max(na - 2, 0))
    for _ in range(3):  # repair floating-point error at row boundaries
        start = i * (2 * na - i - 1) // 2
        i = np.where(start > idx, i - 1, i)
        nxt = (i + 1) * (2 * na - i - 2) // 2
        i = np.where(idx >= nxt, i + 1, i)
    start = i * (2 * na - i - 1) // 2
    return i, idx - start + i + 1


def _sample_pairs_in_block(rng, lo_a, na, lo_b, nb, same, p):
    """Bernoulli(p) edges between blocks A and B (A == B: unordered pairs)."""
    total = na * (na - 1) // 2 if same else na * nb
    if total == 0 or p <= 0.0:
        return np.empty(0, np.int64), np.empty(0, np.int64)
    m = int(rng.binomial(total, p))
    if m == 0:
        return np.empty(0, np.int64), np.empty(0, np.int64)
    # a uniform m-subset of the pair indices: G(n, p) restricted to the block
    if total <= 4 * m or total < 1 << 22:
        idx = rng.choice(total, size=m, replace=False)
    else:
        idx = np.unique(rng.integers(0, total, size=int(m * 1.1) + 16))
        while idx.shape[0] < m:
            idx = np.unique(np.concatenate([idx, rng.integers(0, total, size=m)]))
        idx = rng.permutation(idx)[:m]
    idx = idx.astype(np.int64)
    if same:
        i, j = _upper_triangle_decode(idx, na)
        return lo_a + i, lo_a + j
    return lo_a + idx // nb, lo_b + idx % nb


def sbm(n: int, communities: int, p_in: float, p_out: float, seed: int,
        relabel: bool = False) -> tuple[CSR, np.ndarray]:
    """Planted-partition SBM with ``communities`` near-equal blocks.

    Returns the CSR and the community label of every node.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.full(communities, n // communities, dtype=np.int64)
    sizes[: n % communities] += 1
    lo = np.concatenate([[0], np.cumsum(sizes)])
    src, dst = [], []
    for a in range(communities):
        for b in range(a, communities):
            s, d = _sample_pairs_in_block(rng, lo[a], sizes[a], lo[b], sizes[b], a == b,
                                          p_in if a == b else p_out)
            src.append(s)
            dst.append(d)
    src = np.concatenate(src) if src else np.empty(0, np.int64)
    dst = np.concatenate(dst) if dst else np.empty(0, np.int64)
    labels = np.repeat(np.arange(communities, dtype=np.int32), sizes)
    if relabel:
        perm = rng.permutation(n)
        src, dst = perm[src], perm[dst]
        new_labels = np.empty_like(labels)
        new_labels[perm] = labels
        labels = new_labels
    return csr_from_edges(n, src, dst), labels


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, relabel: bool = True) -> CSR:
    """R-MAT graph with 2**scale nodes and edge_factor * 2**scale drawn edges.

    Each edge picks one quadrant per level with probabilities (a, b, c, d);
    the result is symmetrised, loop-free, deduplicated and (by default)
    relabelled by a seeded random permutation so node ids carry no degree
    order.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 1 << scale
    m = edge_factor * n
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    ab, abc = a + b, a + b + c
    chunk = 1 << 24
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        s = np.zeros(hi - lo, dtype=np.int64)
        t = np.zeros(hi - lo, dtype=np.int64)
        for _level in range(scale):
            r = rng.random(hi - lo, dtype=np.float32)
            ubit = r >= ab
            vbit = ((r >= a) & (r < ab)) | (r >= abc)
            s = (s << 1) | ubit
            t = (t << 1) | vbit
        src[lo:hi] = s
        dst[lo:hi] = t
    if relabel:
        perm = rng.permutation(n).astype(np.int64)
        src, dst = perm[src], perm[dst]
    return csr_from_edges(n, src, dst)


@dataclasses.dataclass
class LinkSplit:
    """Link-prediction split: a training graph plus scored test pairs."""

    train: CSR
    pos: np.ndarray  # int32 [P, 2] held-out edges (u < v)
    neg: np.ndarray  # int32 [P, 2] node pairs that are not edges of the full graph


def link_split(g: CSR, holdout: float, seed: int) -> LinkSplit:
    """Hold out a uniform fraction of undirected edges; draw as many non-edges.

    The held-out edges are removed from the training graph (Section 6.4 uses
    the same protocol with a 50 % hold-out; the workloads here use 10 %).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = g.n
    deg = g.degrees()
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    cols = g.cols.astype(np.int64)
    up = rows < cols
    u, v = rows[up], cols[up]
    m = u.shape[0]
    n_test = int(round(holdout * m))
    pick = np.zeros(m, dtype=bool)
    pick[rng.choice(m, size=n_test, replace=False)] = True
    train = csr_from_edges(n, u[~pick], v[~pick])
    pos = np.stack([u[pick], v[pick]], axis=1).astype(np.int32)
    # negatives: uniform pairs u != v that are not edges of the full graph
    edge_keys = np.sort(rows * np.int64(n) + cols)
    negs = np.empty((0, 2), dtype=np.int64)
    while negs.shape[0] < n_test:
        want = (n_test - negs.shape[0]) * 2 + 16
        a = rng.integers(0, n, size=want)
        b = rng.integers(0, n, size=want)
        ok = a != b
        a, b = a[ok], b[ok]
        key = a * np.int64(n) + b
        pos_in = np.searchsorted(edge_keys, key)
        pos_in = np.minimum(pos_in, edge_keys.shape[0] - 1) if edge_keys.shape[0] else pos_in
        is_edge = (edge_keys[pos_in] == key) if edge_keys.shape[0] else np.zeros_like(ok[ok])
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        negs = np.concatenate([negs, np.stack([lo[~is_edge], hi[~is_edge]], axis=1)])
    neg = negs[:n_test].astype(np.int32)
    return LinkSplit(train, pos, neg)


# ---------------------------------------------------------------------------
# Named workloads.  Sizes follow the synthetic stand-ins for the paper's
# graphs: a CPU-sized planted partition, R-MAT at scale 20 and 22.
# ---------------------------------------------------------------------------

def workload_sbm1000(seed: int = 0) -> tuple[CSR, np.ndarray]:
    """1,000-node SBM, 8 equal communities, p_in 0.04, p_out 0.002."""
    return sbm(1000, 8, 0.04, 0.002, seed)


def workload_rmat(scale: int, seed: int, edge_factor: int = 16) -> CSR:
    """R-MAT with (a, b, c, d) = (0.57, 0.19, 0.19, 0.05)."""
    return rmat(scale, edge_factor, 0.57, 0.19, 0.19, seed=seed)


def sbm_degree(n: int, communities: int, degree: float, seed: int, ratio: float = 20.0) -> CSR:
    """Planted partition with p_in / p_out = ratio and expected degree ~degree."""
    size = n / communities
    p_in = degree / ((size - 1) + (n - size) / ratio)
    p_in = min(p_in, 1.0)
    g, _ = sbm(n, communities, p_in, p_in / ratio, seed)
    return g


def rmat_nodes(n: int, degree: float, seed: int, a=0.57, b=0.19, c=0.19) -> CSR:
    """R-MAT on the smallest power of two >= n, restricted to nodes < n,
    with about degree * n / 2 drawn edges kept."""
    scale = max(1, int(np.ceil(np.log2(n))))
    N = 1 << scale
    keep_frac = (n / N) ** 2
    m = int(degree * n / 2 / max(keep_frac, 1e-3))
    rng = np.random.Generator(np.random.PCG64(seed))
    ab, abc = a + b, a + b + c
    s = np.zeros(m, dtype=np.int64)
    t = np.zeros(m, dtype=np.int64)
    for _level in range(scale):
        r = rng.random(m, dtype=np.float32)
        s = (s << 1) | (r >= ab)
        t = (t << 1) | (((r >= a) & (r < ab)) | (r >= abc))
    perm = rng.permutation(N).astype(np.int64)
    s, t = perm[s], perm[t]
    ok = (s < n) & (t < n)
    return csr_from_edges(n, s[ok], t[ok])


def _mix_one(spec):
    kind, n, k, deg, gseed = spec
    if kind == "sbm":
        return sbm_degree(n, k, deg, seed=gseed)
    return rmat_nodes(n, deg, seed=gseed)


def graph_mix(count: int, seed: int, n_lo: int, n_hi: int, deg_lo: float = 8.0, deg_hi: float = 32.0,
              dims=(64, 128), workers: int = 1):
    """A mix of jobs for the batching and serving forms: half planted
    partitions (4..32 communities), half R-MAT; node counts log-uniform in
    [n_lo, n_hi], average degree uniform in [deg_lo, deg_hi], embedding
    dimension drawn from dims.  Returns a list of (CSR, dim).  Every graph's
    parameters and seed are drawn first, in order, so the graphs do not
    depend on `workers` (> 1: generated in that many spawned processes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs, out_dims = [], []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        deg = float(rng.uniform(deg_lo, deg_hi))
        dim = int(dims[int(rng.integers(0, len(dims)))])
        if i % 2 == 0:
            k = int(rng.integers(4, 33))
            specs.append(("sbm", n, k, deg, int(rng.integers(1 << 31))))
        else:
            specs.append(("rmat", n, 0, deg, int(rng.integers(1 << 31))))
        out_dims.append(dim)
    if workers > 1 and count > 1:
        import concurrent.futures
        import multiprocessing

        ctx = multiprocessing.get_context("spawn")
        with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
            graphs = list(ex.map(_mix_one, specs, chunksize=4))
    else:
        graphs = [_mix_one(sp) for sp in specs]
    return list(zip(graphs, out_dims))
