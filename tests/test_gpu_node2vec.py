"""node2vec walks on the GPU against the oracle: bit-exact rows (same
Philox draws, same binary64 acceptance decisions), fused counts, dead
ends, and a sampled full-size check on R-MAT scale 20."""
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("graph,L,wpr,p,q,rnd", [("sbm", 80, 2, 0.5, 2.0, 0), ("sbm", 13, 1, 4.0, 0.25, 3),
                                                  ("rmat14", 40, 3, 1.0, 1.0, 1), ("rmat14", 80, 1, 0.25, 4.0, 7),
                                                  ("rmat14", 1, 2, 2.0, 2.0, 0)])
def test_node2vec_bit_exact(fl, orc, graph, L, wpr, p, q, rnd):
    g = inputs.workload_sbm1000(0)[0] if graph == "sbm" else inputs.rmat(14, 16, seed=5)
    starts = np.arange(g.n, dtype=np.int32)  # isolated starts included (dead ends)
    ref = orc.walk_node2vec(g.offsets, g.cols, starts, L, wpr, p, q, 9, rnd)
    dg = fl.DeviceGraph.from_host(g)
    counts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    out = fl.felog_walk_node2vec(dg, _dev(starts), starts.size, L, wpr, p, q, 9, rnd, counts=counts)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), orc.counts(ref, g.n).astype(np.int64))


@pytest.mark.parametrize("shift,L", [(1, 80), (2, 21), (0, 9)])
def test_node2vec_rows_off_16_byte_boundary(fl, orc, shift, L):
    """Rows that do not start on 16-byte boundaries (the 8-step groups are
    then stored one id at a time) and lengths that leave a partial group."""
    g = inputs.rmat(12, 16, seed=3)
    starts = np.arange(g.n, dtype=np.int32)
    ref = orc.walk_node2vec(g.offsets, g.cols, starts, L, 1, 0.5, 2.0, 6, 1)
    dg = fl.DeviceGraph.from_host(g)
    big = torch.full((g.n * L + 4,), 7, dtype=torch.int32, device="cuda")
    out = big[shift:shift + g.n * L].view(g.n, L)
    fl.felog_walk_node2vec(dg, _dev(starts), starts.size, L, 1, 0.5, 2.0, 6, 1, out=out)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert int(big[:shift].ne(7).sum()) == 0 and int(big[shift + g.n * L:].ne(7).sum()) == 0


@pytest.mark.parametrize("p,q", [(1e6, 2e6), (1e-6, 3e5)])
def test_node2vec_attempt_cap_bit_exact(fl, orc, p, q):
    """Acceptance ratios near 1e-6: most steps exhaust the 64 attempts and
    take the 64th proposal (the last lane of the last round on the GPU)."""
    g = inputs.rmat(10, 8, seed=2)
    starts = np.arange(g.n, dtype=np.int32)
    ref = orc.walk_node2vec(g.offsets, g.cols, starts, 24, 2, p, q, 3, 5)
    dg = fl.DeviceGraph.from_host(g)
    counts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    out = fl.felog_walk_node2vec(dg, _dev(starts), starts.size, 24, 2, p, q, 3, 5, counts=counts)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), orc.counts(ref, g.n).astype(np.int64))


@pytest.mark.slow
def test_node2vec_rmat20_sampled(fl, orc):
    """Full-size graph, all non-isolated starts on the GPU; 2,000 sampled
    walkers recomputed by the oracle must match their rows (a row depends
    only on its start node, rep and round)."""
    g = inputs.workload_rmat(20, 1)
    starts = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
    dg = fl.DeviceGraph.from_host(g)
    out = fl.felog_walk_node2vec(dg, _dev(starts), starts.size, 80, 1, 0.5, 2.0, 4, 2).cpu().numpy()
    pick = np.random.default_rng(0).choice(starts.size, 2000, replace=False)
    ref = orc.walk_node2vec(g.offsets, g.cols, starts[pick], 80, 1, 0.5, 2.0, 4, 2)
    assert np.array_equal(out[pick], ref)
