"""FaBC codec on the GPU (Section 5.2.2) against the oracle: the selection
(Eq. 8) equal, the encoded bytes identical, decode the exact inverse; at
full size (R-MAT scale 20 corpus) the round trip and the Eq. 7 size."""
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


def _dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def _corpus(orc, scale, L, n_starts, seed):
    g = inputs.rmat(scale, 16, seed=seed)
    starts = np.nonzero(g.degrees() > 0)[0][:n_starts].astype(np.int32)
    W = orc.walk(g.offsets, g.cols, starts, L, 1, seed, 0)
    return g, W


@pytest.mark.parametrize("scale,L,kmax", [(10, 80, 32), (12, 40, 4), (14, 7, 32)])
def test_select_matches_oracle(fl, orc, scale, L, kmax):
    g, W = _corpus(orc, scale, L, 3000, 2)
    counts = orc.counts(W, g.n)
    ids_o, F_o = orc.fabc_select(counts, L, kmax)
    ids_g, F_g = fl.felog_fabc_select(_dev(counts.astype(np.int32)), L, kmax)
    assert ids_g == list(ids_o) and F_g == F_o


def test_select_hand_profile(fl, orc):
    """A profile where two nodes dominate (the paper's example narrative)."""
    counts = np.zeros(1000, np.uint32)
    counts[[500, 17]] = 300_000
    counts[3] = 50_000
    counts[600:1000] = 437  # filler clear of the nodes above
    ids_o, F_o = orc.fabc_select(counts, 80, 32)
    ids_g, F_g = fl.felog_fabc_select(_dev(counts.astype(np.int32)), 80, 32)
    assert ids_g == list(ids_o) == [17, 500] and F_g == F_o


@pytest.mark.parametrize("N,L,k,pad", [(1, 80, 1, False), (333, 80, 2, True), (257, 40, 3, True),
                                       (100, 13, 1, True), (64, 33, 5, False), (77, 80, 0, True),
                                       (50, 1, 2, False), (300, 100, 32, True),
                                       # tails off a 4-byte boundary (N k ceil(L/8) not a multiple of 4)
                                       (101, 13, 1, True), (99, 24, 2, True), (65, 33, 5, True)])
def test_encode_bytes_match_oracle_and_decode_inverts(fl, orc, N, L, k, pad):
    rng = np.random.default_rng(N * 7 + L + k)
    p = np.array([0.25, 0.2, 0.1] + [0.45 / 61] * 61)
    W = rng.choice(64, size=(N, L), p=p / p.sum()).astype(np.int32)
    if pad:
        W[::3, L // 2:] = -1
    ids = rng.permutation(64)[:k].astype(np.int32) if k else np.zeros(0, np.int32)
    ids[:min(k, 3)] = np.arange(min(k, 3))  # the frequent nodes first
    ref = orc.fabc_encode(W, ids)
    buf, tail = fl.felog_fabc_encode(_dev(W), _dev(ids))
    size = fl.fabc_encoded_bytes(N, L, k, int(tail.item()))
    assert size == ref.size
    assert np.array_equal(buf[:size].cpu().numpy(), ref)
    back = fl.felog_fabc_decode(buf[:size].clone(), N, L, k)
    assert np.array_equal(back.cpu().numpy(), W)
    # the oracle's buffer decodes on the GPU too
    back2 = fl.felog_fabc_decode(_dev(ref), N, L, k)
    assert np.array_equal(back2.cpu().numpy(), W)


@pytest.mark.parametrize("N,L,k", [(9, 3000, 2), (5, 7000, 3), (131, 100, 4), (70, 81, 0), (200, 1200, 1),
                                   (3, 1505, 2)])
def test_tile_shapes_and_long_sequences(fl, orc, N, L, k):
    """Tiles of 64 sequences with a ragged last one, tile sizes other than 64
    (L = 100, 1200), and sequences too long to stage (L = 1505 and 3000 for
    encode, 7000 for both) against the oracle's bytes."""
    rng = np.random.default_rng(N + L + k)
    W = rng.integers(0, 16, size=(N, L)).astype(np.int32)
    W[::4, L // 3:] = -1
    ids = np.arange(k, dtype=np.int32) * 2
    ref = orc.fabc_encode(W, ids)
    buf, tail = fl.felog_fabc_encode(_dev(W), _dev(ids))
    size = fl.fabc_encoded_bytes(N, L, k, int(tail.item()))
    assert size == ref.size and np.array_equal(buf[:size].cpu().numpy(), ref)
    assert np.array_equal(fl.felog_fabc_decode(_dev(ref), N, L, k).cpu().numpy(), W)


@pytest.mark.parametrize("shift", [1, 2, 3])
@pytest.mark.parametrize("k", [0, 2])
def test_walks_off_16_byte_boundary(fl, orc, shift, k):
    """Walks starting 4, 8 or 12 bytes past a 16-byte boundary (the staging
    and the k = 0 copy fall back from 16-byte to 4-byte accesses) encode
    and decode the same."""
    N, L = 150, 80
    rng = np.random.default_rng(shift)
    W = rng.integers(0, 8, size=(N, L)).astype(np.int32)
    ids = np.array([1, 5][:k], np.int32)
    big = torch.zeros(N * L + 4, dtype=torch.int32, device="cuda")
    view = big[shift:shift + N * L].view(N, L)
    view.copy_(_dev(W))
    ref = orc.fabc_encode(W, ids)
    buf, tail = fl.felog_fabc_encode(view, _dev(ids))
    size = fl.fabc_encoded_bytes(N, L, k, int(tail.item()))
    assert np.array_equal(buf[:size].cpu().numpy(), ref)
    out = big[shift:shift + N * L].view(N, L)
    out.zero_()
    fl.felog_fabc_decode(buf[:size].clone(), N, L, k, walks=out)
    assert np.array_equal(out.cpu().numpy(), W)


def test_unaligned_buffers_are_refused(fl):
    """The encoded buffer must start on a 4-byte boundary (documented)."""
    W = torch.zeros((4, 80), dtype=torch.int32, device="cuda")
    ids = torch.tensor([0], dtype=torch.int32, device="cuda")
    buf, tail = fl.felog_fabc_encode(W, ids)
    size = fl.fabc_encoded_bytes(4, 80, 1, int(tail.item()))
    raw = torch.zeros(size + 4, dtype=torch.uint8, device="cuda")
    raw[1:1 + size] = buf[:size]
    with pytest.raises(fl.FelogError):
        fl.felog_fabc_decode(raw[1:1 + size], 4, 80, 1)
    assert torch.equal(fl.felog_fabc_decode(raw[1:1 + size].clone(), 4, 80, 1), W)


@pytest.mark.parametrize("k", [0, 1])
def test_damaged_tail_decodes_as_minus_one(fl, orc, k):
    """A buffer cut short inside the tail: the ids past the end come back
    as -1 and nothing past in_bytes is read."""
    N, L = 100, 40
    rng = np.random.default_rng(9)
    W = rng.integers(0, 6, size=(N, L)).astype(np.int32)
    ids = np.array([0][:k], np.int32)
    ref = orc.fabc_encode(W, ids)
    cut = ref.size - 4 * 37
    back = fl.felog_fabc_decode(_dev(ref[:cut]), N, L, k).cpu().numpy()
    want = W.copy()
    tail_pos = np.argwhere(~np.isin(W.ravel(), ids)).ravel()  # tail positions in order
    want.ravel()[tail_pos[-37:]] = -1
    assert np.array_equal(back, want)


def test_encode_into_reused_buffers(fl, orc):
    """A caller's output, tail count and workspace reused across encodes of
    different corpora give each corpus's own bytes."""
    rng = np.random.default_rng(4)
    N, L = 200, 80
    ws = fl.fabc_workspace(N)
    ids = np.array([3, 7], np.int32)
    out = tail = None
    for trial in range(3):
        W = rng.integers(0, 12, size=(N, L)).astype(np.int32)
        ref = orc.fabc_encode(W, ids)
        out, tail = fl.felog_fabc_encode(_dev(W), _dev(ids), workspace=ws, out=out, tail=tail)
        size = fl.fabc_encoded_bytes(N, L, 2, int(tail.item()))
        assert np.array_equal(out[:size].cpu().numpy(), ref), trial


def test_empty_and_degenerate(fl):
    W = torch.zeros((0, 80), dtype=torch.int32, device="cuda")
    ids = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    buf, tail = fl.felog_fabc_encode(W, ids)
    assert int(tail.item()) == 0
    out = fl.felog_fabc_decode(buf, 0, 80, 2)
    assert out.shape == (0, 80)


@pytest.mark.slow
def test_full_size_round_trip_rmat20(fl):
    """One round of walks on the R-MAT scale 20 bench graph (631,609 walks of
    80): round trip exact, size equal to Eq. 7 with the covered fraction, for
    the Eq. 8 selection and for the forced top-2."""
    split = inputs.link_split(inputs.workload_rmat(20, 1), 0.1, 1)
    dg = fl.DeviceGraph.from_host(split.train)
    starts = torch.nonzero(dg.offsets[1:] - dg.offsets[:-1]).flatten().to(torch.int32)
    counts = torch.zeros(dg.n, dtype=torch.int32, device="cuda")
    W = fl.felog_walk(dg, starts, starts.numel(), 80, 1, 1, 0, counts=counts)
    ids, F = fl.felog_fabc_select(counts, 80, 32)
    for sel in (ids, torch.topk(counts.long(), 2).indices.tolist()):
        ids_d = torch.tensor(sel, dtype=torch.int32, device="cuda")
        buf, tail = fl.felog_fabc_encode(W, ids_d)
        N, k = W.shape[0], len(sel)
        size = fl.fabc_encoded_bytes(N, 80, k, int(tail.item()))
        cov = float(torch.isin(W, ids_d).double().mean().item()) if k else 0.0
        assert size == round((1 - cov + k / 80 + k / 32) * 4 * N * 80)
        back = fl.felog_fabc_decode(buf[:size].clone(), N, 80, k)
        assert torch.equal(back, W)
