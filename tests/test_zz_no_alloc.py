"""The allocation-free compaction entry point, called through the C ABI.

Some callers cannot allocate device memory (a serving loop with a fixed
memory plan, or a host framework that owns every device allocation), so they
cannot hand the library a workspace.  felog_compact_active_noalloc keeps its
scratch in a static device array instead.  This file is collected last so a
failure here cannot hide the rest of the suite; it passes alone or after the
other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    from paper_2606_22180_b300 import build, felog

    build.build()
    felog.load()
    return felog


def _run_both(fl, flags):
    active = torch.from_numpy(flags).cuda()
    ref_starts, ref_cnt = fl.felog_compact_active(active)
    starts = torch.full((max(flags.shape[0], 1),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    fl.felog_compact_active_noalloc(active, starts, cnt)
    k = int(ref_cnt.item())
    assert int(cnt.item()) == k == int(flags.sum())
    assert torch.equal(starts[:k], ref_starts[:k])
    assert np.array_equal(starts[:k].cpu().numpy(), np.nonzero(flags)[0])


def test_noalloc_matches_workspace_compaction_twice(fl):
    rng = np.random.default_rng(0)
    # two calls in a row: a large dense input, then a small sparse one, so a
    # second call must not see the first call's tile counts
    big = (rng.random((1 << 22) + 5) < 0.6).astype(np.uint8)
    small = (rng.random(5000) < 0.05).astype(np.uint8)
    _run_both(fl, big)
    _run_both(fl, small)


def test_noalloc_rejects_sizes_beyond_its_scratch(fl):
    lib = fl.load()
    limit = lib.felog_compact_active_noalloc_max_n()
    assert limit == 1 << 24
    # rejected on the host before any launch: the pointers are never touched
    st = lib.felog_compact_active_noalloc(ctypes.c_void_p(16), limit + 1, ctypes.c_void_p(16),
                                          ctypes.c_void_p(16), ctypes.c_void_p(0))
    assert st == 1  # FELOG_ERR_INVALID_ARG
