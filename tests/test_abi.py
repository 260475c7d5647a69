"""The C-ABI library builds for sm_103a, loads, and exports every symbol the
header declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(felog_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_22180_b300 import build, felog

    build.build()
    return felog.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2606_22180_b300 import felog

    assert sorted(felog.SYMBOLS) == _declared()


def test_host_side_argument_checks(lib):
    # argument validation happens before any CUDA call, so these need no GPU
    from paper_2606_22180_b300 import felog

    assert lib.felog_status_string(0) == b"ok"
    bad = felog._TrainParams(100, 5, 5, 0.025, 1, 0, 1, 0, 0, 0)  # dim 100 unsupported
    assert lib.felog_train_workspace_bytes(1, 40, 10, ctypes.byref(bad)) == 0
    good = felog._TrainParams(64, 5, 5, 0.025, 1, 0, 1, 0, 0, 0)
    assert lib.felog_train_workspace_bytes(1, 40, 10, ctypes.byref(good)) > 0
    # TILE mode: dim <= 128, tile_negatives a multiple of 128 in [128, 512] (0 = 512)
    for dim, ns, ok in [(128, 0, True), (64, 128, True), (32, 512, True), (128, 384, True),
                        (256, 0, False), (128, 64, False), (128, 640, False), (128, 200, False)]:
        tp = felog.train_params(dim, 5, 5, 0.025, 1, felog.FELOG_SGNS_TILE, 1, 0, tile_negatives=ns)
        assert (lib.felog_train_workspace_bytes(1, 40, 10, ctypes.byref(tp)) > 0) == ok, (dim, ns)
    wp = felog._WalkParams(0, 1)  # zero-length walks rejected
    csr = felog._Csr(1, 1, 4, 4)
    assert lib.felog_walk(ctypes.byref(csr), 1, 1, ctypes.byref(wp), 0, 0, 1, None, None) == 1
    csr_bad = felog._Csr(1, 1, -1, 4)
    wp = felog._WalkParams(4, 1)
    assert lib.felog_walk(ctypes.byref(csr_bad), 1, 1, ctypes.byref(wp), 0, 0, 1, None, None) == 2
    assert lib.felog_embed_workspace_bytes(10, ctypes.byref(wp), ctypes.byref(bad)) == 0
    # stochastic rounding: negative length or missing buffers rejected, empty input is a no-op
    assert lib.felog_sr_bf16(None, None, -1, None, None) == 1
    assert lib.felog_sr_bf16(None, None, 5, None, None) == 1
    assert lib.felog_sr_bf16(None, None, 0, None, None) == 0
    # grid-barrier check and batch knobs: out-of-range arguments rejected before any CUDA call
    assert lib.felog_grid_barrier_check(-1, 1, 1.0, None, None) == 1
    assert lib.felog_grid_barrier_check(0, 0, 1.0, None, None) == 1
    assert lib.felog_grid_barrier_check(0, 1, 0.0, None, None) == 1
    assert lib.felog_grid_barrier_check(0, 1, 61.0, None, None) == 1
    t = felog.Tuning(256, 2, 16, 0, 2)
    assert lib.felog_batch_set_tuning(None, ctypes.byref(t)) == 1
    assert lib.felog_batch_set_wait_limit(None, 1.0) == 1


def test_product_path_has_no_cpu_fallback():
    import torch

    from paper_2606_22180_b300 import felog

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(felog.FelogError):
        felog.felog_init_tables(4, 64, felog.FELOG_FP32, 0)
