"""Device-side validation of caller graphs at the boundary.

felog_validate_csr reports each kind of malformed CSR through its status
word; felog_embed and felog_batch_create run the check before any kernel
gathers through the graph and return FELOG_ERR_BAD_CSR.  Every malformed
graph here is only ever read by the validation kernel, which reads columns
only where a row's offsets lie inside the column array.
"""
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


def _graph(fl, offsets, cols):
    return fl.DeviceGraph(torch.tensor(offsets, dtype=torch.int32, device="cuda"),
                          torch.tensor(cols, dtype=torch.int32, device="cuda"))


# a path 0 - 1 - 2 - 3 plus the edge 1 - 3
GOOD = ([0, 1, 4, 6, 8], [1, 0, 2, 3, 1, 3, 1, 2])


def _status(fl, g, starts=None):
    st = fl.felog_validate_csr(g, None if starts is None else torch.tensor(starts, dtype=torch.int32, device="cuda"))
    return int(st.item())


def test_valid_graphs_pass(fl):
    assert _status(fl, _graph(fl, *GOOD)) == 0
    assert _status(fl, _graph(fl, *GOOD), [0, 3, 2]) == 0
    g = inputs.rmat(14, 16, seed=5)
    assert _status(fl, fl.DeviceGraph.from_host(g), np.nonzero(g.degrees() > 0)[0]) == 0
    # isolated nodes and an empty graph are valid
    assert _status(fl, _graph(fl, [0, 0, 0], [])) == 0


@pytest.mark.parametrize("offsets,cols,bit", [
    ([1, 1, 4, 6, 8], GOOD[1], 1),                    # offsets[0] != 0
    ([0, 1, 4, 6, 7], GOOD[1], 1),                    # offsets[n] != nnz
    ([0, 1, 4, 6, 9], GOOD[1], 1),                    # a row past the column array
    ([0, 3, 1, 6, 8], GOOD[1], 2),                    # decreasing offsets
    ([0, 1, 4, 6, 8], [1, 0, 2, 7, 1, 3, 1, 2], 4),   # a column >= n
    ([0, 1, 4, 6, 8], [1, 0, 2, -3, 1, 3, 1, 2], 4),  # a negative column
    ([0, 1, 4, 6, 8], [1, 2, 0, 3, 1, 3, 1, 2], 8),   # a row out of order
    ([0, 1, 4, 6, 8], [1, 0, 2, 2, 1, 3, 1, 2], 8),   # a duplicate neighbour
    ([0, 1, 4, 6, 8], [1, 0, 1, 3, 1, 3, 1, 2], 16),  # a self loop (row 1 holds 1)
])
def test_each_malformation_is_reported(fl, offsets, cols, bit):
    st = _status(fl, _graph(fl, offsets, cols))
    assert st & bit, (st, bit)


def test_start_out_of_range(fl):
    assert _status(fl, _graph(fl, *GOOD), [0, 4]) == fl.CSR_START_RANGE
    assert _status(fl, _graph(fl, *GOOD), [-1]) == fl.CSR_START_RANGE


def test_embed_and_batch_reject_a_malformed_device_graph(fl):
    tp = fl.train_params(32, 2, 2, 0.025, 0, fl.FELOG_SGNS_HOGWILD, 64, fl.FELOG_FP32)
    fp = fl.feedback_params(False, 0.65, 8, 2, False)
    bad = _graph(fl, [0, 1, 4, 6, 8], [1, 0, 2, 70000, 1, 3, 1, 2])
    with pytest.raises(fl.FelogError, match="malformed"):
        fl.felog_embed(bad, 8, 1, tp, fp, 1)
    with pytest.raises(fl.FelogError, match="malformed"):
        fl.Batch([_graph(fl, *GOOD), bad], [32, 32], [1, 2], 8, 1, tp, fp)
    # the same calls on the well-formed graph run
    _, _, st = fl.felog_embed(_graph(fl, *GOOD), 8, 1, tp, fp, 1)
    assert len(st) == 2
    torch.cuda.synchronize()
