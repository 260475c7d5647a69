import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU-only case")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.lib()
    return oracle


def tiny_graph(name):
    """Small undirected graphs for brute-force checks, as CSR arrays."""
    from paper_2606_22180_b300.inputs import csr_from_edges

    edges = {
        "path4": (4, [(0, 1), (1, 2), (2, 3)]),
        "star4": (4, [(0, 1), (0, 2), (0, 3)]),
        "triangle_tail": (4, [(0, 1), (1, 2), (0, 2), (2, 3)]),
        "k4": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
        "cycle6": (6, [(i, (i + 1) % 6) for i in range(6)]),
        "with_isolated": (5, [(0, 1), (1, 2)]),
    }[name]
    n, e = edges
    e = np.array(e, dtype=np.int64).reshape(-1, 2)
    return csr_from_edges(n, e[:, 0], e[:, 1])
