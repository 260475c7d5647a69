"""The timed CPU baseline runs the oracle's own routines on every host core.

Walks and Psi are independent per start and per node, so the parallel forms
must equal the single-threaded oracle bit for bit; the Hogwild SGNS form
must train exactly the serial oracle's tables on one thread (chunks in
order; its loss is summed per chunk) and stay close to it on many.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2606_22180_b300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    return inputs.rmat(12, 8, seed=4)


def test_parallel_walks_equal_the_oracle(orc, g):
    starts = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
    for rnd in (0, 3):
        a = orc.walk(g.offsets, g.cols, starts, 30, 1, 9, rnd)
        b = orc.baseline_walk(g.offsets, g.cols, starts, 30, 9, rnd)
        assert np.array_equal(a, b)


def test_parallel_psi_equals_the_oracle(orc, g):
    rng = np.random.default_rng(2)
    phi = rng.normal(size=(g.n, 32))
    nodes = np.nonzero(g.degrees() > 0)[0].astype(np.int32)[:500]
    got = orc.baseline_psi(g.offsets, g.cols, phi, 8, 5, 1, nodes)
    ref = np.array([orc.psi_node(g.offsets, g.cols, phi, 8, 5, 1, int(v)) for v in nodes])
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))


_ONE_THREAD = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
import oracle
from paper_2606_22180_b300 import inputs
g = inputs.rmat(11, 8, seed=4)
starts = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
W = oracle.walk(g.offsets, g.cols, starts, 20, 1, 3, 0)
_, thr, alias, S = oracle.noise_table(oracle.counts(W, g.n))
T = 10 * W.size
a_in, a_out = oracle.init_tables(g.n, 16, 3)
b_in, b_out = a_in.copy(), a_out.copy()
la = oracle.sgns_serial(W, g.n, 16, 3, 3, 0.025, T, thr, alias, S, 3, 0, 0, a_in, a_out)
lb = oracle.baseline_sgns_hogwild(W, g.n, 16, 3, 3, 0.025, T, thr, alias, S, 3, 0, 0, b_in, b_out)
assert oracle.baseline_threads() == 1
# identical tables; the loss is summed per chunk of walks, so only its rounding differs
assert np.array_equal(a_in, b_in) and np.array_equal(a_out, b_out)
assert abs(la - lb) <= 1e-12 * abs(la)
print("ok")
"""


def test_hogwild_on_one_thread_is_the_serial_oracle(orc):
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", _ONE_THREAD.format(root=ROOT)], env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0 and "ok" in out.stdout, out.stderr


def test_hogwild_on_all_threads_stays_close(orc, g):
    starts = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
    W = orc.walk(g.offsets, g.cols, starts, 20, 1, 3, 0)
    _, thr, alias, S = orc.noise_table(orc.counts(W, g.n))
    T = 10 * W.size
    a_in, a_out = orc.init_tables(g.n, 16, 3)
    b_in, b_out = a_in.copy(), a_out.copy()
    la = orc.sgns_serial(W, g.n, 16, 3, 3, 0.025, T, thr, alias, S, 3, 0, 0, a_in, a_out)
    lb = orc.baseline_sgns_hogwild(W, g.n, 16, 3, 3, 0.025, T, thr, alias, S, 3, 0, 0, b_in, b_out)
    assert np.isfinite(b_in).all() and np.isfinite(b_out).all()
    assert abs(la - lb) / la < 0.01
