"""Pins for the oracle's Philox4x32-10 against its published known answers."""
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4] | (w[5] << 32), w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_known_answers(orc, ctr, key, expect):
    assert list(orc.philox(key, ctr)) == expect


def test_uniform_words(orc):
    # chi-square over 256 bins of the top byte of 4 * 20000 words
    words = np.concatenate([orc.philox(12345, (i, 7, 9, 2)) for i in range(20000)])
    hist = np.bincount(words >> 24, minlength=256)
    p = stats.chisquare(hist).pvalue
    assert p > 1e-4


def test_counter_sensitivity(orc):
    # every counter word and the key change the output block
    base = orc.philox(1, (0, 0, 0, 0))
    for i in range(4):
        c = [0, 0, 0, 0]
        c[i] = 1
        assert not np.array_equal(orc.philox(1, c), base)
    assert not np.array_equal(orc.philox(2, (0, 0, 0, 0)), base)
    assert not np.array_equal(orc.philox(1 << 32, (0, 0, 0, 0)), base)
