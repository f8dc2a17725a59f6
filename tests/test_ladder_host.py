"""Host side of the length ladder: the lengths N_j = floor(n_min * 2^(j/steps))
(repeats dropped) from the C ABI against the formula written out here."""
import math

import pytest

from paper_2603_22245_gb300 import rotormap as rm


def formula(n_min, n_max, spo):
    out = []
    j = 0
    while True:
        v = math.floor(n_min * 2 ** (j / spo))
        if v > n_max:
            return out
        if not out or out[-1] != v:
            out.append(v)
        j += 1


@pytest.mark.parametrize("n_min,n_max,spo", [(100, 10000, 8), (100, 3000, 8), (1, 50, 8), (150, 150, 8),
                                             (40, 20000, 3), (100, 99, 8)])
def test_lengths_match_formula(n_min, n_max, spo):
    if n_max < n_min:
        assert rm.load().rope_ladder_lengths(n_min, n_max, spo, None, 0) == -1
        return
    assert rm.rope_ladder_lengths(n_min, n_max, spo) == formula(n_min, n_max, spo)


def test_default_ladder_has_54_lengths():
    lens = rm.rope_ladder_lengths(100, 10000, 8)
    assert len(lens) == 54 and lens[0] == 100 and lens[8] == 200 and lens[-1] <= 10000


@pytest.mark.parametrize("bad", [(0, 10, 8), (10, 5, 8), (10, 100, 0), (10, 100, 65)])
def test_invalid(bad):
    assert rm.load().rope_ladder_lengths(*bad, None, 0) == -1
