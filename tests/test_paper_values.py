"""Closed forms against the numbers the paper prints (tests/golden)."""
import math
import os

import pytest

from paper_1101_0876_gb300.analysis import (exact_energies, latent_heat,
                                            magnetization_jump_series)
from paper_1101_0876_gb300.workloads import beta_at, tc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden",
                      "paper_printed_values.txt")


def _rows(kind):
    out = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line and line[0] == kind:
                out.append([int(line[1])] + [float(x) for x in line[2:]])
    return out


@pytest.mark.parametrize("row", _rows("tc"))
def test_tc_printed(row):
    q, val = row
    # printed to seven decimals, truncated ("...")
    assert math.floor(tc(q) * 1e7) / 1e7 == pytest.approx(val, abs=1e-12)


def test_tc_range_q9():
    (q, lo, hi), = _rows("tcrange")
    assert lo < tc(q) and abs(tc(q) - hi) < 1e-6
    assert beta_at(9, 1.0) == pytest.approx(math.log(4.0), rel=0, abs=1e-15)


@pytest.mark.parametrize("row", _rows("exact_e"))
def test_exact_transition_energies(row):
    q, minus_eo, minus_ed = row
    e_o, e_d = exact_energies(q)
    # printed values are truncated to six decimals
    assert math.floor(-e_o * 1e6) / 1e6 == pytest.approx(minus_eo, abs=1e-9)
    assert math.floor(-e_d * 1e6) / 1e6 == pytest.approx(minus_ed, abs=1e-9)


def test_latent_heat_limits():
    assert latent_heat(4) == 0.0
    # q -> infinity: e_o -> -2, e_d -> 0
    e_o, e_d = exact_energies(10**8)
    assert abs(e_o + 2.0) < 1e-3 and abs(e_d) < 1e-3


@pytest.mark.parametrize("row", _rows("exact_dm"))
def test_exact_dm_column_is_the_truncated_series(row):
    """The "exact" Delta m column equals the printed series (Eq. 8) with
    five subtracted terms, and neither four nor six terms give it."""
    q, val = row
    assert round(magnetization_jump_series(q, 5), 6) == pytest.approx(val, abs=1e-12)
    if q < 50:
        assert round(magnetization_jump_series(q, 4), 6) != val
        assert round(magnetization_jump_series(q, 6), 6) != val
