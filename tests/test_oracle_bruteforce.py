"""The oracle's long-run averages agree with exact Boltzmann enumeration.

On 3x3 periodic lattices (q = 2..5, q^9 states) and 4x4 (q = 2, 3) the
exact <e>, <e^2>, <m>, <m^2> come from tests/brute_force.c, which shares no
code with the oracle.  A dropped term, a wrong sign of dE, a wrong neighbour
or an acceptance rule that is not min(1, exp(-beta dE)) moves at least one
of these averages by many standard errors.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1101_0876_gb300.analysis import batch_means, energy_magnetization

CASES = [
    (3, 2, 0.5), (3, 2, math.log1p(math.sqrt(2))), (3, 3, 1.0),
    (3, 4, math.log1p(2.0)), (3, 5, 0.7), (3, 5, 1.6),
    (4, 2, 0.6), (4, 2, 1.2), (4, 3, math.log1p(math.sqrt(3))),
]


@pytest.mark.parametrize("L,q,beta", CASES)
def test_long_run_averages_match_enumeration(brute_force, L, q, beta):
    exact = brute_force(L, q, beta)
    lat = oracle.Lattice(L, q, 1, 1000 + 17 * q + L)
    lat.sweep(beta, 2000, records=False)            # equilibrate
    n = 300_000 if L == 3 else 200_000
    rec = lat.sweep(beta, n)
    e, m = energy_magnetization(rec, L, q)
    for k, x in enumerate([e, e * e, m, m * m]):
        mean, err = batch_means(x, 200)
        assert abs(mean - exact[k]) < 4.0 * err + 1e-12, (k, mean, exact[k], err)


def test_enumeration_sanity(brute_force):
    # beta = 0: every state equally likely; <e> = -(2N bonds)(1/q)/N = -2/q
    for q in (2, 3, 5):
        ex = brute_force(3, q, 0.0)
        assert abs(ex[0] + 2.0 / q) < 1e-12
    # large beta: ground state dominates, e -> -2, m -> 1
    ex = brute_force(3, 3, 30.0)
    assert abs(ex[0] + 2.0) < 1e-9 and abs(ex[2] - 1.0) < 1e-9
