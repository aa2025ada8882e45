"""Host analysis of the integer series (CPU): reweighting, cumulant,
susceptibility and specific heat against exact enumeration on tiny lattices
(the series come from the oracle, the exact values from tests/brute_force.c).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1101_0876_gb300.analysis import (batch_means, cumulant_VL,
                                            energy_magnetization, reweight,
                                            specific_heat, susceptibility)


def _series(L, q, beta, n, seed):
    lat = oracle.Lattice(L, q, 1, seed)
    lat.sweep(beta, 2000, records=False)
    return lat.sweep(beta, n)


@pytest.mark.parametrize("beta0,beta1", [(0.9, 1.0), (1.0, 0.92)])
def test_reweighting_matches_enumeration(brute_force, beta0, beta1):
    L, q = 3, 3
    rec = _series(L, q, beta0, 300_000, 5)
    exact = brute_force(L, q, beta1)
    nb = 100
    blocks = np.array_split(rec, nb)
    est = np.array([reweight(b, L, q, beta0, beta1) for b in blocks])
    for k in range(4):
        mean = est[:, k].mean()
        err = est[:, k].std(ddof=1) / math.sqrt(nb)
        assert abs(mean - exact[k]) < 4 * err + 1e-12, (k, mean, exact[k], err)
    # no reweighting: plain averages
    e, m = energy_magnetization(rec, L, q)
    assert reweight(rec, L, q, beta0, beta0)[0] == pytest.approx(e.mean())


def test_cumulant_susceptibility_specific_heat(brute_force):
    L, q, beta = 3, 4, 0.9
    rec = _series(L, q, beta, 300_000, 9)
    ex = brute_force(L, q, beta)   # <e>, <e^2>, <m>, <m^2>, <e^4>
    N = L * L
    VL_exact = 1 - ex[4] / (3 * ex[1] ** 2)        # H = N e: N cancels
    chi_exact = N * beta * (ex[3] - ex[2] ** 2)     # (N/T)(<m^2> - <m>^2)
    C_exact = beta ** 2 * N * (ex[1] - ex[0] ** 2)
    blocks = np.array_split(rec, 50)
    for fn, exact in [(lambda b: cumulant_VL(b), VL_exact),
                      (lambda b: susceptibility(b, L, q, 1 / beta), chi_exact),
                      (lambda b: specific_heat(b, L, q, beta), C_exact)]:
        vals = np.array([fn(b) for b in blocks])
        mean, err = vals.mean(), vals.std(ddof=1) / math.sqrt(len(vals))
        assert abs(mean - exact) < 4 * err + 1e-3 * abs(exact), (mean, exact)


def test_batch_means_of_iid():
    x = np.random.default_rng(0).normal(1.0, 2.0, 100_000)
    m, e = batch_means(x, 100)
    assert abs(m - 1.0) < 4 * e and 0.5 * 2 / math.sqrt(1e5) < e < 2 * 2 / math.sqrt(1e5)
