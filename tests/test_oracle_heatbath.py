"""Pins of the oracle's heat-bath update against what fixes it independently
of the oracle's code:

- the integer weights against exp evaluated with mpmath, and the choice of
  the scale 2^m against the 32-bit bound on every normaliser;
- the single-site rule's output distribution against the conditional
  Boltzmann distribution exp(beta n_x) / sum_y exp(beta n_y), for every
  neighbour configuration met on random lattices;
- long-run averages on 3x3 and 4x4 lattices against exact enumeration
  (tests/brute_force.c);
- beta = 0 gives i.i.d. uniform spins after one sweep; incremental counts
  equal a recount after every sweep.
"""
import math
from collections import defaultdict

import numpy as np
import pytest

import oracle
from paper_1101_0876_gb300.analysis import batch_means, energy_magnetization

HB = oracle.HEATBATH
SPLITS = [(4,), (3, 1), (2, 2), (2, 1, 1), (1, 1, 1, 1)]


def _zmax(w, q):
    return max(sum(w[c] for c in sp) + (q - len(sp)) * w[0]
               for sp in SPLITS if len(sp) <= q)


@pytest.mark.parametrize("q", [2, 3, 9, 15, 96, 256])
@pytest.mark.parametrize("beta", [0.0, 0.3, 1.0986122886681098, 2.0, 3.5])
def test_weights_against_mpmath(q, beta):
    try:
        W, m = oracle.heatbath_weights(beta, q)
    except ValueError:
        # only when even W[0] = 1 cannot hold exp(4 beta) in 32 bits
        assert math.exp(4 * beta) + q - 1 > 2**32 - 1
        return
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    assert int(W[0]) == 2**m
    exact = [mpmath.ldexp(mpmath.exp(mpmath.mpf(beta) * n), m) for n in range(5)]
    for n in range(5):
        frac = exact[n] - mpmath.floor(exact[n])
        if abs(frac - 0.5) > 1e-4:                 # not a rounding tie
            assert int(W[n]) == int(mpmath.floor(exact[n] + 0.5)), (n, W[n])
    assert _zmax([int(x) for x in W], q) <= 2**32 - 1
    if m < 31:                                     # m is the largest that fits
        up = [int(mpmath.floor(mpmath.ldexp(mpmath.exp(mpmath.mpf(beta) * n),
                                            m + 1) + 0.5)) for n in range(5)]
        assert up[4] >= 2**32 or _zmax(up, q) > 2**32 - 1


def test_weights_reject_large_beta():
    with pytest.raises(ValueError):
        oracle.heatbath_weights(6.0, 9)
    with pytest.raises(ValueError):
        oracle.heatbath_weights(-1.0, 9)


def _white_outcomes(L, q, beta, seed, nsweeps, rng):
    """Outcome counts of the white-site update grouped by the neighbour
    configuration: {sorted neighbour tuple: {state: count}}.  Neighbours
    take only states 0..2, so that each configuration recurs often and
    states >= 3 are held by no neighbour."""
    pre = rng.integers(0, min(q, 3), size=(L, L), dtype=np.uint8)
    ii, jj = np.nonzero((np.add.outer(np.arange(L), np.arange(L)) % 2) == 0)
    idx = (ii * L + jj).astype(np.int64)
    nb = np.stack([pre[(ii - 1) % L, jj], pre[(ii + 1) % L, jj],
                   pre[ii, (jj - 1) % L], pre[ii, (jj + 1) % L]], axis=1)
    keys = [tuple(sorted(r)) for r in nb]
    counts = defaultdict(lambda: np.zeros(q, dtype=np.int64))
    for t in range(nsweeps):
        out = oracle.sweep_sites(pre, q, seed, t, beta, idx, update=HB)
        for k, s in zip(keys, out):
            counts[k][s] += 1
    return counts


@pytest.mark.parametrize("q,beta", [(3, 0.8), (5, 1.3), (9, 1.0986122886681098)])
def test_rule_samples_conditional_boltzmann(q, beta):
    rng = np.random.default_rng(q)
    counts = _white_outcomes(32, q, beta, 5, 300, rng)
    checked = 0
    for key, c in counts.items():
        n = c.sum()
        if n < 3000:
            continue
        nx = np.array([key.count(x) for x in range(q)], dtype=np.float64)
        p = np.exp(beta * nx)
        p /= p.sum()
        chi2 = float(((c - n * p) ** 2 / (n * p)).sum())
        # q - 1 degrees of freedom; 1e-4 tail is below 3 (q - 1) + 25
        assert chi2 < 3 * (q - 1) + 25, (key, c, n * p)
        checked += 1
    assert checked >= 5


CASES = [(3, 2, 0.5), (3, 3, 1.0), (3, 4, math.log1p(2.0)), (3, 5, 1.6),
         (4, 2, 1.2), (4, 3, math.log1p(math.sqrt(3)))]


@pytest.mark.parametrize("L,q,beta", CASES)
def test_long_run_averages_match_enumeration(brute_force, L, q, beta):
    exact = brute_force(L, q, beta)
    lat = oracle.Lattice(L, q, 1, 2000 + 17 * q + L)
    lat.sweep(beta, 2000, records=False, update=HB)
    rec = lat.sweep(beta, 200_000, update=HB)
    e, m = energy_magnetization(rec, L, q)
    for k, x in enumerate([e, e * e, m, m * m]):
        mean, err = batch_means(x, 200)
        assert abs(mean - exact[k]) < 4.0 * err + 1e-12, (k, mean, exact[k], err)


def test_beta_zero_gives_uniform_spins():
    q, L = 7, 256
    lat = oracle.Lattice(L, q, 0, 9)
    lat.sweep(0.0, 1, update=HB)
    s = lat.spins().ravel()
    c = np.bincount(s, minlength=q)
    e = s.size / q
    assert ((c - e) ** 2 / e).sum() < 3 * (q - 1) + 25
    pair = s.reshape(L, L)
    pc = np.bincount((pair[:, :-1] * q + pair[:, 1:]).ravel(), minlength=q * q)
    pe = pc.sum() / q**2
    assert ((pc - pe) ** 2 / pe).sum() < 3 * (q * q - 1) + 60


@pytest.mark.parametrize("q", [2, 3, 9, 24, 200])
def test_incremental_counts_equal_recount(q):
    lat = oracle.Lattice(12, q, 1, q)
    lat.sweep(1.2, 30, check=True, update=HB)
    lat2 = oracle.Lattice(13, q, 0, q)
    lat2.sweep(0.4, 30, check=True, update=HB)
