"""Pins of the CPU oracle against things other than itself (CPU only).

- Philox4x32-10 against PyTorch's independent header-only CPU engine;
- the Boltzmann threshold table against the closed form at high precision;
- invariants the paper and the mathematics fix (ground state e = -2,
  Sum hist = N, 0 <= B <= 2N, incremental counts equal a recount, beta = 0
  accepts every proposal and leaves i.i.d. uniform spins, beta -> infinity
  freezes the ground state);
- serial raster order equals reverse order for even L (the property the
  parallel checkerboard relies on);
- the one-site sampled update equals the full sweep.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle


# ---------------------------------------------------------------- Philox

def test_philox_matches_torch_engine(torch_philox):
    rng = np.random.default_rng(12345)
    n = 4000
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # edge counters / keys
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    ref = torch_philox(ctr, key)
    mine = np.stack([oracle.philox4x32_10(c, k) for c, k in zip(ctr, key)])
    assert np.array_equal(ref, mine)


def test_site_word_counter_layout(torch_philox):
    """site word = Philox(ctr=(k>>2, sweep_lo, domain, sweep_hi),
    key=(seed_lo, seed_hi))[k & 3], cross-checked through torch's engine."""
    cases = [(1, 0, 0, 0), (1, 7, 1, 5), (2**40 + 3, 2**33 + 9, 2, 123456),
             (0xFFFFFFFFFFFFFFFF, 1, 3, 2**31 - 1)]
    for seed, sweep, dom, k in cases:
        ctr = np.array([[k >> 2, sweep & 0xFFFFFFFF, dom, sweep >> 32]],
                       dtype=np.uint64).astype(np.uint32)
        key = np.array([[seed & 0xFFFFFFFF, seed >> 32]],
                       dtype=np.uint64).astype(np.uint32)
        ref = torch_philox(ctr, key)[0, k & 3]
        assert oracle.site_word(seed, sweep, dom, k) == int(ref)


def test_philox_uniform_and_avalanche():
    rng = np.random.default_rng(7)
    words = []
    for g in range(4096):
        words.extend(oracle.philox4x32_10([g, 0, 0, 0], [1, 0]))
    w = np.array(words, dtype=np.uint64)
    hist = np.bincount((w >> 28).astype(np.int64), minlength=16)
    chi2 = stats.chisquare(hist)
    assert chi2.pvalue > 1e-4
    flips = []
    for _ in range(200):
        c = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        k = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        b = int(rng.integers(0, 128))
        c2 = c.copy()
        c2[b // 32] ^= np.uint32(1 << (b % 32))
        x = oracle.philox4x32_10(c, k) ^ oracle.philox4x32_10(c2, k)
        flips.append(sum(bin(int(v)).count("1") for v in x))
    assert abs(np.mean(flips) - 64) < 2.0


# ------------------------------------------------------------ thresholds

def _exact_floor(beta: float, d: int) -> int:
    import mpmath
    mpmath.mp.prec = 200
    v = mpmath.ldexp(mpmath.exp(-mpmath.mpf(beta) * d), 32)
    return int(mpmath.floor(v)), v


def test_thresholds_closed_form():
    rng = np.random.default_rng(3)
    betas = list(rng.uniform(0.01, 6.0, 200)) + [math.log(4.0), 0.5, 2.0]
    for beta in betas:
        thr = oracle.thresholds(beta)
        assert int(thr[0]) == 2**32
        for d in range(1, 5):
            fl, v = _exact_floor(beta, d)
            # glibc exp is within one ulp: the floor can only differ when the
            # exact value sits within ~2^-20 of an integer.
            if abs(v - round(v)) > 1e-4:
                assert int(thr[d]) == fl, (beta, d)
            else:
                assert abs(int(thr[d]) - fl) <= 1
            assert 0 <= int(thr[d]) < 2**32
        assert all(int(thr[d]) >= int(thr[d + 1]) for d in range(1, 4))


def test_thresholds_special_values():
    assert [int(x) for x in oracle.thresholds(0.0)] == [2**32] * 5
    big = oracle.thresholds(40.0)
    assert [int(x) for x in big[1:]] == [0, 0, 0, 0]
    for bad in (-1e-9, float("nan"), float("inf")):
        with pytest.raises(ValueError):
            oracle.thresholds(bad)


# ------------------------------------------------------------ invariants

@pytest.mark.parametrize("L,q", [(8, 9), (16, 2), (12, 256), (10, 15)])
def test_ordered_start_ground_state(L, q):
    lat = oracle.Lattice(L, q, 0, 1)
    B, hist = lat.counts()
    assert B == 2 * L * L
    assert int(hist[0]) == L * L and int(hist[1:].sum()) == 0
    e, m = oracle.observables(np.array([[B] + list(hist)]), L, q)
    assert e[0] == -2.0 and m[0] == 1.0


def test_frozen_at_large_beta():
    """thr = 0 for every dE >= 1: from the ordered state every proposal that
    changes a spin costs dE = +4 and is refused."""
    lat = oracle.Lattice(16, 9, 0, 5)
    rec = lat.sweep(40.0, 20, check=True)
    assert np.all(rec[:, 0] == 2 * 256)
    assert np.all(rec[:, 1] == 256)
    assert np.array_equal(lat.spins(), np.zeros((16, 16), np.uint8))


@pytest.mark.parametrize("L,q,start,beta", [
    (8, 9, 0, math.log(4.0)), (16, 9, 1, math.log(4.0)), (10, 2, 1, 0.9),
    (12, 256, 1, 3.0), (14, 5, 0, 0.3), (9, 6, 1, 1.1), (3, 4, 1, 0.8),
])
def test_incremental_equals_recount(L, q, start, beta):
    lat = oracle.Lattice(L, q, start, 17)
    rec = lat.sweep(beta, 200, check=True)     # raises on any mismatch
    N = L * L
    assert np.all(rec[:, 1:].sum(axis=1) == N)
    assert np.all(rec[:, 0] <= 2 * N)
    B, hist = oracle.recount(lat.spins(), q)
    assert B == int(rec[-1, 0]) and np.array_equal(hist, rec[-1, 1:])


def test_recount_by_hand():
    s = np.array([[0, 0, 1, 1],
                  [0, 2, 2, 1],
                  [3, 3, 2, 0],
                  [0, 1, 1, 0]], dtype=np.uint8)
    # Satisfied right bonds (j -> j+1 mod 4), counted by hand per row:
    #   row 0: (0,1) (2,3) = 2;  row 1: (1,2) = 1;  row 2: (0,1) = 1;
    #   row 3: (1,2) and the wrap (3,0) = 2            -> 6
    # Satisfied down bonds (i -> i+1 mod 4), per column:
    #   col 0: rows 0-1 and the wrap 3-0 = 2;  col 1: none;
    #   col 2: rows 1-2 and the wrap 3-0 = 2;  col 3: rows 0-1, 2-3 = 2  -> 6
    B, hist = oracle.recount(s, 4)
    assert B == 12
    assert list(hist) == [6, 5, 3, 2]


def test_beta_zero_accepts_everything():
    """At beta = 0 every proposal is accepted, so after one sweep each site
    holds its own proposal floor(u q / 2^32): i.i.d. uniform over q states."""
    q, L = 9, 64
    counts = np.zeros(q, dtype=np.int64)
    for seed in range(8):
        lat = oracle.Lattice(L, q, 0, seed)
        lat.sweep(0.0, 1, records=False)
        counts += np.bincount(lat.spins().ravel(), minlength=q)
    assert stats.chisquare(counts).pvalue > 1e-4
    # neighbouring sites are independent: joint (left, right) pairs uniform
    lat = oracle.Lattice(L, q, 0, 99)
    lat.sweep(0.0, 1, records=False)
    s = lat.spins()
    pairs = (s[:, :-1].astype(np.int64) * q + s[:, 1:]).ravel()
    assert stats.chisquare(np.bincount(pairs, minlength=q * q)).pvalue > 1e-4


def test_random_start_uniform():
    lat = oracle.Lattice(128, 15, 1, 11)
    s = lat.spins()
    assert stats.chisquare(np.bincount(s.ravel(), minlength=15)).pvalue > 1e-4
    # the two colour classes are drawn from different words
    white = s[(np.add.outer(np.arange(128), np.arange(128)) % 2) == 0]
    black = s[(np.add.outer(np.arange(128), np.arange(128)) % 2) == 1]
    assert np.mean(white == black) < 0.2


@pytest.mark.parametrize("L,q,start", [(8, 9, 1), (16, 3, 0), (12, 200, 1)])
def test_reverse_order_identical_for_even_L(L, q, start):
    a = oracle.Lattice(L, q, start, 4)
    b = oracle.Lattice(L, q, start, 4)
    ra = a.sweep(1.2, 50, order=0)
    rb = b.sweep(1.2, 50, order=1)
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.spins(), b.spins())


def test_odd_L_order_matters():
    """On odd L same-coloured sites touch through the boundary, so the order
    inside a colour is part of the definition (a sanity check that the
    reverse-order test above has teeth)."""
    a = oracle.Lattice(5, 3, 1, 4)
    b = oracle.Lattice(5, 3, 1, 4)
    a.sweep(0.3, 30, order=0, records=False)
    b.sweep(0.3, 30, order=1, records=False)
    assert not np.array_equal(a.spins(), b.spins())


@pytest.mark.parametrize("L,q,start,beta", [(8, 9, 1, 1.386), (16, 4, 0, 0.7),
                                            (10, 256, 1, 2.0)])
def test_sampled_sites_equal_full_sweep(L, q, start, beta):
    lat = oracle.Lattice(L, q, start, 21)
    lat.sweep(beta, 3, records=False)
    pre = lat.spins()
    t = lat.sweep_index
    lat.sweep(beta, 1, records=False)
    post = lat.spins()
    idx = np.arange(L * L, dtype=np.int64)
    got = oracle.sweep_sites(pre, q, 21, t, beta, idx)
    assert np.array_equal(got.reshape(L, L), post)


def test_set_state_resume_is_exact():
    a = oracle.Lattice(16, 9, 1, 8)
    a.sweep(1.3, 10, records=False)
    snap, t = a.spins(), a.sweep_index
    ra = a.sweep(1.3, 5)
    b = oracle.Lattice(16, 9, 0, 8)
    b.set_state(snap, t)
    rb = b.sweep(1.3, 5)
    assert np.array_equal(ra, rb)
