"""The oracle's band pass (one colour pass over a band of rows with the rows
just above and below supplied), which the row-strip decomposition of one
lattice (Sec. 7, multi-GPU extension) is checked against.

Pinned to the whole-lattice oracle sweep: for any split of the rows into
bands, white passes on every band (after the black halo rows are copied in)
followed by black passes (after the white halo rows are copied in) give the
same spins as oracle_sweep, and the bands' partial records summed give the
same record {B, hist} after every sweep.  A wrong halo row breaks it.
"""
import numpy as np
import pytest

import oracle


def _bands_sweep(spins, cuts, q, seed, t, beta, update, halo_shift=0):
    """One sweep of the L x L lattice `spins` done band by band; returns the
    summed record.  cuts: band start rows (first 0).  halo_shift != 0 plants
    a wrong halo (the row two away instead of the adjacent one)."""
    L = spins.shape[0]
    bounds = list(cuts) + [L]
    rec = np.zeros(1 + q, dtype=np.uint64)
    for c in (0, 1):
        new = spins.copy()
        for r0, r1 in zip(bounds[:-1], bounds[1:]):
            n = r1 - r0
            rows = np.empty((n + 2, L), np.uint8)
            rows[1:n + 1] = spins[r0:r1]
            rows[0] = spins[(r0 - 1 - halo_shift) % L]
            rows[n + 1] = spins[(r1 + halo_shift) % L]
            oracle.band_pass(rows, L, q, r0, seed, t, c, beta, rec, update)
            new[r0:r1] = rows[1:n + 1]
        spins[:] = new
    return rec


@pytest.mark.parametrize("L,q,cuts,update", [
    (8, 2, [0], oracle.METROPOLIS),
    (8, 9, [0, 4], oracle.METROPOLIS),
    (12, 9, [0, 1, 5, 6, 10], oracle.METROPOLIS),
    (16, 24, [0, 2, 4, 10], oracle.METROPOLIS),
    (32, 9, [0, 8, 16, 24], oracle.METROPOLIS),
    (16, 9, [0, 6, 7], oracle.HEATBATH),
    (32, 96, [0, 16], oracle.HEATBATH),
])
def test_bands_equal_whole_lattice_sweep(L, q, cuts, update):
    seed, beta = 5, 0.9 * np.log1p(np.sqrt(q))
    whole = oracle.Lattice(L, q, 1, seed)
    spins = whole.spins()
    for t in range(6):
        rec = _bands_sweep(spins, cuts, q, seed, t, beta, update)
        want = whole.sweep(beta, 1, update=update)[0]
        assert np.array_equal(rec, want), t
        assert np.array_equal(spins, whole.spins()), t


def test_wrong_halo_row_is_caught():
    L, q, seed, beta = 16, 9, 3, 1.0
    whole = oracle.Lattice(L, q, 1, seed)
    spins = whole.spins()
    rec = _bands_sweep(spins, [0, 8], q, seed, 0, beta, oracle.METROPOLIS,
                       halo_shift=1)
    want = whole.sweep(beta, 1)[0]
    assert not (np.array_equal(rec, want)
                and np.array_equal(spins, whole.spins()))


def test_band_pass_rejects_bad_arguments():
    rows = np.zeros((4, 8), np.uint8)
    part = np.zeros(10, np.uint64)
    with pytest.raises(ValueError):
        oracle.band_pass(rows, 8, 9, 7, 1, 0, 0, 1.0, part)   # r0 + n > L
    with pytest.raises(ValueError):
        oracle.band_pass(rows, 8, 9, 0, 1, 0, 2, 1.0, part)   # colour 2
