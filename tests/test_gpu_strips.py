"""Row-strip decomposition of one lattice on the GPU (the multi-GPU extension
of Sec. 7), checked bit for bit against the CPU oracle.

potts_create_sharded splits a lattice into 1, 2 or 4 strips held by this
process (all on the one visible GPU here; the halo rows move by
device-to-device copies between the strips' streams): spins and every
record must equal the oracle's whole-lattice sweep, for both update rules
and both layouts, and at the paper's scale equal the single-lattice path.
The strip handles (potts_strip_*), which a one-strip-per-process run drives
with its own halo exchange, are driven here by the same exchange logic in
one process.
"""
import numpy as np
import pytest

import oracle
from paper_1101_0876_gb300 import potts, strips, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1101_0876_gb300 import build
    build.build()


@pytest.mark.parametrize("L,q,nstrips,layout,update", [
    (64, 9, 1, potts.LAYOUT_U8, potts.UPDATE_METROPOLIS),
    (64, 9, 2, potts.LAYOUT_U8, potts.UPDATE_METROPOLIS),
    (256, 9, 4, potts.LAYOUT_U8, potts.UPDATE_METROPOLIS),
    (544, 24, 3, potts.LAYOUT_U8, potts.UPDATE_METROPOLIS),
    (256, 15, 4, potts.LAYOUT_U4, potts.UPDATE_METROPOLIS),
    (128, 96, 2, potts.LAYOUT_U8, potts.UPDATE_METROPOLIS),
    (128, 9, 4, potts.LAYOUT_U8, potts.UPDATE_HEATBATH),
    (96, 9, 48, potts.LAYOUT_U8, potts.UPDATE_METROPOLIS),   # 2-row strips
])
def test_sharded_equals_oracle(L, q, nstrips, layout, update):
    seed = 13
    beta = workloads.beta_at(q, 1.0)
    g = potts.Lattice(L, q, potts.START_RANDOM, seed, layout=layout,
                      nstrips=nstrips)
    o = oracle.Lattice(L, q, 1, seed)
    assert np.array_equal(g.spins(), o.spins())
    if update == potts.UPDATE_HEATBATH:
        g.set_update(update)
    upd = oracle.HEATBATH if update == potts.UPDATE_HEATBATH else 0
    for n in (1, 3, 4):
        assert np.array_equal(g.sweep(beta, n), o.sweep(beta, n, update=upd))
        assert np.array_equal(g.spins(), o.spins())
    obs = g.observables()
    assert obs["sweep"] == 8
    B, hist = o.counts()
    assert obs["bonds"] == B


def test_sharded_ordered_start_beta_zero_and_state():
    L, q = 128, 9
    g = potts.Lattice(L, q, potts.START_ORDERED, 2, nstrips=2)
    o = oracle.Lattice(L, q, 0, 2)
    assert g.observables()["bonds"] == 2 * L * L
    assert np.array_equal(g.sweep(0.0, 2), o.sweep(0.0, 2))
    s = workloads.random_spins(L, q, 9)
    g.set_state(s, 40)
    o.set_state(s, 40)
    assert np.array_equal(g.spins(), s)
    beta = workloads.beta_at(q, 0.99)
    assert np.array_equal(g.sweep(beta, 3), o.sweep(beta, 3))
    bad = s.copy()
    bad[L - 1, 5] = q
    with pytest.raises(potts.PottsError):
        g.set_state(bad, 0)
    assert np.array_equal(g.spins(), o.spins())   # nothing changed


def test_sharded_rejects():
    with pytest.raises(potts.PottsError):
        potts.Lattice(64, 9, 1, 1, nstrips=33)     # more strips than row pairs
    with pytest.raises(potts.PottsError):
        potts.Lattice(64, 9, 1, 1, nstrips=2, devices=[0, 99])
    g = potts.Lattice(64, 9, 1, 1, nstrips=2)
    with pytest.raises(potts.PottsError):
        g.set_schedule(potts.SCHEDULE_FUSED)
    with pytest.raises(potts.PottsError):
        g.set_stream(None)


def test_sharded_paper_scale_equals_single_lattice():
    """L = 32768, q = 9 at T_c: four strips give the single-lattice path's
    records bit for bit (that path is checked against the oracle by sampled
    sites at this size)."""
    L, q, seed = 32768, 9, 11
    beta = workloads.beta_at(q, 1.0)
    one = potts.Lattice(L, q, potts.START_RANDOM, seed)
    r1 = one.sweep(beta, 3)
    one.close()
    four = potts.Lattice(L, q, potts.START_RANDOM, seed, nstrips=4)
    r4 = four.sweep(beta, 3)
    assert np.array_equal(r1, r4)


def _local_exchange(bands, plane):
    """Halo rows of `plane` for strips held in one process."""
    S = len(bands)
    for s, b in enumerate(bands):
        prev, nxt = bands[(s - 1) % S], bands[(s + 1) % S]
        _, _, above, below = b.rows(plane)
        above.copy_(prev.rows(plane)[1])
        below.copy_(nxt.rows(plane)[0])


@pytest.mark.parametrize("L,q,cuts", [(64, 9, [0, 32]),
                                      (256, 24, [0, 64, 100, 200])])
def test_strip_handles_equal_oracle(L, q, cuts):
    """Strip handles (the one-strip-per-process interface) with the halo
    rows moved by the caller: bit-exact records and spins."""
    import torch
    seed, beta = 5, workloads.beta_at(q, 1.0)
    bounds = cuts + [L]
    bands = [strips.StripBand(L, q, potts.START_RANDOM, seed, r0, r1 - r0)
             for r0, r1 in zip(bounds[:-1], bounds[1:])]
    o = oracle.Lattice(L, q, 1, seed)
    for t in range(4):
        rec = bands[0].new_record()
        for c in (0, 1):
            _local_exchange(bands, c ^ 1)
            for b in bands:
                b.pass_(beta, c, rec)
        torch.cuda.synchronize()
        want = o.sweep(beta, 1)[0]
        assert np.array_equal(rec.cpu().numpy().astype(np.uint64), want), t
    spins = np.concatenate([b.h.spins() for b in bands])
    assert np.array_equal(spins, o.spins())


def test_strip_sweeper_single_rank():
    """StripSweeper with one rank: the whole lattice as one periodic strip,
    halo rows copied from its own edge rows."""
    L, q, seed = 128, 15, 3
    beta = workloads.beta_at(q, 1.0)
    band = strips.StripBand(L, q, potts.START_RANDOM, seed, 0, L)
    sw = strips.StripSweeper(band, 0, 1)
    o = oracle.Lattice(L, q, 1, seed)
    for t in range(3):
        rec = sw.sweep(beta)
        assert np.array_equal(rec.cpu().numpy().astype(np.uint64),
                              o.sweep(beta, 1)[0]), t
    assert np.array_equal(band.h.spins(), o.spins())


def test_strip_create_rejects():
    with pytest.raises(potts.PottsError):
        potts.Strip(64, 9, 1, 1, 1, 10)     # odd first row
    with pytest.raises(potts.PottsError):
        potts.Strip(64, 9, 1, 1, 60, 6)     # beyond the lattice
    s = potts.Strip(64, 9, 1, 1, 0, 8)
    assert potts.lib().potts_sweep(s._h, 1.0, 1, None) == potts.POTTS_EINVAL
