"""The fused sweep schedule (both colour passes in one kernel, needs a GPU):
records and spins bit for bit equal to the oracle's for every spin-width
class, both acceptance rules, tile counts of one and several CTAs per row,
and equal to the two-pass schedule at a large size; switching schedules,
reading and replacing the state between fused sweeps (the planes move between
two buffers), and the cases the schedule refuses."""
import numpy as np
import pytest

import oracle
from paper_1101_0876_gb300 import potts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1101_0876_gb300 import build
    build.build()


def _fused(L, q, start, seed):
    g = potts.Lattice(L, q, start, seed, layout=potts.LAYOUT_U8)
    g.set_schedule(potts.SCHEDULE_FUSED)
    return g


@pytest.mark.parametrize("L,q,start,beta,sweeps", [
    (1024, 2, 1, 0.44, 3),      # one CTA column, 4-bit class
    (1024, 9, 0, 1.4, 2),       # ordered start
    (1024, 16, 1, 0.9, 2),      # largest q of the pair histogram
    (2048, 17, 1, 1.0, 2),      # 5-bit class, two CTA columns
    (1024, 31, 1, 0.0, 2),      # beta = 0: every proposal accepted
    (1024, 64, 1, 1.3, 2),      # byte class
    (1024, 200, 0, 2.0, 2),
    (1024, 256, 1, 0.7, 2),
    (1024, 9, 1, 40.0, 2),      # thr[d] = 0: the strict acceptance rule
    (3072, 5, 1, 1.1, 2),       # three CTA columns, 96 CTA rows
])
def test_fused_matches_oracle(L, q, start, beta, sweeps):
    g = _fused(L, q, start, 11 + q)
    o = oracle.Lattice(L, q, start, 11 + q)
    assert np.array_equal(g.sweep(beta, sweeps), o.sweep(beta, sweeps))
    assert np.array_equal(g.spins(), o.spins())


def test_fused_equals_two_pass_at_l16384():
    L, q, beta = 16384, 9, 1.0 / 0.7213
    f = _fused(L, q, 1, 5)
    t = potts.Lattice(L, q, 1, 5, layout=potts.LAYOUT_U8)
    assert np.array_equal(f.sweep(beta, 7), t.sweep(beta, 7))
    assert np.array_equal(f.spins(), t.spins())


def test_switching_schedules_and_state_between_sweeps():
    L, q, beta = 1024, 9, 1.35
    g = _fused(L, q, 1, 21)
    o = oracle.Lattice(L, q, 1, 21)
    # odd number of fused sweeps: the planes end in the second buffer
    assert np.array_equal(g.sweep(beta, 3), o.sweep(beta, 3))
    g.set_schedule(potts.SCHEDULE_TWO_PASS)
    assert np.array_equal(g.sweep(beta, 2), o.sweep(beta, 2))
    g.set_schedule(potts.SCHEDULE_FUSED)
    assert np.array_equal(g.sweep(beta, 1), o.sweep(beta, 1))
    assert np.array_equal(g.spins(), o.spins())
    # replace the state, continue fused from it
    rng = np.random.default_rng(4)
    s = rng.integers(0, q, size=(L, L), dtype=np.uint8)
    g.set_state(s, 100)
    o.set_state(s, 100)
    assert np.array_equal(g.sweep(beta, 2), o.sweep(beta, 2))
    assert np.array_equal(g.spins(), o.spins())
    obs = g.observables()
    assert obs["sweep"] == 102


def test_heatbath_keeps_two_passes_under_fused_schedule():
    L, q, beta = 1024, 9, 1.2
    g = _fused(L, q, 1, 8)
    g.set_update(potts.UPDATE_HEATBATH)
    o = oracle.Lattice(L, q, 1, 8)
    assert np.array_equal(g.sweep(beta, 2),
                          o.sweep(beta, 2, update=oracle.HEATBATH))


@pytest.mark.parametrize("L,layout", [(96, potts.LAYOUT_U8),
                                      (1536, potts.LAYOUT_U8),
                                      (1024, potts.LAYOUT_U4)])
def test_fused_refuses_unsupported_lattices(L, layout):
    g = potts.Lattice(L, 9, 1, 1, layout=layout)
    with pytest.raises(potts.PottsError):
        g.set_schedule(potts.SCHEDULE_FUSED)
    with pytest.raises(potts.PottsError):
        g.set_schedule(7)
    g.set_schedule(potts.SCHEDULE_TWO_PASS)
