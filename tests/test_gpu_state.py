"""Moving a state between the caller's row-major host bytes and the device
planes (needs a GPU): set_state / get_spins round trips for both layouts and
sizes from one to many CTAs, sweeps continuing from an uploaded state equal
to the oracle's, and an out-of-range spin refused before anything changes
(the first bad site is the one reported)."""
import numpy as np
import pytest

import oracle
from paper_1101_0876_gb300 import potts, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1101_0876_gb300 import build
    build.build()


@pytest.mark.parametrize("L,q,layout", [
    (32, 2, potts.LAYOUT_U8), (96, 9, potts.LAYOUT_U8),
    (1024, 256, potts.LAYOUT_U8), (8192, 9, potts.LAYOUT_U8),
    (64, 16, potts.LAYOUT_U4), (96, 3, potts.LAYOUT_U4),
    (8192, 12, potts.LAYOUT_U4)])
def test_round_trip(L, q, layout):
    spins = workloads.random_spins(L, q, L + q)
    g = potts.Lattice(L, q, 0, 1, layout=layout)
    g.set_state(spins, 77)
    assert np.array_equal(g.spins(), spins)
    B, hist = oracle.recount(spins, q)
    obs = g.observables()
    assert obs["bonds"] == B and obs["sweep"] == 77


@pytest.mark.parametrize("layout", [potts.LAYOUT_U8, potts.LAYOUT_U4])
def test_sweeps_continue_from_uploaded_state(layout):
    L, q, beta = 160, 7, 1.2
    spins = workloads.random_spins(L, q, 5)
    g = potts.Lattice(L, q, 1, 3, layout=layout)
    g.sweep(beta, 2)
    g.set_state(spins, 40)
    o = oracle.Lattice(L, q, 1, 3)
    o.set_state(spins, 40)
    assert np.array_equal(g.sweep(beta, 3), o.sweep(beta, 3))
    assert np.array_equal(g.spins(), o.spins())


def test_out_of_range_spin_changes_nothing():
    L, q = 128, 5
    g = potts.Lattice(L, q, 1, 8)
    g.sweep(1.0, 2)
    before = g.spins()
    obs0 = g.observables()
    bad = workloads.random_spins(L, q, 2)
    bad[100, 7] = 200
    bad[3, 4] = 5          # first bad site in row-major order
    with pytest.raises(potts.PottsError) as ei:
        g.set_state(bad, 999)
    assert ei.value.code == potts.POTTS_EINVAL
    assert f"at {3 * L + 4} " in potts.last_error()
    assert np.array_equal(g.spins(), before)
    obs1 = g.observables()
    assert obs1["sweep"] == obs0["sweep"] and obs1["bonds"] == obs0["bonds"]
    o = oracle.Lattice(L, q, 1, 8)
    o.sweep(1.0, 2)
    assert np.array_equal(g.sweep(1.0, 2), o.sweep(1.0, 2))


def test_batch_member_spins():
    Ls, qs = [64, 96, 256], [3, 9, 24]
    b = potts.Batch(Ls, qs, [1, 0, 1], [4, 5, 6])
    b.sweep([0.9, 1.1, 1.3], 3)
    for i, (L, q, s) in enumerate(zip(Ls, qs, [1, 0, 1])):
        o = oracle.Lattice(L, q, s, 4 + i)
        o.sweep([0.9, 1.1, 1.3][i], 3)
        assert np.array_equal(b.spins(i), o.spins())
