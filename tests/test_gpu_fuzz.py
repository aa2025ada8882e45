"""Seeded random parity cases (needs a GPU): lattice sizes across the
geometry rules (one or several CTAs per row, ragged widths, short and long
walks, one or several tiles per CTA), every spin-width class, both layouts,
both update rules, the fused sweep schedule and the whole range of beta,
each checked bit for bit against the oracle."""
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


def _cases(n=24, seed=2026):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        L = 32 * int(rng.integers(1, 71))
        q = int(rng.choice([2, 3, 5, 9, 12, 16, 17, 24, 31, 40, 64, 100, 129,
                            200, 256]))
        beta = float(rng.choice([0.0, rng.uniform(0.2, 3.0),
                                 rng.uniform(0.2, 3.0), 40.0]))
        layout = potts.LAYOUT_U4 if (q <= 16 and rng.random() < 0.4) \
            else potts.LAYOUT_U8
        update = potts.UPDATE_HEATBATH if (beta < 5 and rng.random() < 0.35) \
            else potts.UPDATE_METROPOLIS
        out.append((L, q, int(rng.integers(0, 2)), beta, int(rng.integers(2, 7)),
                    layout, update, 7000 + i))
    return out


@pytest.mark.parametrize("L,q,start,beta,sweeps,layout,update,seed", _cases())
def test_random_case(L, q, start, beta, sweeps, layout, update, seed):
    g = potts.Lattice(L, q, start, seed, layout=layout)
    g.set_update(update)
    o = oracle.Lattice(L, q, start, seed)
    assert np.array_equal(g.sweep(beta, sweeps),
                          o.sweep(beta, sweeps, update=update))
    assert np.array_equal(g.spins(), o.spins())


def _fused_cases(n=6, seed=2027):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        L = 1024 * int(rng.integers(1, 3))
        q = int(rng.choice([2, 3, 9, 16, 17, 31, 40, 100, 256]))
        beta = float(rng.choice([0.0, rng.uniform(0.2, 3.0), 40.0]))
        out.append((L, q, int(rng.integers(0, 2)), beta, int(rng.integers(1, 4)),
                    9000 + i))
    return out


@pytest.mark.parametrize("L,q,start,beta,sweeps,seed", _fused_cases())
def test_random_fused_case(L, q, start, beta, sweeps, seed):
    g = potts.Lattice(L, q, start, seed, layout=potts.LAYOUT_U8)
    g.set_schedule(potts.SCHEDULE_FUSED)
    o = oracle.Lattice(L, q, start, seed)
    assert np.array_equal(g.sweep(beta, sweeps), o.sweep(beta, sweeps))
    assert np.array_equal(g.spins(), o.spins())
