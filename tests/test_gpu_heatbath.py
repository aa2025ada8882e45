"""Heat-bath colour passes against the CPU oracle's heat-bath rule, bit for
bit (needs a GPU): spins and per-sweep records for every q class, ragged
widths, both layouts and the range of beta; sampled parity at full size."""
import math

import numpy as np
import pytest

import oracle
from paper_1101_0876_gb300 import potts, workloads

pytestmark = pytest.mark.gpu
HB = potts.UPDATE_HEATBATH


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1101_0876_gb300 import build
    build.build()


def test_small_config_every_sweep():
    """L=64, q=9, ordered start, T = T_c, seed 1: records and spins after
    every sweep for 200 sweeps."""
    cfg = workloads.SMALL
    beta = workloads.beta_at(cfg.q, 1.0)
    g = potts.Lattice(cfg.L, cfg.q, cfg.start, cfg.seed)
    g.set_update(HB)
    o = oracle.Lattice(cfg.L, cfg.q, cfg.start, cfg.seed)
    for step in range(200):
        assert np.array_equal(g.sweep(beta, 1),
                              o.sweep(beta, 1, update=oracle.HEATBATH)), step
        assert np.array_equal(g.spins(), o.spins()), step


CASES = [
    # L, q, start, beta, sweeps, layout
    (32, 2, 1, 0.44, 40, potts.LAYOUT_U8),
    (96, 3, 1, 1.0, 30, potts.LAYOUT_U8),     # 3 chunks per row
    (160, 16, 0, 1.3, 25, potts.LAYOUT_U8),
    (288, 17, 1, 1.2, 20, potts.LAYOUT_U8),
    (544, 32, 1, 1.1, 12, potts.LAYOUT_U8),   # ragged tail over 128 threads
    (224, 96, 1, workloads.beta_at(96, 1.0), 20, potts.LAYOUT_U8),
    (64, 256, 1, 3.0, 30, potts.LAYOUT_U8),   # q = 256: every byte value
    (128, 9, 1, 0.0, 5, potts.LAYOUT_U8),     # beta = 0: uniform draws
    (128, 9, 0, 5.5, 10, potts.LAYOUT_U8),    # near the largest beta (m = 3)
    (4160, 15, 1, workloads.beta_at(15, 1.0), 2, potts.LAYOUT_U8),
    (96, 9, 1, math.log(4.0), 20, potts.LAYOUT_U4),
    (544, 15, 1, 1.1, 8, potts.LAYOUT_U4),
]


@pytest.mark.parametrize("L,q,start,beta,sweeps,layout", CASES)
def test_sizes_classes_and_layouts(L, q, start, beta, sweeps, layout):
    seed = 500 + L + q
    g = potts.Lattice(L, q, start, seed, layout=layout)
    g.set_update(HB)
    o = oracle.Lattice(L, q, start, seed)
    rg = g.sweep(beta, sweeps)
    ro = o.sweep(beta, sweeps, check=True, update=oracle.HEATBATH)
    assert np.array_equal(rg, ro)
    assert np.array_equal(g.spins(), o.spins())


def test_switching_rules_between_calls():
    g = potts.Lattice(128, 9, 1, 21)
    o = oracle.Lattice(128, 9, 1, 21)
    for rule in (HB, potts.UPDATE_METROPOLIS, HB):
        g.set_update(rule)
        assert np.array_equal(g.sweep(1.2, 4), o.sweep(1.2, 4, update=rule))
    assert np.array_equal(g.spins(), o.spins())


def test_rejects_bad_rule_and_beta():
    g = potts.Lattice(64, 9, 0, 1)
    with pytest.raises(potts.PottsError) as ei:
        g.set_update(7)
    assert ei.value.code == potts.POTTS_EINVAL
    g.set_update(HB)
    with pytest.raises(potts.PottsError) as ei:
        g.sweep(6.0, 1)
    assert ei.value.code == potts.POTTS_EINVAL
    assert g.sweep_index == 0


@pytest.mark.parametrize("L,q,layout", [(32768, 9, potts.LAYOUT_U8),
                                        (16384, 96, potts.LAYOUT_U8),
                                        (32768, 15, potts.LAYOUT_U4)])
def test_full_size_sampled(L, q, layout):
    seed = 11
    beta = workloads.beta_at(q, 1.0)
    g = potts.Lattice(L, q, 1, seed, layout=layout)
    g.set_update(HB)
    g.sweep(beta, 2, records=False)
    pre, t = g.spins(), g.sweep_index
    rec = g.sweep(beta, 1)
    post = g.spins()
    idx = np.random.default_rng(L + q).integers(0, L * L, 200_000,
                                                dtype=np.int64)
    expect = oracle.sweep_sites(pre, q, seed, t, beta, idx,
                                update=oracle.HEATBATH)
    assert np.array_equal(post.ravel()[idx], expect)
    B, hist = oracle.recount(post, q)
    assert int(rec[0, 0]) == B and np.array_equal(rec[0, 1:], hist)


@pytest.mark.parametrize("q,t_over_tc", [(9, 0.95), (9, 1.05), (24, 1.1)])
def test_heatbath_and_metropolis_sample_the_same_ensemble(q, t_over_tc):
    """Both rules leave the Boltzmann distribution invariant, so long-run
    <e> and <m> agree within their statistical errors (L = 256, away from
    the transition so both relax quickly)."""
    from paper_1101_0876_gb300.analysis import batch_means, energy_magnetization
    L = 256
    beta = workloads.beta_at(q, t_over_tc)
    res = {}
    for rule in (potts.UPDATE_METROPOLIS, HB):
        g = potts.Lattice(L, q, 0 if t_over_tc < 1 else 1, 40 + rule)
        g.set_update(rule)
        g.sweep(beta, 3000, records=False)
        e, m = energy_magnetization(g.sweep(beta, 20000), L, q)
        res[rule] = (batch_means(e, 50), batch_means(m, 50))
    for k in range(2):
        (a, ea), (b, eb) = res[potts.UPDATE_METROPOLIS][k], res[HB][k]
        assert abs(a - b) < 5 * math.hypot(ea, eb) + 1e-6, (k, a, b, ea, eb)
