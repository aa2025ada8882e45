"""CUDA path against the CPU oracle, bit for bit (needs a GPU).

Every random variate is a pure function of (seed, sweep, colour, site), so
the GPU must reproduce the oracle's spins and per-sweep records {B, hist}
exactly, for every size, q class, start and acceptance rule.
"""
import math

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


def test_small_config_every_sweep():
    """L=64, q=9, ordered start, T = T_c, seed 1, 1000 sweeps: records of
    every sweep and the spins after every sweep."""
    cfg = workloads.SMALL
    beta = workloads.beta_at(cfg.q, 1.0)
    g = potts.Lattice(cfg.L, cfg.q, cfg.start, cfg.seed)
    o = oracle.Lattice(cfg.L, cfg.q, cfg.start, cfg.seed)
    assert np.array_equal(g.spins(), o.spins())
    for step in range(cfg.sweeps // 50):
        for _ in range(50):
            rg = g.sweep(beta, 1)
            ro = o.sweep(beta, 1)
            assert np.array_equal(rg, ro), step
            assert np.array_equal(g.spins(), o.spins()), step
    obs = g.observables()
    assert obs["sweep"] == cfg.sweeps
    e, m = oracle.observables(ro, cfg.L, cfg.q)
    assert obs["e"] == e[0] and obs["m"] == m[0]


CASES = [
    # L, q, start, beta, sweeps
    (32, 2, 1, 0.44, 40),           # minimum L (one 16-byte chunk per row)
    (96, 9, 1, math.log(4.0), 30),  # 3 chunks per row: ragged CTA width
    (160, 16, 0, 1.3, 25),          # q = 16 (largest 4-bit class)
    (288, 17, 1, 1.2, 20),          # q = 17 (5-bit class)
    (544, 32, 1, 1.1, 12),          # 17 chunks: ragged tail over 128 threads
    (224, 33, 1, 1.0, 20),          # 6-bit class
    (192, 64, 0, 1.6, 20),
    (256, 65, 1, 1.0, 20),          # 7-bit class
    (128, 128, 1, 2.0, 20),
    (96, 129, 1, 1.0, 20),          # exact zero-byte test
    (64, 256, 1, 3.0, 30),          # q = 256 (all byte values)
    (128, 9, 1, 0.0, 5),            # beta = 0: every proposal accepted
    (128, 9, 0, 40.0, 5),           # thr = 0: frozen, rule "dE <= 0 or a < thr"
    (128, 6, 1, 6.0, 10),           # thr[4] = 0 only: mixed rule
    (4160, 15, 1, workloads.beta_at(15, 1.0), 2),   # 2080 B rows: 2 CTAs wide
]


@pytest.mark.parametrize("L,q,start,beta,sweeps", CASES)
def test_sizes_and_classes(L, q, start, beta, sweeps):
    seed = 1000 + L + q
    g = potts.Lattice(L, q, start, seed)
    o = oracle.Lattice(L, q, start, seed)
    assert np.array_equal(g.spins(), o.spins())
    rg = g.sweep(beta, sweeps)
    ro = o.sweep(beta, sweeps, check=True)
    assert np.array_equal(rg, ro)
    assert np.array_equal(g.spins(), o.spins())


def test_sweep_index_continues_across_calls_and_zero_sweeps():
    a = potts.Lattice(128, 9, 1, 5)
    b = potts.Lattice(128, 9, 1, 5)
    ra = np.concatenate([a.sweep(1.3, 5), a.sweep(1.3, 0), a.sweep(1.3, 7)])
    rb = b.sweep(1.3, 12)
    assert np.array_equal(ra, rb)
    assert a.observables()["sweep"] == 12


def test_temperature_ladder_matches_oracle():
    """The paper's protocol: spins carry over from one T to the next."""
    g = potts.Lattice(128, 9, 0, 7)
    o = oracle.Lattice(128, 9, 0, 7)
    for t in workloads.mid_ladder()[:6]:
        beta = workloads.beta_at(9, t)
        assert np.array_equal(g.sweep(beta, 10), o.sweep(beta, 10))
    assert np.array_equal(g.spins(), o.spins())


def test_set_state_resume_and_recount():
    L, q = 256, 12
    spins = workloads.random_spins(L, q, 3)
    g = potts.Lattice(L, q, 0, 9)
    g.set_state(spins, 123456789012)
    assert np.array_equal(g.spins(), spins)
    B, hist = oracle.recount(spins, q)
    obs = g.observables()
    assert obs["bonds"] == B and obs["sweep"] == 123456789012
    o = oracle.Lattice(L, q, 0, 9)
    o.set_state(spins, 123456789012)
    assert np.array_equal(g.sweep(1.5, 4), o.sweep(1.5, 4))
    assert np.array_equal(g.spins(), o.spins())


def test_set_state_rejects_out_of_range():
    g = potts.Lattice(64, 5, 0, 1)
    bad = np.zeros((64, 64), np.uint8)
    bad[3, 4] = 5
    with pytest.raises(potts.PottsError) as ei:
        g.set_state(bad, 0)
    assert ei.value.code == potts.POTTS_EINVAL


def test_running_sums_from_records():
    g = potts.Lattice(128, 9, 1, 2)
    g.reset_averages()
    rec = g.sweep(math.log(4.0), 40)
    e, m = oracle.observables(rec, 128, 9)
    obs = g.observables()
    assert obs["nsamples"] == 40
    assert obs["sum_e"] == pytest.approx(e.sum(), rel=1e-14)
    assert obs["sum_e2"] == pytest.approx((e * e).sum(), rel=1e-14)
    assert obs["sum_e4"] == pytest.approx((e ** 4).sum(), rel=1e-14)
    assert obs["sum_m"] == pytest.approx(m.sum(), rel=1e-14)
    assert obs["sum_m2"] == pytest.approx((m * m).sum(), rel=1e-14)


def test_torch_stream():
    import torch
    s = torch.cuda.Stream()
    g = potts.Lattice(128, 9, 1, 4)
    g.set_stream(s.cuda_stream)
    o = oracle.Lattice(128, 9, 1, 4)
    assert np.array_equal(g.sweep(1.4, 6), o.sweep(1.4, 6))
    g.set_stream(None)
    assert np.array_equal(g.sweep(1.4, 3), o.sweep(1.4, 3))


# ---------------------------------------------------------- full size
def _sampled_sweep_parity(L, q, start, seed, t_over_tc, warm, nsample=200_000):
    beta = workloads.beta_at(q, t_over_tc)
    g = potts.Lattice(L, q, start, seed)
    rng = np.random.default_rng(L + q)
    idx = rng.integers(0, L * L, nsample, dtype=np.int64)
    pre = g.spins()
    assert np.array_equal(pre.ravel()[idx],
                          oracle.init_sites(L, q, start, seed, idx))
    if warm:
        g.sweep(beta, warm, records=False)
        pre = g.spins()
    t = g.sweep_index
    rec = g.sweep(beta, 1)
    post = g.spins()
    expect = oracle.sweep_sites(pre, q, seed, t, beta, idx)
    assert np.array_equal(post.ravel()[idx], expect)
    B, hist = oracle.recount(post, q)
    assert int(rec[0, 0]) == B
    assert np.array_equal(rec[0, 1:], hist)


@pytest.mark.parametrize("q,t_over_tc", [(9, 1.0), (15, 0.995)])
def test_paper_scale_sampled(q, t_over_tc):
    cfg = workloads.PAPER_Q9
    _sampled_sweep_parity(cfg.L, q, cfg.start, cfg.seed, t_over_tc, warm=3)


def test_maximum_size_L65536_sampled():
    """The largest lattice the library accepts (L = 65536: 4.3e9 sites, two
    2 GiB planes; site indices up to 2^31, Philox counters up to 2^30)."""
    _sampled_sweep_parity(65536, 9, 1, 5, 1.0, warm=0, nsample=100_000)


def test_q96_L16384_sampled():
    cfg = workloads.PAPER_Q96
    _sampled_sweep_parity(cfg.L, cfg.q, cfg.start, cfg.seed, 1.005, warm=2)


# ------------------------------------------------------------ mid config
@pytest.mark.parametrize("start,ladder_dir", [(0, 1), (1, -1)])
def test_mid_config_protocol(start, ladder_dir):
    """L=4096, q=9, seed 7: heating from the ordered start (T ascending) and
    cooling from the random start (T descending) over the ladder in
    [0.97, 1.03] T_c.  The first two temperatures (2 sweeps each) are
    compared with the oracle in full; after 3 x 40 more sweeps one sweep is
    compared on sampled sites."""
    L, q, seed = workloads.MID["L"], workloads.MID["q"], workloads.MID["seed"]
    ladder = list(workloads.MID["ladder"])[::ladder_dir]
    g = potts.Lattice(L, q, start, seed)
    o = oracle.Lattice(L, q, start, seed)
    for t in ladder[:2]:
        b = workloads.beta_at(q, t)
        assert np.array_equal(g.sweep(b, 2), o.sweep(b, 2)), t
    assert np.array_equal(g.spins(), o.spins())
    for t in ladder[2:5]:
        g.sweep(workloads.beta_at(q, t), 40, records=False)
    b = workloads.beta_at(q, ladder[5])
    pre, tidx = g.spins(), g.sweep_index
    rec = g.sweep(b, 1)
    idx = np.random.default_rng(5).integers(0, L * L, 200_000, dtype=np.int64)
    assert np.array_equal(g.spins().ravel()[idx],
                          oracle.sweep_sites(pre, q, seed, tidx, b, idx))
    B, hist = oracle.recount(g.spins(), q)
    assert int(rec[0, 0]) == B and np.array_equal(rec[0, 1:], hist)


# ------------------------------------------------------- packed 4-bit layout
U4_CASES = [(4096, 16, 0, 40.0, 2),       # 32-site nibble walks, rule LT0
            (32, 2, 1, 0.44, 30), (96, 9, 0, math.log(4.0), 20),
            (160, 16, 1, 1.3, 15), (544, 15, 1, 1.1, 8), (128, 9, 0, 40.0, 4),
            (128, 6, 1, 0.0, 4), (64, 9, 1, 1.1, 10),
            (4160, 9, 1, workloads.beta_at(9, 1.0), 2)]


@pytest.mark.parametrize("L,q,start,beta,sweeps", U4_CASES)
def test_u4_layout_matches_oracle(L, q, start, beta, sweeps):
    seed = 77 + L
    g = potts.Lattice(L, q, start, seed, layout=potts.LAYOUT_U4)
    o = oracle.Lattice(L, q, start, seed)
    assert np.array_equal(g.spins(), o.spins())
    assert np.array_equal(g.sweep(beta, sweeps), o.sweep(beta, sweeps))
    assert np.array_equal(g.spins(), o.spins())
    assert g.device_planes()[2] == L // 4


def test_u4_equals_u8_and_rejects_large_q():
    a = potts.Lattice(2048, 12, 1, 3, layout=potts.LAYOUT_U4)
    b = potts.Lattice(2048, 12, 1, 3, layout=potts.LAYOUT_U8)
    assert np.array_equal(a.sweep(1.2, 20), b.sweep(1.2, 20))
    assert np.array_equal(a.spins(), b.spins())
    spins = workloads.random_spins(256, 16, 9)
    c = potts.Lattice(256, 16, 0, 4, layout=potts.LAYOUT_U4)
    c.set_state(spins, 5)
    assert np.array_equal(c.spins(), spins)
    with pytest.raises(potts.PottsError) as ei:
        potts.Lattice(64, 17, 0, 1, layout=potts.LAYOUT_U4)
    assert ei.value.code == potts.POTTS_EINVAL


def test_u4_paper_scale_sampled():
    L, q, seed = 32768, 9, 11
    beta = workloads.beta_at(q, 1.0)
    g = potts.Lattice(L, q, 1, seed, layout=potts.LAYOUT_U4)
    g.sweep(beta, 2, records=False)
    pre, t = g.spins(), g.sweep_index
    rec = g.sweep(beta, 1)
    idx = np.random.default_rng(3).integers(0, L * L, 200_000, dtype=np.int64)
    assert np.array_equal(g.spins().ravel()[idx],
                          oracle.sweep_sites(pre, q, seed, t, beta, idx))
    B, hist = oracle.recount(g.spins(), q)
    assert int(rec[0, 0]) == B and np.array_equal(rec[0, 1:], hist)


def test_shared_memory_opt_in_across_sizes():
    """Passes whose per-lane counters need more than 48 KB of shared memory
    (q = 200 and q = 256: 200 and 256 bins of 256 bytes) alternating in one
    process with each other and with a small one: every launch opts in, and
    records and spins stay equal to the oracle's."""
    for L, q in [(64, 200), (64, 256), (96, 200), (64, 9), (64, 256)]:
        seed, beta = 40 + q + L, 1.5
        g = potts.Lattice(L, q, 1, seed)
        o = oracle.Lattice(L, q, 1, seed)
        assert np.array_equal(g.sweep(beta, 3), o.sweep(beta, 3)), (L, q)
        assert np.array_equal(g.spins(), o.spins()), (L, q)


@pytest.mark.parametrize("L,q,start,beta", [
    (4096, 2, 1, 0.44), (4096, 16, 0, 40.0), (4096, 9, 1, 0.0),
    (4160, 9, 1, workloads.beta_at(9, 1.0)),    # 65 chunks of 32 per row
])
def test_wide_walks_match_oracle(L, q, start, beta):
    """Planes of 2^23 sites and more take the 32-site byte walks with the
    cross-plane histogram (the white pass counts nothing, the black pass
    both planes): whole-lattice records and spins equal the oracle's."""
    seed = 7 + q + L
    g = potts.Lattice(L, q, start, seed)
    o = oracle.Lattice(L, q, start, seed)
    assert np.array_equal(g.sweep(beta, 2), o.sweep(beta, 2))
    assert np.array_equal(g.spins(), o.spins())
