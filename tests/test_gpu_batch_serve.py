"""Batched and served paths against the oracle and the single-lattice path.

A lattice's records must be identical whether it runs alone
(potts_create/potts_sweep), inside a batch, or as a served request mixed
with others: every variate depends only on (seed, sweep, colour, site).
"""
import math
import time

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


MIX = [  # L, q, start, seed, beta
    (64, 9, 0, 1, math.log(4.0)),
    (96, 6, 1, 2, workloads.beta_at(6, 1.01)),
    (128, 15, 1, 3, workloads.beta_at(15, 0.99)),
    (160, 24, 0, 4, workloads.beta_at(24, 1.0)),
    (32, 2, 1, 5, 0.44),
    (224, 96, 1, 6, workloads.beta_at(96, 1.02)),
    (64, 256, 1, 7, 3.0),
    (288, 9, 1, 8, 0.0),
    (96, 9, 0, 9, 40.0),
    (544, 15, 1, 10, workloads.beta_at(15, 1.0)),
    (128, 9, 1, 11, 40.0),              # 32-site walks, acceptance rule LT0
    (320, 6, 0, 12, workloads.beta_at(6, 1.0)),  # 32-site walks, 5 per row
]


def _oracle_run(L, q, start, seed, beta, n):
    o = oracle.Lattice(L, q, start, seed)
    return o.sweep(beta, n), o


def test_batch_matches_oracle_every_lattice():
    L, q, st, sd, be = zip(*MIX)
    b = potts.Batch(L, q, st, sd)
    recs = b.sweep(be, 37)              # crosses several graph steps
    recs2 = b.sweep(be, 5)
    for i, (Li, qi, si, sdi, bi) in enumerate(MIX):
        ro, o = _oracle_run(Li, qi, si, sdi, bi, 42)
        assert np.array_equal(np.concatenate([recs[i], recs2[i]]), ro), i
        assert np.array_equal(b.spins(i), o.spins()), i
        obs = b.observables(i)
        assert obs["sweep"] == 42 and obs["nsamples"] == 42


def test_batch_equals_single_lattice_path():
    spec = workloads.batched(n=16, L_lo=512, L_hi=2048, sweeps=30)
    b = potts.Batch(spec.L, spec.q, spec.start, spec.seed)
    recs = b.sweep(spec.beta, spec.sweeps)
    for i in range(0, 16, 3):
        g = potts.Lattice(spec.L[i], spec.q[i], spec.start[i], spec.seed[i])
        rg = g.sweep(spec.beta[i], spec.sweeps)
        assert np.array_equal(recs[i], rg), i
        assert np.array_equal(b.spins(i), g.spins()), i


def test_batched_config_sampled():
    """The batched configuration (256 lattices, L 64..2048, q in
    {6, 9, 15, 24}, 500 sweeps): small lattices fully against the oracle,
    a sample of the large ones against the single-lattice path."""
    spec = workloads.batched()
    b = potts.Batch(spec.L, spec.q, spec.start, spec.seed)
    recs = b.sweep(spec.beta, spec.sweeps)
    order = np.argsort(spec.L)
    for i in order[:4]:
        ro, o = _oracle_run(spec.L[i], spec.q[i], spec.start[i], spec.seed[i],
                            spec.beta[i], spec.sweeps)
        assert np.array_equal(recs[i], ro), i
        assert np.array_equal(b.spins(i), o.spins()), i
    for i in order[-3:]:
        g = potts.Lattice(spec.L[i], spec.q[i], spec.start[i], spec.seed[i])
        assert np.array_equal(recs[i], g.sweep(spec.beta[i], spec.sweeps)), i


def test_batch_rejects_bad_input():
    with pytest.raises(potts.PottsError):
        potts.Batch([64, 48], [9, 9], [0, 0], [1, 2])
    b = potts.Batch([64], [9], [0], [1])
    with pytest.raises(potts.PottsError):
        b.sweep([-1.0], 3)


# ----------------------------------------------------------------- serve
def _drain(srv, rids, timeout=120.0):
    out = {r: [] for r in rids}
    pending = set(rids)
    t0 = time.time()
    while pending and time.time() - t0 < timeout:
        for r in list(pending):
            rec, done = srv.poll(r)
            if len(rec):
                out[r].append(rec)
            if done:
                pending.discard(r)
        time.sleep(0.002)
    assert not pending, "requests did not finish"
    return {r: np.concatenate(v) for r, v in out.items()}


def test_serve_alone_equals_mixed():
    srv = potts.Server(hbm_budget_bytes=1 << 30, max_slots=4,
                       sweeps_per_step=8)
    reqs = [(64, 9, 0.9 * math.log(4.0), 30, 11), (128, 15, 1.2, 45, 12),
            (96, 24, 1.0, 17, 13), (32, 2, 0.5, 60, 14), (160, 96, 2.0, 9, 15),
            (64, 6, 1.1, 33, 16), (224, 9, 1.3, 25, 17)]
    rids = [srv.submit(L, q, b, n, s) for (L, q, b, n, s) in reqs]
    got = _drain(srv, rids)
    st = srv.stats()
    srv.stop()
    assert st["completed"] == len(reqs) and st["bytes_in_use"] == 0
    for rid, (L, q, b, n, s) in zip(rids, reqs):
        ro, _ = _oracle_run(L, q, 1, s, b, n)
        assert np.array_equal(got[rid], ro), rid
        g = potts.Lattice(L, q, 1, s)
        assert np.array_equal(got[rid], g.sweep(b, n)), rid


def test_serve_budget_queue_cancel_and_busy():
    one = 256 * 256
    srv = potts.Server(hbm_budget_bytes=one, max_slots=4, sweeps_per_step=4,
                       queue_capacity=1)
    with pytest.raises(potts.PottsError) as ei:   # can never fit
        srv.submit(512, 9, 1.0, 10, 1)
    assert ei.value.code == potts.POTTS_EINVAL
    with pytest.raises(potts.PottsError):
        srv.submit(48, 9, 1.0, 10, 1)
    a = srv.submit(256, 9, 1.0, 10**7, 2)         # holds the whole budget
    t0 = time.time()
    while srv.stats()["active"] < 1 and time.time() - t0 < 30:
        time.sleep(0.01)
    b = srv.submit(64, 9, 1.0, 5, 3)              # waits for memory
    with pytest.raises(potts.PottsError) as ei:   # queue (capacity 1) full
        srv.submit(64, 9, 1.0, 5, 4)
    assert ei.value.code == potts.POTTS_EBUSY
    time.sleep(0.2)
    assert srv.stats()["queued"] == 1             # b not admitted: no budget
    srv.cancel(a)
    t0 = time.time()
    while True:
        try:
            srv.poll(a)
        except potts.PottsError as e:
            assert e.code == potts.POTTS_ECANCELLED
            break
        assert time.time() - t0 < 30
        time.sleep(0.01)
    got = _drain(srv, [b])                        # b runs once a is gone
    ro, _ = _oracle_run(64, 9, 1, 3, 1.0, 5)
    assert np.array_equal(got[b], ro)
    with pytest.raises(potts.PottsError) as ei:
        srv.poll(12345)
    assert ei.value.code == potts.POTTS_ENOTFOUND
    srv.stop()


# ------------------------------------------------------------- heat bath
def test_batch_mixed_update_rules():
    """Heat-bath and Metropolis lattices in one batch: each lattice's records
    equal the oracle's with its own rule."""
    L, q, st, sd, be = zip(*MIX)
    rules = [potts.UPDATE_HEATBATH if i % 2 == 0 else potts.UPDATE_METROPOLIS
             for i in range(len(MIX))]
    be = [min(b, 5.0) for b in be]           # inside the heat-bath range
    b = potts.Batch(L, q, st, sd)
    b.set_update(rules)
    recs = b.sweep(be, 23)
    for i, (Li, qi, si, sdi, _) in enumerate(MIX):
        o = oracle.Lattice(Li, qi, si, sdi)
        ro = o.sweep(be[i], 23, update=rules[i])
        assert np.array_equal(recs[i], ro), i
        assert np.array_equal(b.spins(i), o.spins()), i
    with pytest.raises(potts.PottsError):
        b.set_update([5] * len(MIX))
    b.close()


def test_serve_heatbath_requests_alone_equal_mixed():
    srv = potts.Server(hbm_budget_bytes=1 << 30, max_slots=3,
                       sweeps_per_step=8)
    reqs = [(64, 9, math.log(4.0), 30, 21, 1), (128, 15, 1.2, 20, 22, 0),
            (96, 24, 1.0, 17, 23, 1), (160, 96, 2.0, 9, 24, 1),
            (224, 9, 1.3, 25, 25, 0)]
    rids = [srv.submit(L, q, b, n, s, update=u) for (L, q, b, n, s, u) in reqs]
    got = _drain(srv, rids)
    with pytest.raises(potts.PottsError) as ei:     # beyond the weights
        srv.submit(64, 9, 7.0, 5, 1, update=potts.UPDATE_HEATBATH)
    assert ei.value.code == potts.POTTS_EINVAL
    srv.stop()
    for rid, (L, q, b, n, s, u) in zip(rids, reqs):
        o = oracle.Lattice(L, q, 1, s)
        assert np.array_equal(got[rid], o.sweep(b, n, update=u)), rid


@pytest.mark.parametrize("policy", [potts.ADMIT_FIFO, potts.ADMIT_SMALLEST])
def test_serve_admission_policy(policy):
    """One slot, held by a long request while a large and then a small
    request queue up: FIFO runs the large one first, SMALLEST the small
    one; both give the oracle's records."""
    srv = potts.Server(hbm_budget_bytes=1 << 30, max_slots=1,
                       sweeps_per_step=4, policy=policy)
    a = srv.submit(256, 9, 1.0, 10**7, 1)
    t0 = time.time()
    while srv.stats()["active"] < 1 and time.time() - t0 < 30:
        time.sleep(0.01)
    big = srv.submit(512, 9, 1.0, 120, 2)
    small = srv.submit(64, 9, 1.0, 20, 3)
    srv.cancel(a)
    order, got, pending = [], {big: [], small: []}, {big, small}
    t0 = time.time()
    while pending and time.time() - t0 < 60:
        for r in list(pending):
            rec, done = srv.poll(r)
            if rec.size:
                got[r].append(rec)
            if done:
                order.append(r)
                pending.discard(r)
        time.sleep(0.002)
    srv.stop()
    assert not pending
    assert order == ([big, small] if policy == potts.ADMIT_FIFO
                     else [small, big])
    for r, (L, n, s) in ((big, (512, 120, 2)), (small, (64, 20, 3))):
        ro, _ = _oracle_run(L, 9, 1, s, 1.0, n)
        assert np.array_equal(np.concatenate(got[r]), ro), r


def test_serve_concurrent_clients():
    """Four host threads submit, poll and cancel on one server at once (the
    serving calls are thread-safe): every finished request equals the same
    lattice run alone, the cancelled one reports ECANCELLED, and the
    server's counts add up."""
    import threading
    srv = potts.Server(hbm_budget_bytes=1 << 30, max_slots=3,
                       sweeps_per_step=4)
    plans = {t: [(32 + 32 * ((t + k) % 4), [6, 9, 15, 24][(t + 2 * k) % 4],
                  0.8 + 0.1 * t + 0.05 * k, 10 + 7 * k, 100 * t + k)
                 for k in range(3)] for t in range(4)}
    results, errors = {}, []

    def client(t):
        try:
            mine = [(srv.submit(L, q, b, n, s), (L, q, b, n, s))
                    for (L, q, b, n, s) in plans[t]]
            victim = None
            if t == 0:  # a long request, cancelled while the others run
                victim = srv.submit(256, 9, 1.0, 10**7, 999)
            got = _drain(srv, [r for r, _ in mine])
            for rid, spec in mine:
                results[(t, rid)] = (got[rid], spec)
            if victim is not None:
                srv.cancel(victim)
                t0 = time.time()
                while True:
                    try:
                        srv.poll(victim)
                    except potts.PottsError as e:
                        assert e.code == potts.POTTS_ECANCELLED
                        break
                    assert time.time() - t0 < 30
                    time.sleep(0.01)
        except Exception as e:  # reported on the main thread
            errors.append(e)

    threads = [threading.Thread(target=client, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    st = srv.stats()
    srv.stop()
    assert not errors, errors
    assert len(results) == 12
    assert st["completed"] == 12 and st["cancelled"] == 1
    for (t, rid), (rec, (L, q, b, n, s)) in results.items():
        alone = potts.Lattice(L, q, 1, s).sweep(b, n)
        assert np.array_equal(rec, alone), (t, rid)
