"""Bookkeeping of the host protocols (ladder, transition) on the CPU: the
batch is replaced by a stand-in of serial oracle lattices with the same
interface, and every reported mean is recomputed from lattices driven by
hand through the same sequence."""
import numpy as np

import oracle
from paper_1101_0876_gb300 import protocol, workloads
from paper_1101_0876_gb300.analysis import energy_magnetization


class OracleBatch:
    def __init__(self, L, q, start, seed):
        self.q = list(q)
        self.lat = [oracle.Lattice(a, b, c, d) for a, b, c, d in
                    zip(L, q, start, seed)]
        self.closed = False

    def set_update(self, update):
        self.update = list(update)

    def sweep(self, beta, n, records=True):
        upd = getattr(self, "update", [0] * len(self.lat))
        out = [x.sweep(b, n, records=records, update=u)
               for x, b, u in zip(self.lat, beta, upd)]
        return out if records else None

    def close(self):
        self.closed = True


def _means(rec, L, q):
    e, m = energy_magnetization(rec, L, q)
    return e.mean(), m.mean()


def test_ladder_matches_hand_driven_lattices():
    L, q, S = 8, 3, 2
    temps = [1.2, 1.0, 0.8]
    rows, secs, upd = protocol.ladder(L, q, temps, 5, 7, S,
                                      protocol.START_RANDOM, seed0=40,
                                      batch_factory=OracleBatch, chunk=3)
    assert [r["T"] for r in rows] == temps
    assert upd == L * L * S * 3 * 12
    hand = [oracle.Lattice(L, q, 1, 40 + s) for s in range(S)]
    for r, T in zip(rows, temps):
        es, ms = [], []
        for h in hand:
            h.sweep(1.0 / T, 5, records=False)
            e, m = _means(h.sweep(1.0 / T, 7), L, q)
            es.append(e)
            ms.append(m)
        assert np.isclose(r["e"], np.mean(es), rtol=0, atol=1e-12)
        assert np.isclose(r["m"], np.mean(ms), rtol=0, atol=1e-12)
        assert np.isclose(r["e_err"], np.std(es, ddof=1) / np.sqrt(S))


def test_transition_groups_branches_per_q():
    L, S, qs = 8, 2, [3, 5]
    table, secs, upd = protocol.transition(qs, L, S, t_eq=6, t_meas=9,
                                           seed0=3, batch_factory=OracleBatch,
                                           chunk=4)
    assert upd == L * L * len(qs) * 2 * S * 15
    for q in qs:
        beta = workloads.beta_at(q, 1.0)
        br = {}
        for branch in (0, 1):
            es, ms = [], []
            for s in range(S):
                h = oracle.Lattice(L, q, branch, 3 + 1000 * q + 500 * branch + s)
                h.sweep(beta, 6, records=False)
                e, m = _means(h.sweep(beta, 9), L, q)
                es.append(e)
                ms.append(m)
            br[branch] = (np.mean(es), np.mean(ms))
        t = table[q]
        assert np.isclose(t["e_o"], br[0][0], rtol=0, atol=1e-12)
        assert np.isclose(t["e_d"], br[1][0], rtol=0, atol=1e-12)
        assert np.isclose(t["dm"], br[0][1] - br[1][1], rtol=0, atol=1e-12)


def test_heatbath_rule_reaches_every_lattice():
    L, q, S = 8, 3, 2
    rows, _, _ = protocol.ladder(L, q, [1.1], 3, 5, S, protocol.START_RANDOM,
                                 seed0=9, batch_factory=OracleBatch,
                                 update=oracle.HEATBATH)
    es = []
    for s in range(S):
        h = oracle.Lattice(L, q, 1, 9 + s)
        h.sweep(1.0 / 1.1, 3, records=False, update=oracle.HEATBATH)
        es.append(_means(h.sweep(1.0 / 1.1, 5, update=oracle.HEATBATH), L, q)[0])
    assert np.isclose(rows[0]["e"], np.mean(es), rtol=0, atol=1e-12)
