"""Host protocols of the paper's runs, driven through the batch engine.

- `ladder`: the heating / cooling protocol (Sec. 3): a sequence of
  temperatures visited in order, the spins carried over from one
  temperature to the next, t_tran unmeasured sweeps then t_max measured
  sweeps at each; heating starts ordered and walks T upwards, cooling starts
  at random and walks T downwards.  Several independent samples run as
  members of one batch.
- `transition`: the two phases at exactly T_c (Sec. 4, Table 2): for each q,
  samples started ordered stay on the ordered branch (e_o, m_o) and samples
  started at random relax to the disordered one (e_d, m_d) on a large
  lattice; equilibration and measurement sweeps, averages per sample, and
  the spread over samples as the error.

Every quantity is formed in FP64 from the exact per-sweep integer records
{B, hist} (e = -B/N, m = (q N_max/N - 1)/(q - 1)).  `batch_factory` builds
the batch (default: potts.Batch, or potts.Lattice for a single sample); the
tests pass a CPU stand-in with the same interface to check the bookkeeping.

Command line:
    python -m paper_1101_0876_gb300.protocol x9          # Sec. 5 end-to-end run
    python -m paper_1101_0876_gb300.protocol mid         # L=4096 heating+cooling
    python -m paper_1101_0876_gb300.protocol transition  # Table 2 at L=2048
    python -m paper_1101_0876_gb300.protocol fig3        # Fig. 3 curves, L=2048
Each prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import workloads
from .analysis import energy_magnetization, exact_energies

START_ORDERED, START_RANDOM = 0, 1


class _OneLattice:
    """A single lattice behind the batch interface: one sample runs on the
    single-lattice path, whose direct launches beat a one-member batch."""

    def __init__(self, L, q, start, seed):
        from . import potts
        self._lat = potts.Lattice(L[0], q[0], start[0], seed[0])

    def set_update(self, update):
        self._lat.set_update(int(update[0]))

    def sweep(self, beta, n, records=True):
        out = self._lat.sweep(beta[0], n, records=records)
        return [out] if records else None

    def close(self):
        self._lat.close()


def _default_factory(L, q, start, seed):
    from . import potts
    if len(L) == 1:
        return _OneLattice(L, q, start, seed)
    return potts.Batch(L, q, start, seed)


def ladder(L: int, q: int, temps, t_tran: int, t_max: int, samples: int,
           start: int, seed0: int = 1, batch_factory=None, chunk: int = 4000,
           update: int = 0):
    """Runs `samples` independent lattices (seeds seed0 + s) through the
    temperature sequence `temps` (absolute T, visited in the given order).
    Returns (rows, seconds, updates): rows[k] = dict(T, e, m, e_err, m_err)
    with means over the t_max measured sweeps of each sample, then over the
    samples (error: standard error over samples)."""
    factory = batch_factory or _default_factory
    b = factory([L] * samples, [q] * samples, [start] * samples,
                [seed0 + s for s in range(samples)])
    if update:
        b.set_update([update] * samples)
    rows = []
    t0 = time.perf_counter()
    for T in temps:
        beta = [1.0 / float(T)] * samples
        if t_tran:
            b.sweep(beta, t_tran, records=False)
        se = np.zeros(samples)
        sm = np.zeros(samples)
        left = t_max
        while left > 0:
            n = min(chunk, left)
            recs = b.sweep(beta, n)
            for s in range(samples):
                e, m = energy_magnetization(recs[s], L, q)
                se[s] += e.sum()
                sm[s] += m.sum()
            left -= n
        e_s, m_s = se / t_max, sm / t_max
        rows.append(dict(T=float(T), e=float(e_s.mean()), m=float(m_s.mean()),
                         e_err=_sem(e_s), m_err=_sem(m_s)))
    secs = time.perf_counter() - t0
    b.close()
    upd = L * L * samples * len(list(temps)) * (t_tran + t_max)
    return rows, secs, upd


def transition(qs, L: int, samples: int, t_eq: int, t_meas: int,
               seed0: int = 100, batch_factory=None, chunk: int = 2000,
               update: int = 0):
    """Both branches at exactly T_c for every q in qs, all in one batch:
    per q, `samples` lattices started ordered and `samples` started at
    random (seeds seed0 + 1000 q + s and seed0 + 1000 q + 500 + s).
    Returns (table, seconds, updates), table[q] = dict(e_o, e_o_err, e_d,
    e_d_err, dm, dm_err, m_o, m_d, exact_e_o, exact_e_d)."""
    factory = batch_factory or _default_factory
    Ls, qq, st, sd, beta = [], [], [], [], []
    for q in qs:
        for branch in (START_ORDERED, START_RANDOM):
            for s in range(samples):
                Ls.append(L)
                qq.append(q)
                st.append(branch)
                sd.append(seed0 + 1000 * q + 500 * branch + s)
                beta.append(workloads.beta_at(q, 1.0))
    n = len(Ls)
    b = factory(Ls, qq, st, sd)
    if update:
        b.set_update([update] * n)
    t0 = time.perf_counter()
    left = t_eq
    while left > 0:
        k = min(left, 100000)
        b.sweep(beta, k, records=False)
        left -= k
    se = np.zeros(n)
    sm = np.zeros(n)
    left = t_meas
    while left > 0:
        k = min(chunk, left)
        recs = b.sweep(beta, k)
        for i in range(n):
            e, m = energy_magnetization(recs[i], L, qq[i])
            se[i] += e.sum()
            sm[i] += m.sum()
        left -= k
    secs = time.perf_counter() - t0
    b.close()
    se /= t_meas
    sm /= t_meas
    table = {}
    i = 0
    for q in qs:
        eo, mo = se[i:i + samples], sm[i:i + samples]
        ed, md = se[i + samples:i + 2 * samples], sm[i + samples:i + 2 * samples]
        i += 2 * samples
        x_o, x_d = exact_energies(q)
        table[q] = dict(e_o=float(eo.mean()), e_o_err=_sem(eo),
                        e_d=float(ed.mean()), e_d_err=_sem(ed),
                        dm=float(mo.mean() - md.mean()),
                        dm_err=math.hypot(_sem(mo), _sem(md)),
                        m_o=float(mo.mean()), m_d=float(md.mean()),
                        exact_e_o=x_o, exact_e_d=x_d)
    upd = L * L * n * (t_eq + t_meas)
    return table, secs, upd


def _sem(x) -> float:
    x = np.asarray(x, dtype=np.float64)
    if x.size < 2:
        return float("nan")
    return float(x.std(ddof=1) / math.sqrt(x.size))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("run", choices=["x9", "mid", "transition", "fig3"])
    ap.add_argument("--t-tran", type=int, default=10000)
    ap.add_argument("--t-max", type=int, default=20000)
    ap.add_argument("--L", type=int, default=0)
    ap.add_argument("--samples", type=int, default=0)
    ap.add_argument("--t-eq", type=int, default=500000)
    ap.add_argument("--t-meas", type=int, default=500000)
    ap.add_argument("--q", type=int, nargs="*", default=[6, 9, 15, 96])
    ap.add_argument("--update", choices=["metropolis", "heatbath"],
                    default="metropolis")
    a = ap.parse_args(argv)
    upd_rule = 1 if a.update == "heatbath" else 0
    out = {"run": a.run, "update": a.update}
    if a.run == "x9":
        # Sec. 5 end-to-end run: q=9, L=1024, 3 samples, T from 0.71 to
        # 0.73 in steps of 0.002, t_tran = 2000, t_max = 8000 (records every
        # sweep, a superset of the paper's delta t = 50); both directions.
        L, q, S = a.L or 1024, 9, a.samples or 3
        temps = [0.71 + 0.002 * k for k in range(11)]
        heat = ladder(L, q, temps, 2000, 8000, S, START_ORDERED, 1,
                      update=upd_rule)
        cool = ladder(L, q, temps[::-1], 2000, 8000, S, START_RANDOM, 101,
                      update=upd_rule)
        out.update(L=L, q=q, samples=S,
                   heating=dict(rows=heat[0], seconds=heat[1],
                                updates_per_s=heat[2] / heat[1]),
                   cooling=dict(rows=cool[0], seconds=cool[1],
                                updates_per_s=cool[2] / cool[1]),
                   seconds_total=heat[1] + cool[1])
    elif a.run == "mid":
        cfg = workloads.MID
        L, q = a.L or cfg["L"], cfg["q"]
        temps = [workloads.tc(q) * t for t in cfg["ladder"]]
        n = cfg["sweeps_per_t"]
        heat = ladder(L, q, temps, 0, n, 1, START_ORDERED, cfg["seed"],
                      update=upd_rule)
        cool = ladder(L, q, temps[::-1], 0, n, 1, START_RANDOM, cfg["seed"],
                      update=upd_rule)
        out.update(L=L, q=q,
                   heating=dict(rows=heat[0], seconds=heat[1],
                                updates_per_s=heat[2] / heat[1]),
                   cooling=dict(rows=cool[0], seconds=cool[1],
                                updates_per_s=cool[2] / cool[1]))
    elif a.run == "fig3":
        # Sec. 4, Fig. 3: e(T) and m(T) near T_c for q = 9, 12, 15, 96 on
        # L = 2048, 10 samples, heating from the ordered start and cooling
        # from the random start over T / T_c in [0.97, 1.03]
        L, S = a.L or 2048, a.samples or 10
        ratios = [0.97 + 0.005 * k for k in range(13)]
        curves, secs_all, upd_all = {}, 0.0, 0
        for q in (9, 12, 15, 96):
            temps = [workloads.tc(q) * r for r in ratios]
            heat = ladder(L, q, temps, a.t_tran, a.t_max, S, START_ORDERED,
                          1000 * q, update=upd_rule)
            cool = ladder(L, q, temps[::-1], a.t_tran, a.t_max, S,
                          START_RANDOM, 1000 * q + 500, update=upd_rule)
            curves[str(q)] = dict(heating=heat[0], cooling=cool[0][::-1])
            secs_all += heat[1] + cool[1]
            upd_all += heat[2] + cool[2]
        out.update(L=L, samples=S, t_tran=a.t_tran, t_max=a.t_max,
                   t_over_tc=ratios, curves=curves, seconds=secs_all,
                   updates_per_s=upd_all / secs_all)
    else:
        L, S = a.L or 2048, a.samples or 10
        table, secs, upd = transition(a.q, L, S, a.t_eq, a.t_meas,
                                      update=upd_rule)
        out.update(L=L, samples=S, t_eq=a.t_eq, t_meas=a.t_meas,
                   seconds=secs, updates_per_s=upd / secs,
                   table={str(k): v for k, v in table.items()})
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
