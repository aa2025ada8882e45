"""Seeded synthetic workloads shaped like the paper's runs.

This module holds input recipes only (lattice sizes, q, temperatures, seeds,
request streams, random spin arrays for state uploads).  It contains none of
the sweep's arithmetic, imports neither the CUDA binding nor the oracle, and
is the one module both sides (tests, benchmark) draw inputs from.

Temperatures are given relative to the exact transition temperature
k_B T_c / J = 1/ln(1 + sqrt(q)) of the square-lattice model (Sec. 2.1,
Eq. 2); the sweep itself takes beta = 1/T.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def tc(q: int) -> float:
    """Exact transition temperature 1/ln(1+sqrt(q)) (Sec. 2.1, Eq. 2)."""
    return 1.0 / math.log1p(math.sqrt(q))


def beta_at(q: int, t_over_tc: float) -> float:
    """beta = 1/T for T = t_over_tc * T_c(q), formed as ln(1+sqrt q)/t."""
    return math.log1p(math.sqrt(q)) / float(t_over_tc)


# --- single-lattice configurations -------------------------------------

@dataclass(frozen=True)
class Single:
    name: str
    L: int
    q: int
    start: int          # 0 ordered (all 0), 1 random
    seed: int
    sweeps: int
    t_over_tc: tuple = (1.0,)


# L=64, q=9, ordered start, T = T_c (beta = ln 4), 1000 sweeps, seed 1.
SMALL = Single("small_L64_q9", 64, 9, 0, 1, 1000, (1.0,))

# Paper scale (Sec. 5 sweeps L up to 32768): q=9 and q=15 near T_c,
# random start, 200 sweeps, seed 11; plus q=96 at L=16384.
PAPER_Q9 = Single("paper_L32768_q9", 32768, 9, 1, 11, 200,
                  (0.995, 1.0, 1.005))
PAPER_Q15 = Single("paper_L32768_q15", 32768, 15, 1, 11, 200,
                   (0.995, 1.0, 1.005))
PAPER_Q96 = Single("paper_L16384_q96", 16384, 96, 1, 11, 200,
                   (0.995, 1.0, 1.005))


def mid_ladder(q: int = 9, n: int = 41, lo: float = 0.97,
               hi: float = 1.03) -> np.ndarray:
    """T/T_c values of the heating/cooling protocol (Sec. 3): n evenly
    spaced points in [lo, hi]."""
    return np.linspace(lo, hi, n)


MID = dict(L=4096, q=9, seed=7, sweeps_per_t=2000, ladder=mid_ladder())


# --- batched configuration ---------------------------------------------

@dataclass
class BatchSpec:
    L: list = field(default_factory=list)
    q: list = field(default_factory=list)
    start: list = field(default_factory=list)
    seed: list = field(default_factory=list)
    beta: list = field(default_factory=list)
    sweeps: int = 500


def batched(n: int = 256, harness_seed: int = 0, sweeps: int = 500,
            L_lo: int = 64, L_hi: int = 2048,
            q_choices=(6, 9, 15, 24)) -> BatchSpec:
    """n independent lattices: L log-uniform over [L_lo, L_hi] rounded to a
    multiple of 32, q uniform from q_choices, T uniform in [0.98, 1.02] T_c,
    even i ordered / odd i random, seed 1000 + i."""
    rng = np.random.default_rng(harness_seed)
    spec = BatchSpec(sweeps=sweeps)
    for i in range(n):
        Lf = math.exp(rng.uniform(math.log(L_lo), math.log(L_hi)))
        L = int(32 * round(Lf / 32))
        L = min(max(L, L_lo), L_hi)
        q = int(rng.choice(q_choices))
        t = float(rng.uniform(0.98, 1.02))
        spec.L.append(L)
        spec.q.append(q)
        spec.start.append(i & 1)
        spec.seed.append(1000 + i)
        spec.beta.append(beta_at(q, t))
    return spec


# --- served configuration ----------------------------------------------

@dataclass(frozen=True)
class Request:
    rid: int
    arrival_s: float
    L: int
    q: int
    beta: float
    nsweeps: int
    seed: int
    start: int = 1


def served(n: int = 10000, rate_hz: float = 200.0, harness_seed: int = 1,
           L_lo: int = 128, L_hi: int = 8192,
           q_choices=(6, 9, 15, 24, 96), sweeps_lo: int = 100,
           sweeps_hi: int = 5000) -> list:
    """Poisson request stream: exponential gaps of mean 1/rate, L
    log-uniform over [L_lo, L_hi] (multiple of 32), q from q_choices,
    T uniform in [0.97, 1.03] T_c, nsweeps uniform in [sweeps_lo,
    sweeps_hi], seed = request id, random start."""
    rng = np.random.default_rng(harness_seed)
    t = 0.0
    out = []
    for rid in range(n):
        t += float(rng.exponential(1.0 / rate_hz))
        Lf = math.exp(rng.uniform(math.log(L_lo), math.log(L_hi)))
        L = min(max(int(32 * round(Lf / 32)), L_lo), L_hi)
        q = int(rng.choice(q_choices))
        tt = float(rng.uniform(0.97, 1.03))
        ns = int(rng.integers(sweeps_lo, sweeps_hi + 1))
        out.append(Request(rid, t, L, q, beta_at(q, tt), ns, rid, 1))
    return out


def random_spins(L: int, q: int, seed: int) -> np.ndarray:
    """An L x L uint8 array of i.i.d. uniform states in 0..q-1."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, q, size=(L, L), dtype=np.uint8)
