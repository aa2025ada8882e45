"""Host-side analysis of the exact integer series the sweep emits.

Everything here works in FP64 on the per-sweep integer records
{B, hist[0..q-1]} (B = satisfied bonds, H = -B):

- e = H/N and the order parameter m (Sec. 2.1, Eq. 7, read as
  m = (q N_max/N - 1)/(q - 1), which is 1 when ordered and 0 when
  disordered; the printed q(N_max/N - 1)/(q - 1) is -1 when disordered);
- the energy cumulant V_L = 1 - <H^4>/(3 <H^2>^2) (Sec. 4, Eq. 9);
- the susceptibility chi = (N/T)(<m^2> - <m>^2) (Sec. 4, Eq. 11);
- the exact transition values e_o, e_d from the latent heat (Eq. 3) and
  e_d + e_o = -2(1 + 1/sqrt q) (Eq. 6), with the latent heat read as
  2(1 + 1/sqrt q) tanh(Theta/2) prod_n tanh^2(n Theta),
  Theta = arccosh(sqrt(q)/2) (the printed 1/sqrt 2 and arccos cannot hold
  for q > 4; this reading reproduces the table of Sec. 4 digit for digit);
- single-histogram (Ferrenberg-Swendsen) reweighting of a series taken at
  beta0 to a nearby beta1: the Boltzmann weight is exp(-beta H) =
  exp(beta B), so each sample gets weight exp((beta1 - beta0) B);
- the specific heat per spin C = beta^2 N (<e^2> - <e>^2);
- the printed large-q series of the magnetization jump (Eq. 8);
- batch-means error bars.
"""
from __future__ import annotations

import math

import numpy as np

from .workloads import tc  # noqa: F401  (re-exported)


def energy_magnetization(records: np.ndarray, L: int, q: int):
    """Per-record e = -B/N and m = (q N_max/N - 1)/(q - 1), in FP64."""
    rec = np.asarray(records)
    N = float(L) * float(L)
    e = -rec[:, 0].astype(np.float64) / N
    nmax = rec[:, 1:1 + q].max(axis=1).astype(np.float64)
    m = (q * nmax / N - 1.0) / (q - 1.0)
    return e, m


def cumulant_VL(records: np.ndarray) -> float:
    """V_L = 1 - <H^4> / (3 <H^2>^2) with H = -B."""
    H = -np.asarray(records)[:, 0].astype(np.float64)
    h2 = np.mean(H * H)
    h4 = np.mean(H ** 4)
    return 1.0 - h4 / (3.0 * h2 * h2)


def susceptibility(records: np.ndarray, L: int, q: int, T: float) -> float:
    """chi = (N/T) (<m^2> - <m>^2)."""
    _, m = energy_magnetization(records, L, q)
    N = float(L) * float(L)
    return N / T * (np.mean(m * m) - np.mean(m) ** 2)


def batch_means(x: np.ndarray, nbatch: int = 100):
    """Mean and its standard error from nbatch contiguous batch means."""
    x = np.asarray(x, dtype=np.float64)
    n = (x.size // nbatch) * nbatch
    b = x[:n].reshape(nbatch, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nbatch))


def latent_heat(q: int, nterms: int = 2000) -> float:
    """e_d - e_o for q > 4 (Eq. 3, corrected reading)."""
    if q <= 4:
        return 0.0
    theta = math.acosh(math.sqrt(q) / 2.0)
    prod = 1.0
    for n in range(1, nterms + 1):
        t = math.tanh(n * theta)
        prod *= t * t
        if 1.0 - t * t < 1e-18:
            break
    return 2.0 * (1.0 + 1.0 / math.sqrt(q)) * math.tanh(theta / 2.0) * prod


def exact_energies(q: int):
    """(e_o, e_d): ordered / disordered energy per spin at T_c (Eqs. 3, 6)."""
    s = -2.0 * (1.0 + 1.0 / math.sqrt(q))
    d = latent_heat(q)
    e_d = (s + d) / 2.0
    e_o = (s - d) / 2.0
    return e_o, e_d


def magnetization_jump_series(q: int, terms: int = 5) -> float:
    """The large-q expansion of the order-parameter jump at T_c (Sec. 2.1,
    Eq. 8), 1 - q^-1 - 3 q^-2 - 9 q^-3 - 27 q^-4 - ..., continued in its
    printed pattern (coefficient 3^k of q^-(k+1)) for `terms` subtracted
    terms.  With five terms it reproduces the "exact" Delta m column of the
    table of Sec. 4 digit for digit, so that column is this truncated
    series, not a closed form (its truncation error is about 3^5 q^-6:
    5e-4 for q = 9, 2e-2 for q = 6)."""
    return 1.0 - sum(3.0 ** k / float(q) ** (k + 1) for k in range(terms))


def reweight(records: np.ndarray, L: int, q: int, beta0: float,
             beta1: float):
    """<e>, <e^2>, <m>, <m^2> at beta1 from records sampled at beta0
    (single-histogram reweighting; log-sum-exp for stability)."""
    rec = np.asarray(records)
    B = rec[:, 0].astype(np.float64)
    lw = (beta1 - beta0) * B
    lw -= lw.max()
    w = np.exp(lw)
    w /= w.sum()
    e, m = energy_magnetization(rec, L, q)
    return (float(np.dot(w, e)), float(np.dot(w, e * e)),
            float(np.dot(w, m)), float(np.dot(w, m * m)))


def specific_heat(records: np.ndarray, L: int, q: int, beta: float) -> float:
    """C = beta^2 N (<e^2> - <e>^2) per spin."""
    e, _ = energy_magnetization(records, L, q)
    N = float(L) * float(L)
    return beta * beta * N * (np.mean(e * e) - np.mean(e) ** 2)
