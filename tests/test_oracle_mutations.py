"""The pins have teeth: plausible mistakes planted in a copy of the oracle
(CPU only) make at least one pin fail.

Each case rewrites one spot of oracle/potts_oracle.c in a temporary copy,
builds it, and runs the pin meant to catch it: PyTorch's Philox engine for
the generator and its counter layout, exact enumeration for the Metropolis
rule and the threshold table, the incremental-vs-recount check for the
bookkeeping, the colour-independence check for the random start, and for
the heat bath its conditional-Boltzmann outcome distribution and the recount.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1101_0876_gb300.analysis import batch_means

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "potts_oracle.c")

MUTATIONS = {
    # name: (original text, planted text, pin)
    "philox_multiplier": ("#define PHILOX_M0 0xD2511F53u",
                          "#define PHILOX_M0 0xD2511F52u", "philox"),
    "philox_key_bump": ("      k1 += PHILOX_W1;", "      k1 += PHILOX_W0;",
                        "philox"),
    "counter_words_swapped": ("  ctr[1] = (uint32_t)sweep;\n  ctr[2] = domain;",
                              "  ctr[1] = domain;\n  ctr[2] = (uint32_t)sweep;",
                              "site_word"),
    "site_word_index": ("  return out[k & 3u];", "  return out[(k + 1) & 3u];",
                        "site_word"),
    "dE_sign": ("  int dE = n_old - n_new;", "  int dE = n_new - n_old;",
                "enumeration"),
    "dropped_neighbour": ("  for (int n = 0; n < 4; ++n) {",
                          "  for (int n = 0; n < 3; ++n) {", "enumeration"),
    "threshold_half_beta": ("    double p = exp(-beta * (double)d);",
                            "    double p = exp(-0.5 * beta * (double)d);",
                            "enumeration"),
    # (dE < 0 in place of dE <= 0 is an equivalent mutant: thr[0] = 2^32)
    "proposal_misses_a_state": ("  uint64_t prod = (uint64_t)u * (uint64_t)q;",
                                "  uint64_t prod = (uint64_t)u * (uint64_t)(q - 1);",
                                "enumeration"),
    "right_neighbour_is_left": (
        "  nb[3] = s[(int64_t)i * L + wrap(j + 1, L)];",
        "  nb[3] = s[(int64_t)i * L + wrap(j - 1, L)];", "enumeration"),
    "bond_bookkeeping": ("        lat->B = (uint64_t)((int64_t)lat->B + dB);",
                         "        lat->B = (uint64_t)((int64_t)lat->B - dB);",
                         "recount"),
    "random_start_domain": ("oracle_site_word(seed, 0, 2u + (uint32_t)c,",
                            "oracle_site_word(seed, 0, 2u,", "random_start"),
    # heat bath
    "hb_weights_half_beta": (
        "      double x = ldexp(exp(beta * (double)n), m);",
        "      double x = ldexp(exp(0.5 * beta * (double)n), m);",
        "hb_distribution"),
    "hb_excess_includes_base": (
        "    const uint64_t excess = W[cnt[b]] - W[0];",
        "    const uint64_t excess = W[cnt[b]];", "hb_distribution"),
    "hb_normaliser_misses_held_bases": (
        "  uint64_t Z = (uint64_t)q * W[0];",
        "  uint64_t Z = (uint64_t)(q - k) * W[0];", "hb_distribution"),
    "hb_dB_sign": ("  *dB = n_now - n_old;", "  *dB = n_old - n_now;",
                   "hb_recount"),
}


def _build(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, name
    src = tmp_path / f"{name}.c"
    src.write_text(text.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-I",
                    os.path.join(ROOT, "oracle"), "-o", str(so), str(src),
                    "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    P32 = ctypes.POINTER(ctypes.c_uint32)
    P64 = ctypes.POINTER(ctypes.c_uint64)
    lib.oracle_philox4x32_10.argtypes = [P32, P32, P32]
    lib.oracle_site_word.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_uint64]
    lib.oracle_site_word.restype = ctypes.c_uint32
    lib.oracle_create.argtypes = [ctypes.c_int32] * 3 + [ctypes.c_uint64]
    lib.oracle_create.restype = ctypes.c_void_p
    lib.oracle_destroy.argtypes = [ctypes.c_void_p]
    lib.oracle_sweep.argtypes = [ctypes.c_void_p, ctypes.c_double,
                                 ctypes.c_int64, P64, ctypes.c_int32,
                                 ctypes.c_int32]
    lib.oracle_get_spins.argtypes = [ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_uint8)]
    lib.oracle_sweep_ex.argtypes = [ctypes.c_void_p, ctypes.c_double,
                                    ctypes.c_int64, P64, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32]
    lib.oracle_sweep_sites_ex.argtypes = [
        ctypes.POINTER(ctypes.c_uint8), ctypes.c_int32, ctypes.c_int32,
        ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int64,
        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint8),
        ctypes.c_int32]
    return lib


def _philox_pin(lib, torch_philox):
    rng = np.random.default_rng(1)
    c = rng.integers(0, 2**32, (64, 4), dtype=np.uint64).astype(np.uint32)
    k = rng.integers(0, 2**32, (64, 2), dtype=np.uint64).astype(np.uint32)
    ref = torch_philox(c, k)
    P32 = ctypes.POINTER(ctypes.c_uint32)
    for i in range(64):
        out = np.zeros(4, np.uint32)
        ci, ki = np.ascontiguousarray(c[i]), np.ascontiguousarray(k[i])
        lib.oracle_philox4x32_10(ci.ctypes.data_as(P32), ki.ctypes.data_as(P32),
                                 out.ctypes.data_as(P32))
        if not np.array_equal(out, ref[i]):
            return False
    return True


def _site_word_pin(lib, torch_philox):
    for seed, sweep, dom, kk in [(1, 7, 1, 5), (2**40 + 3, 9, 0, 123457)]:
        ctr = np.array([[kk >> 2, sweep & 0xFFFFFFFF, dom, sweep >> 32]],
                       dtype=np.uint64).astype(np.uint32)
        key = np.array([[seed & 0xFFFFFFFF, seed >> 32]],
                       dtype=np.uint64).astype(np.uint32)
        if lib.oracle_site_word(seed, sweep, dom, kk) != int(
                torch_philox(ctr, key)[0, kk & 3]):
            return False
    return True


def _enumeration_pin(lib, brute_force):
    L, q, beta = 3, 3, 1.0
    h = lib.oracle_create(L, q, 1, 77)
    lib.oracle_sweep(h, beta, 2000, ctypes.POINTER(ctypes.c_uint64)(), 0, 0)
    n = 200_000
    rec = np.zeros((n, 1 + q), np.uint64)
    lib.oracle_sweep(h, beta, n, rec.ctypes.data_as(
        ctypes.POINTER(ctypes.c_uint64)), 0, 0)
    lib.oracle_destroy(h)
    e = -rec[:, 0].astype(np.float64) / (L * L)
    mean, err = batch_means(e, 200)
    return abs(mean - brute_force(L, q, beta)[0]) < 4 * err


def _recount_pin(lib):
    h = lib.oracle_create(12, 5, 1, 3)
    rc = lib.oracle_sweep(h, 0.8, 50, ctypes.POINTER(ctypes.c_uint64)(), 0, 1)
    lib.oracle_destroy(h)
    return rc == 0


def _random_start_pin(lib):
    L = 128
    h = lib.oracle_create(L, 15, 1, 11)
    s = np.zeros((L, L), np.uint8)
    lib.oracle_get_spins(h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    lib.oracle_destroy(h)
    par = np.add.outer(np.arange(L), np.arange(L)) % 2
    return np.mean(s[par == 0] == s[par == 1]) < 0.2


def _hb_distribution_pin(lib):
    """Heat-bath outcomes of white sites whose neighbours are (0, 0, 1, 1)
    against exp(beta n_x) / sum_y exp(beta n_y)."""
    L, q, beta = 16, 5, 1.3
    pre = np.zeros((L, L), np.uint8)
    pre[1::2, 0::2] = 0       # up/down neighbours of white (even, even) sites
    pre[0::2, 1::2] = 1       # left/right neighbours
    ii, jj = np.meshgrid(np.arange(0, L, 2), np.arange(0, L, 2), indexing="ij")
    idx = (ii * L + jj).ravel().astype(np.int64)
    c = np.zeros(q, np.int64)
    out = np.zeros(idx.size, np.uint8)
    for t in range(200):
        rc = lib.oracle_sweep_sites_ex(
            pre.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), L, q, 3, t,
            beta, idx.size, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), 1)
        assert rc == 0
        c += np.bincount(out, minlength=q)[:q]
    p = np.exp(beta * np.array([2, 2, 0, 0, 0.0]))
    p /= p.sum()
    n = c.sum()
    return float(((c - n * p) ** 2 / (n * p)).sum()) < 3 * (q - 1) + 25


def _hb_recount_pin(lib):
    h = lib.oracle_create(12, 5, 1, 3)
    rc = lib.oracle_sweep_ex(h, 0.8, 40, ctypes.POINTER(ctypes.c_uint64)(),
                             0, 1, 1)
    lib.oracle_destroy(h)
    return rc == 0


def test_unmutated_copy_passes_every_pin(tmp_path, torch_philox, brute_force):
    lib = _build(tmp_path, "clean", "#define PHILOX_M0",
                 "#define PHILOX_M0")
    assert _philox_pin(lib, torch_philox)
    assert _site_word_pin(lib, torch_philox)
    assert _enumeration_pin(lib, brute_force)
    assert _recount_pin(lib)
    assert _random_start_pin(lib)
    assert _hb_distribution_pin(lib)
    assert _hb_recount_pin(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, torch_philox, brute_force, name):
    old, new, pin = MUTATIONS[name]
    lib = _build(tmp_path, name, old, new)
    passed = {
        "philox": lambda: _philox_pin(lib, torch_philox),
        "site_word": lambda: _site_word_pin(lib, torch_philox),
        "enumeration": lambda: _enumeration_pin(lib, brute_force),
        "recount": lambda: _recount_pin(lib),
        "random_start": lambda: _random_start_pin(lib),
        "hb_distribution": lambda: _hb_distribution_pin(lib),
        "hb_recount": lambda: _hb_recount_pin(lib),
    }[pin]()
    assert not passed, f"pin '{pin}' did not catch mutation '{name}'"
