"""Serial CPU oracle for the checkerboard Metropolis sweep of the 2D q-state
Potts model (Ferrero et al., Sec. 2.1, Sec. 3, Sec. 3.3-3.4, Sec. 5), and of
the heat-bath variant (one of the single-flip algorithms Sec. 6 proposes).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may load
this package.  The product path (the CUDA library and its Python binding)
never imports it, and it imports nothing from the product.

The arithmetic lives in ``potts_oracle.c`` (plain C, serial); this module
only compiles it (``build()``) and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "potts_oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_philox4x32_10.restype = None
        L.oracle_site_word.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_uint64]
        L.oracle_site_word.restype = ctypes.c_uint32
        L.oracle_thresholds.argtypes = [ctypes.c_double, u64p]
        L.oracle_thresholds.restype = ctypes.c_int
        L.oracle_recount.argtypes = [u8p, ctypes.c_int32, ctypes.c_int32,
                                     u64p, u64p]
        L.oracle_recount.restype = None
        L.oracle_create.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_uint64]
        L.oracle_create.restype = ctypes.c_void_p
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_destroy.restype = None
        L.oracle_sweep.argtypes = [ctypes.c_void_p, ctypes.c_double,
                                   ctypes.c_int64, u64p, ctypes.c_int32,
                                   ctypes.c_int32]
        L.oracle_sweep.restype = ctypes.c_int
        L.oracle_get_spins.argtypes = [ctypes.c_void_p, u8p]
        L.oracle_get_spins.restype = None
        L.oracle_set_state.argtypes = [ctypes.c_void_p, u8p, ctypes.c_uint64]
        L.oracle_set_state.restype = ctypes.c_int
        L.oracle_sweep_index.argtypes = [ctypes.c_void_p]
        L.oracle_sweep_index.restype = ctypes.c_uint64
        L.oracle_counts.argtypes = [ctypes.c_void_p, u64p, u64p]
        L.oracle_counts.restype = None
        L.oracle_sweep_sites.argtypes = [u8p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_double, ctypes.c_int64,
                                         i64p, u8p]
        L.oracle_sweep_sites.restype = ctypes.c_int
        L.oracle_init_sites.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.c_int64, i64p, u8p]
        L.oracle_init_sites.restype = ctypes.c_int
        L.oracle_heatbath_weights.argtypes = [
            ctypes.c_double, ctypes.c_int32, u64p,
            ctypes.POINTER(ctypes.c_int32)]
        L.oracle_heatbath_weights.restype = ctypes.c_int
        L.oracle_sweep_ex.argtypes = [ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_int64, u64p, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32]
        L.oracle_sweep_ex.restype = ctypes.c_int
        L.oracle_sweep_sites_ex.argtypes = [
            u8p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
            ctypes.c_uint64, ctypes.c_double, ctypes.c_int64, i64p, u8p,
            ctypes.c_int32]
        L.oracle_sweep_sites_ex.restype = ctypes.c_int
        L.oracle_band_pass.argtypes = [u8p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_int32, u64p]
        L.oracle_band_pass.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x u32) under one key (2 x u32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32),
                               _ptr(k, ctypes.c_uint32),
                               _ptr(out, ctypes.c_uint32))
    return out


def site_word(seed: int, sweep: int, domain: int, k: int) -> int:
    return int(lib().oracle_site_word(seed, sweep, domain, k))


def thresholds(beta: float) -> np.ndarray:
    out = np.zeros(5, dtype=np.uint64)
    rc = lib().oracle_thresholds(float(beta), _ptr(out, ctypes.c_uint64))
    if rc != 0:
        raise ValueError(f"invalid beta {beta!r}")
    return out


METROPOLIS, HEATBATH = 0, 1


def heatbath_weights(beta: float, q: int):
    """(W[0..4], m) of the heat-bath rule; ValueError when beta is out of
    range."""
    W = np.zeros(5, dtype=np.uint64)
    m = ctypes.c_int32()
    rc = lib().oracle_heatbath_weights(float(beta), int(q),
                                       _ptr(W, ctypes.c_uint64),
                                       ctypes.byref(m))
    if rc != 0:
        raise ValueError(f"no heat-bath weights for beta={beta!r}, q={q}")
    return W, int(m.value)


def recount(spins: np.ndarray, q: int):
    """(B, hist) of an L x L row-major uint8 lattice, from the definition."""
    s = np.ascontiguousarray(spins, dtype=np.uint8)
    L = s.shape[0]
    assert s.shape == (L, L)
    B = np.zeros(1, dtype=np.uint64)
    hist = np.zeros(q, dtype=np.uint64)
    lib().oracle_recount(_ptr(s, ctypes.c_uint8), L, q,
                         _ptr(B, ctypes.c_uint64), _ptr(hist, ctypes.c_uint64))
    return int(B[0]), hist


def sweep_sites(pre: np.ndarray, q: int, seed: int, sweep: int, beta: float,
                idx: np.ndarray, update: int = METROPOLIS) -> np.ndarray:
    """Values after sweep `sweep` of the sites idx (= i*L + j), computed one
    by one from the pre-sweep lattice `pre`."""
    s = np.ascontiguousarray(pre, dtype=np.uint8)
    L = s.shape[0]
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(ix.size, dtype=np.uint8)
    rc = lib().oracle_sweep_sites_ex(_ptr(s, ctypes.c_uint8), L, q, seed,
                                     sweep, float(beta), ix.size,
                                     _ptr(ix, ctypes.c_int64),
                                     _ptr(out, ctypes.c_uint8), int(update))
    if rc != 0:
        raise ValueError("oracle_sweep_sites: bad arguments")
    return out


def init_sites(L: int, q: int, start: int, seed: int,
               idx: np.ndarray) -> np.ndarray:
    """Initial spins of the sites idx (= i*L + j)."""
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(ix.size, dtype=np.uint8)
    rc = lib().oracle_init_sites(L, q, start, seed, ix.size,
                                 _ptr(ix, ctypes.c_int64),
                                 _ptr(out, ctypes.c_uint8))
    if rc != 0:
        raise ValueError("oracle_init_sites: bad arguments")
    return out


def band_pass(rows: np.ndarray, L: int, q: int, r0: int, seed: int,
              sweep: int, colour: int, beta: float, partial: np.ndarray,
              update: int = METROPOLIS) -> None:
    """One colour pass over the band held in `rows` ((n + 2) x L bytes, the
    first and last rows being the rows just above and below the band; the
    band is global rows r0 .. r0 + n - 1), updated in place; the band's
    partial record {B (black pass), hist} is added to `partial`."""
    assert rows.dtype == np.uint8 and rows.flags.c_contiguous
    assert rows.shape[1] == L and rows.shape[0] >= 3
    assert partial.dtype == np.uint64 and partial.size == 1 + q
    rc = lib().oracle_band_pass(_ptr(rows, ctypes.c_uint8), rows.shape[0] - 2,
                                L, q, r0, seed, sweep, colour, float(beta),
                                int(update), _ptr(partial, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("oracle_band_pass: bad arguments")


class Lattice:
    """One oracle lattice: L x L, q states, ordered (0) or random (1) start."""

    def __init__(self, L: int, q: int, start: int, seed: int):
        self.L, self.q, self.seed = int(L), int(q), int(seed)
        self._h = lib().oracle_create(L, q, start, seed)
        if not self._h:
            raise ValueError(f"oracle_create({L}, {q}, {start}) failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_destroy(h)
            self._h = None

    def sweep(self, beta: float, nsweeps: int, order: int = 0,
              check: bool = False, records: bool = True,
              update: int = METROPOLIS):
        out = (np.zeros((nsweeps, 1 + self.q), dtype=np.uint64)
               if records else None)
        ptr = (_ptr(out, ctypes.c_uint64) if records
               else ctypes.POINTER(ctypes.c_uint64)())
        rc = lib().oracle_sweep_ex(self._h, float(beta), int(nsweeps), ptr,
                                   order, 1 if check else 0, int(update))
        if rc == -2:
            raise AssertionError("incremental counts differ from a recount")
        if rc != 0:
            raise ValueError("oracle_sweep: bad arguments")
        return out

    def spins(self) -> np.ndarray:
        out = np.zeros((self.L, self.L), dtype=np.uint8)
        lib().oracle_get_spins(self._h, _ptr(out, ctypes.c_uint8))
        return out

    def set_state(self, spins: np.ndarray, sweep: int) -> None:
        s = np.ascontiguousarray(spins, dtype=np.uint8)
        assert s.shape == (self.L, self.L)
        if lib().oracle_set_state(self._h, _ptr(s, ctypes.c_uint8), sweep):
            raise ValueError("spin value out of range")

    @property
    def sweep_index(self) -> int:
        return int(lib().oracle_sweep_index(self._h))

    def counts(self):
        B = np.zeros(1, dtype=np.uint64)
        hist = np.zeros(self.q, dtype=np.uint64)
        lib().oracle_counts(self._h, _ptr(B, ctypes.c_uint64),
                            _ptr(hist, ctypes.c_uint64))
        return int(B[0]), hist


def observables(records: np.ndarray, L: int, q: int):
    """e = -B/N and m = (q N_max / N - 1)/(q - 1) per record (Sec. 2.1:
    e = <H>/N with H = -B; the order parameter of Eq. 7 read so that it is
    1 when ordered and 0 when disordered)."""
    N = float(L) * float(L)
    rec = np.asarray(records, dtype=np.float64)
    e = -rec[:, 0] / N
    nmax = rec[:, 1:].max(axis=1)
    m = (q * nmax / N - 1.0) / (q - 1.0)
    return e, m
