"""Thin Python binding of libpotts (ctypes).  Argument marshalling only:
every step of the sweep runs in the library's CUDA kernels.  If the library
is missing the binding raises; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpotts.so")

POTTS_OK, POTTS_EINVAL, POTTS_ENOMEM, POTTS_ECUDA = 0, 1, 2, 3
POTTS_ETIMEOUT, POTTS_EBUSY, POTTS_ECANCELLED, POTTS_ENOTFOUND = 4, 5, 6, 7
START_ORDERED, START_RANDOM = 0, 1
LAYOUT_AUTO, LAYOUT_U8, LAYOUT_U4 = 0, 1, 2
UPDATE_METROPOLIS, UPDATE_HEATBATH = 0, 1
ADMIT_FIFO, ADMIT_SMALLEST = 0, 1
SCHEDULE_TWO_PASS, SCHEDULE_FUSED = 0, 1

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dblp = ctypes.POINTER(ctypes.c_double)


class PottsObs(ctypes.Structure):
    _fields_ = [("sweep", ctypes.c_uint64), ("bonds", ctypes.c_uint64),
                ("nmax", ctypes.c_uint64), ("e", ctypes.c_double),
                ("m", ctypes.c_double), ("nsamples", ctypes.c_uint64),
                ("sum_e", ctypes.c_double), ("sum_e2", ctypes.c_double),
                ("sum_e4", ctypes.c_double), ("sum_m", ctypes.c_double),
                ("sum_m2", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServeCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64),
                ("max_slots", ctypes.c_int32),
                ("sweeps_per_step", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32),
                ("policy", ctypes.c_int32)]


class Req(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("q", ctypes.c_int32),
                ("start", ctypes.c_int32), ("update", ctypes.c_int32),
                ("beta", ctypes.c_double), ("nsweeps", ctypes.c_int64),
                ("seed", ctypes.c_uint64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("steps", ctypes.c_uint64), ("sweeps_done", ctypes.c_uint64),
                ("updates_done", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_uint64),
                ("active", ctypes.c_int32), ("queued", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# name -> (restype, argtypes)
_SIGS = {
    "potts_last_error": (ctypes.c_char_p, []),
    "potts_version": (ctypes.c_int, []),
    "potts_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_void_p)]),
    "potts_create_ex": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_uint64,
                                       ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "potts_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double,
                                   ctypes.c_int64, _u64p]),
    "potts_set_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "potts_set_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "potts_batch_set_update": (ctypes.c_int, [
        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "potts_heatbath_weights": (ctypes.c_int, [
        ctypes.c_double, ctypes.c_int32, _u64p,
        ctypes.POINTER(ctypes.c_int32)]),
    "potts_observables": (ctypes.c_int, [ctypes.c_void_p,
                                         ctypes.POINTER(PottsObs)]),
    "potts_reset_averages": (ctypes.c_int, [ctypes.c_void_p]),
    "potts_get_spins": (ctypes.c_int, [ctypes.c_void_p, _u8p]),
    "potts_set_state": (ctypes.c_int, [ctypes.c_void_p, _u8p,
                                       ctypes.c_uint64]),
    "potts_threshold_table": (ctypes.c_int, [ctypes.c_double, _u64p]),
    "potts_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "potts_device_planes": (ctypes.c_int, [ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p),
                                           _i64p, _i32p]),
    "potts_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "potts_sweep_planes_noalloc": (ctypes.c_int, [
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int64,
        _u64p, ctypes.c_void_p]),
    "potts_create_sharded": (ctypes.c_int, [
        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
        ctypes.c_int32, ctypes.c_int32, _i32p,
        ctypes.POINTER(ctypes.c_void_p)]),
    "potts_strip_create": (ctypes.c_int, [
        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
        ctypes.POINTER(ctypes.c_void_p)]),
    "potts_strip_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_void_p),
                                        _i64p]),
    "potts_strip_pass": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double,
                                        ctypes.c_int32, ctypes.c_void_p]),
    "potts_batch_create": (ctypes.c_int, [ctypes.c_int32, _i32p, _i32p,
                                          _i32p, _u64p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "potts_batch_sweep": (ctypes.c_int, [ctypes.c_void_p, _dblp,
                                         ctypes.c_int64,
                                         ctypes.POINTER(_u64p)]),
    "potts_batch_get_spins": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                             _u8p]),
    "potts_batch_observables": (ctypes.c_int, [ctypes.c_void_p,
                                               ctypes.c_int32,
                                               ctypes.POINTER(PottsObs)]),
    "potts_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "potts_serve_start": (ctypes.c_int, [ctypes.POINTER(ServeCfg),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "potts_serve_submit": (ctypes.c_int, [ctypes.c_void_p,
                                          ctypes.POINTER(Req), _u64p]),
    "potts_serve_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                        _u64p, ctypes.c_int64, _i64p,
                                        ctypes.POINTER(ctypes.c_int)]),
    "potts_serve_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "potts_serve_stats_get": (ctypes.c_int, [ctypes.c_void_p,
                                             ctypes.POINTER(ServeStats)]),
    "potts_serve_stop": (ctypes.c_int, [ctypes.c_void_p]),
}

_lib = None


class PottsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libpotts error {code}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded library.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().potts_last_error().decode()


def check(rc: int) -> None:
    if rc != POTTS_OK:
        raise PottsError(rc, last_error())


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def heatbath_weights(beta: float, q: int):
    """(W[0..4], m) of the heat-bath rule for beta and q."""
    W = np.zeros(5, dtype=np.uint64)
    m = ctypes.c_int32()
    check(lib().potts_heatbath_weights(float(beta), int(q),
                                       _ptr(W, ctypes.c_uint64),
                                       ctypes.byref(m)))
    return W, int(m.value)


def threshold_table(beta: float) -> np.ndarray:
    out = np.zeros(5, dtype=np.uint64)
    check(lib().potts_threshold_table(float(beta), _ptr(out, ctypes.c_uint64)))
    return out


def sweep_planes_noalloc(white_ptr: int, black_ptr: int, L: int, q: int,
                         seed: int, sweep: int, beta: float, nsweeps: int,
                         out: np.ndarray | None = None,
                         stream: int | None = None):
    """Sweeps caller-owned device planes without any allocation in the
    library (potts_sweep_planes_noalloc).  Returns the (nsweeps, 1+q)
    records, in `out` if given."""
    if out is None:
        out = np.empty((int(nsweeps), 1 + int(q)), dtype=np.uint64)
    assert out.dtype == np.uint64 and out.flags.c_contiguous
    check(lib().potts_sweep_planes_noalloc(
        ctypes.c_void_p(white_ptr), ctypes.c_void_p(black_ptr), int(L),
        int(q), int(seed), int(sweep), float(beta), int(nsweeps),
        _ptr(out, ctypes.c_uint64), ctypes.c_void_p(stream or None)))
    return out


class Lattice:
    """One L x L lattice with q states resident on the current GPU."""

    def __init__(self, L: int, q: int, start: int = START_ORDERED,
                 seed: int = 0, layout: int = LAYOUT_AUTO,
                 nstrips: int = 0, devices=None):
        """nstrips > 0: the lattice split into that many row strips
        (potts_create_sharded), strip s on devices[s] (default: the current
        device for all)."""
        self.L, self.q, self.seed = int(L), int(q), int(seed)
        h = ctypes.c_void_p()
        if nstrips:
            dev = None
            if devices is not None:
                devs = np.ascontiguousarray(devices, dtype=np.int32)
                assert devs.size == int(nstrips)
                dev = _ptr(devs, ctypes.c_int32)
            check(lib().potts_create_sharded(
                self.L, self.q, int(start), self.seed, int(layout),
                int(nstrips), dev, ctypes.byref(h)))
        else:
            check(lib().potts_create_ex(self.L, self.q, int(start),
                                        self.seed, int(layout),
                                        ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            check(lib().potts_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sweep(self, beta: float, nsweeps: int, out: np.ndarray | None = None,
              records: bool = True):
        """Runs nsweeps sweeps.  Returns the (nsweeps, 1+q) uint64 records
        {B, hist} (into `out` if given), or None with records=False."""
        if out is None and records:
            out = np.empty((int(nsweeps), 1 + self.q), dtype=np.uint64)
        if out is not None:
            assert out.dtype == np.uint64 and out.flags.c_contiguous
            assert out.size >= int(nsweeps) * (1 + self.q)
            p = _ptr(out, ctypes.c_uint64)
        else:
            p = ctypes.POINTER(ctypes.c_uint64)()
        check(lib().potts_sweep(self._h, float(beta), int(nsweeps), p))
        return out

    def set_update(self, update: int) -> None:
        """UPDATE_METROPOLIS (default) or UPDATE_HEATBATH for later
        sweeps."""
        check(lib().potts_set_update(self._h, int(update)))

    def set_schedule(self, schedule: int) -> None:
        """SCHEDULE_TWO_PASS (default) or SCHEDULE_FUSED (one kernel per
        Metropolis sweep; U8 layout, L a multiple of 1024) for later
        sweeps."""
        check(lib().potts_set_schedule(self._h, int(schedule)))

    def observables(self) -> dict:
        o = PottsObs()
        check(lib().potts_observables(self._h, ctypes.byref(o)))
        return o.as_dict()

    def reset_averages(self) -> None:
        check(lib().potts_reset_averages(self._h))

    def spins(self, out: np.ndarray | None = None) -> np.ndarray:
        """Row-major L x L spins; into `out` (C-contiguous uint8, e.g. a
        pinned buffer) when given."""
        if out is None:
            out = np.empty((self.L, self.L), dtype=np.uint8)
        assert out.dtype == np.uint8 and out.flags.c_contiguous
        assert out.size == self.L * self.L
        check(lib().potts_get_spins(self._h, _ptr(out, ctypes.c_uint8)))
        return out

    def set_state(self, spins: np.ndarray, sweep: int) -> None:
        s = np.ascontiguousarray(spins, dtype=np.uint8)
        assert s.shape == (self.L, self.L)
        check(lib().potts_set_state(self._h, _ptr(s, ctypes.c_uint8),
                                    int(sweep)))

    def set_stream(self, stream_handle: int | None) -> None:
        check(lib().potts_set_stream(self._h, ctypes.c_void_p(
            stream_handle or None)))

    def device_planes(self):
        w, b = ctypes.c_void_p(), ctypes.c_void_p()
        rb, lay = ctypes.c_int64(), ctypes.c_int32()
        check(lib().potts_device_planes(self._h, ctypes.byref(w),
                                        ctypes.byref(b), ctypes.byref(rb),
                                        ctypes.byref(lay)))
        return w.value, b.value, rb.value, lay.value

    @property
    def sweep_index(self) -> int:
        return int(self.observables()["sweep"])


class Strip:
    """One row strip of an L x L lattice on the current GPU: lattice rows
    [row0, row0 + nrows) of both colour planes plus one halo row above and
    below (potts_strip_create).  The caller moves the halo rows between
    strips (rows()) and sums the partial records of the strips."""

    def __init__(self, L: int, q: int, start: int, seed: int, row0: int,
                 nrows: int, layout: int = LAYOUT_AUTO):
        self.L, self.q, self.seed = int(L), int(q), int(seed)
        self.row0, self.nrows = int(row0), int(nrows)
        h = ctypes.c_void_p()
        check(lib().potts_strip_create(self.L, self.q, int(start), self.seed,
                                       int(layout), self.row0, self.nrows,
                                       ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            check(lib().potts_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rows(self, colour: int):
        """(first own, last own, halo above, halo below) device addresses of
        plane `colour`, and the bytes per row."""
        arr = (ctypes.c_void_p * 4)()
        rb = ctypes.c_int64()
        check(lib().potts_strip_rows(self._h, int(colour), arr,
                                     ctypes.byref(rb)))
        return tuple(int(a or 0) for a in arr), int(rb.value)

    def pass_(self, beta: float, colour: int, d_record: int) -> None:
        """Queues the colour pass on the strip's stream; its partial counts
        are added to the 1 + q uint64 at device address d_record."""
        check(lib().potts_strip_pass(self._h, float(beta), int(colour),
                                     ctypes.c_void_p(d_record)))

    def set_stream(self, stream_handle: int | None) -> None:
        check(lib().potts_set_stream(self._h, ctypes.c_void_p(
            stream_handle or None)))

    def set_update(self, update: int) -> None:
        check(lib().potts_set_update(self._h, int(update)))

    def spins(self, out: np.ndarray | None = None) -> np.ndarray:
        """The strip's own rows, nrows x L row-major."""
        if out is None:
            out = np.empty((self.nrows, self.L), dtype=np.uint8)
        assert out.dtype == np.uint8 and out.flags.c_contiguous
        assert out.size == self.nrows * self.L
        check(lib().potts_get_spins(self._h, _ptr(out, ctypes.c_uint8)))
        return out

    def set_state(self, rows: np.ndarray, sweep: int) -> None:
        s = np.ascontiguousarray(rows, dtype=np.uint8)
        assert s.shape == (self.nrows, self.L)
        check(lib().potts_set_state(self._h, _ptr(s, ctypes.c_uint8),
                                    int(sweep)))


class Batch:
    """n independent lattices swept together (one launch per colour pass)."""

    def __init__(self, L, q, start, seed):
        self.n = len(L)
        self.L = [int(x) for x in L]
        self.q = [int(x) for x in q]
        a_L = np.ascontiguousarray(L, dtype=np.int32)
        a_q = np.ascontiguousarray(q, dtype=np.int32)
        a_s = np.ascontiguousarray(start, dtype=np.int32)
        a_seed = np.ascontiguousarray(seed, dtype=np.uint64)
        h = ctypes.c_void_p()
        check(lib().potts_batch_create(self.n, _ptr(a_L, ctypes.c_int32),
                                       _ptr(a_q, ctypes.c_int32),
                                       _ptr(a_s, ctypes.c_int32),
                                       _ptr(a_seed, ctypes.c_uint64),
                                       ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            check(lib().potts_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, beta, nsweeps: int, records: bool = True):
        b = np.ascontiguousarray(beta, dtype=np.float64)
        assert b.size == self.n
        outs = None
        if records:
            outs = [np.empty((int(nsweeps), 1 + q), dtype=np.uint64)
                    for q in self.q]
            arr = (_u64p * self.n)(*[_ptr(o, ctypes.c_uint64) for o in outs])
            parr = ctypes.cast(arr, ctypes.POINTER(_u64p))
        else:
            parr = ctypes.POINTER(_u64p)()
        check(lib().potts_batch_sweep(self._h, _ptr(b, ctypes.c_double),
                                      int(nsweeps), parr))
        return outs

    def set_update(self, update) -> None:
        """Per-lattice rule (UPDATE_METROPOLIS / UPDATE_HEATBATH) for
        later sweeps."""
        u = np.ascontiguousarray(update, dtype=np.int32)
        assert u.size == self.n
        check(lib().potts_batch_set_update(self._h, _ptr(u, ctypes.c_int32)))

    def spins(self, i: int) -> np.ndarray:
        out = np.empty((self.L[i], self.L[i]), dtype=np.uint8)
        check(lib().potts_batch_get_spins(self._h, int(i),
                                          _ptr(out, ctypes.c_uint8)))
        return out

    def observables(self, i: int) -> dict:
        o = PottsObs()
        check(lib().potts_batch_observables(self._h, int(i), ctypes.byref(o)))
        return o.as_dict()


class Server:
    """Continuous-batching request loop running on a library host thread."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int,
                 sweeps_per_step: int, queue_capacity: int = 0,
                 policy: int = ADMIT_FIFO):
        cfg = ServeCfg(int(hbm_budget_bytes), int(max_slots),
                       int(sweeps_per_step), int(queue_capacity), int(policy))
        h = ctypes.c_void_p()
        check(lib().potts_serve_start(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._q = {}

    def submit(self, L, q, beta, nsweeps, seed, start=START_RANDOM,
               update=UPDATE_METROPOLIS) -> int:
        r = Req(int(L), int(q), int(start), int(update), float(beta),
                int(nsweeps), int(seed))
        rid = ctypes.c_uint64()
        check(lib().potts_serve_submit(self._h, ctypes.byref(r),
                                       ctypes.byref(rid)))
        self._q[rid.value] = int(q)
        return rid.value

    def try_submit(self, *a, **k):
        """submit() that returns None instead of raising on EBUSY."""
        try:
            return self.submit(*a, **k)
        except PottsError as e:
            if e.code == POTTS_EBUSY:
                return None
            raise

    def poll(self, rid: int, max_sweeps: int = 4096, out=None):
        """Returns (records array (n, 1+q), done).  Raises PottsError for a
        cancelled, failed or unknown request.  `out` (uint64, C-contiguous,
        at least max_sweeps * (1+q) values) is reused if given."""
        q = self._q.get(rid)
        n = ctypes.c_int64()
        done = ctypes.c_int()
        if q is None:
            check(lib().potts_serve_poll(self._h, int(rid),
                                         ctypes.POINTER(ctypes.c_uint64)(), 0,
                                         ctypes.byref(n), ctypes.byref(done)))
            return np.empty((0, 0), dtype=np.uint64), bool(done.value)
        if out is None:
            out = np.empty((int(max_sweeps), 1 + q), dtype=np.uint64)
        else:
            assert out.dtype == np.uint64 and out.flags.c_contiguous
            assert out.size >= int(max_sweeps) * (1 + q)
            out = out.reshape(-1)[:int(max_sweeps) * (1 + q)].reshape(
                int(max_sweeps), 1 + q)
        rc = lib().potts_serve_poll(self._h, int(rid),
                                    _ptr(out, ctypes.c_uint64),
                                    int(max_sweeps), ctypes.byref(n),
                                    ctypes.byref(done))
        if done.value:
            self._q.pop(rid, None)
        check(rc)
        return out[:n.value], bool(done.value)

    def cancel(self, rid: int) -> None:
        check(lib().potts_serve_cancel(self._h, int(rid)))

    def stats(self) -> dict:
        s = ServeStats()
        check(lib().potts_serve_stats_get(self._h, ctypes.byref(s)))
        return s.as_dict()

    def stop(self):
        if getattr(self, "_h", None) and self._h.value:
            check(lib().potts_serve_stop(self._h))
            self._h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
