"""The entry point that allocates nothing (potts_sweep_planes_noalloc).

It serves callers that must not allocate device memory where they sweep
(code inside a framework whose caching allocator already holds the device
memory, or loops that cannot afford the synchronisation an allocation may
cause): they own the planes and the output, and the library accumulates the
records in one fixed device array.  Its results must equal the CPU oracle's
and the allocating entry point's bit for bit, call after call, whether the
records go to host memory, to device memory or nowhere.  This file is
collected last so that a stop at the first failure has run every other test;
it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1101_0876_gb300 import potts, workloads

pytestmark = pytest.mark.gpu


def _to_planes(spins):
    """Row-major L x L spins -> (white, black) planes of L x L/2 bytes."""
    L = spins.shape[0]
    white = np.empty((L, L // 2), np.uint8)
    black = np.empty((L, L // 2), np.uint8)
    white[0::2] = spins[0::2, 0::2]
    white[1::2] = spins[1::2, 1::2]
    black[0::2] = spins[0::2, 1::2]
    black[1::2] = spins[1::2, 0::2]
    return white, black


def _from_planes(white, black):
    L = white.shape[0]
    s = np.empty((L, L), np.uint8)
    s[0::2, 0::2] = white[0::2]
    s[1::2, 1::2] = white[1::2]
    s[0::2, 1::2] = black[0::2]
    s[1::2, 0::2] = black[1::2]
    return s


def _call(dw, db, L, q, seed, t, beta, n, out_ptr, stream):
    """One call through the C ABI; out_ptr: host or device address, or None."""
    u64p = ctypes.POINTER(ctypes.c_uint64)
    out = ctypes.cast(ctypes.c_void_p(out_ptr), u64p) if out_ptr else None
    rc = potts.lib().potts_sweep_planes_noalloc(
        ctypes.c_void_p(dw.data_ptr()), ctypes.c_void_p(db.data_ptr()), L, q,
        seed, t, beta, n, out, ctypes.c_void_p(stream))
    assert rc == 0, potts.last_error()


@pytest.mark.parametrize("L,q,use_torch_stream", [(256, 9, False),
                                                  (544, 24, True),
                                                  (4096, 9, False)])
def test_noalloc_equals_oracle_and_allocating_path(L, q, use_torch_stream):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1101_0876_gb300 import build
    build.build()
    seed, beta = 21, workloads.beta_at(q, 1.0)
    ora = oracle.Lattice(L, q, 1, seed)           # the CPU reference
    ref = potts.Lattice(L, q, potts.START_RANDOM, seed)   # allocating path
    start = ora.spins()
    assert np.array_equal(ref.spins(), start)
    w, b = _to_planes(start)
    dw = torch.from_numpy(w).cuda()
    db = torch.from_numpy(b).cuda()
    stream = torch.cuda.Stream() if use_torch_stream else None
    handle = stream.cuda_stream if stream is not None else 0
    torch.cuda.synchronize()
    t = 0
    # two calls in a row with records in host memory
    for n in (7, 5):
        host = np.zeros((n, 1 + q), dtype=np.uint64)
        _call(dw, db, L, q, seed, t, beta, n, host.ctypes.data, handle)
        assert np.array_equal(host, ora.sweep(beta, n)), (t, n)
        assert np.array_equal(host, ref.sweep(beta, n)), (t, n)
        t += n
    # no records at all
    _call(dw, db, L, q, seed, t, beta, 3, None, handle)
    ora.sweep(beta, 3, records=False)
    ref.sweep(beta, 3, records=False)
    t += 3
    # records into device memory
    dev = torch.zeros((4, 1 + q), dtype=torch.int64, device="cuda")
    _call(dw, db, L, q, seed, t, beta, 4, dev.data_ptr(), handle)
    got = dev.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, ora.sweep(beta, 4))
    assert np.array_equal(got, ref.sweep(beta, 4))
    spins = _from_planes(dw.cpu().numpy(), db.cpu().numpy())
    assert np.array_equal(spins, ora.spins())
    assert np.array_equal(spins, ref.spins())


def test_noalloc_rejects_oversize_and_bad_planes():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    d = torch.zeros(2 * 64 * 32, dtype=torch.uint8, device="cuda")
    p = d.data_ptr()
    with pytest.raises(potts.PottsError) as ei:
        potts.sweep_planes_noalloc(p, p + 64 * 32, 64, 256, 1, 0, 1.0, 40)
    assert ei.value.code == potts.POTTS_EINVAL
    assert "8192" in potts.last_error()
    with pytest.raises(potts.PottsError):
        potts.sweep_planes_noalloc(p + 1, p + 64 * 32, 64, 9, 1, 0, 1.0, 1)
