"""The entry point that allocates nothing (potts_sweep_planes_noalloc).

It serves callers that cannot allocate device memory when they sweep (code
running during CUDA graph capture, or inside a framework whose allocator
already holds the memory): they own the planes and the output, and the
library accumulates records in a fixed device array.  Its results must
equal the allocating entry point's bit for bit, call after call.  This file
is collected last so that a stop at the first failure has run every other
test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("L,q,use_torch_stream", [(256, 9, False),
                                                  (544, 24, True)])
def test_noalloc_equals_allocating_path(L, q, use_torch_stream):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1101_0876_gb300 import build
    build.build()
    seed, beta = 21, workloads.beta_at(q, 1.0)
    ref = potts.Lattice(L, q, potts.START_RANDOM, seed)
    w, b = _to_planes(ref.spins())
    dw = torch.from_numpy(w).cuda()
    db = torch.from_numpy(b).cuda()
    stream = torch.cuda.Stream() if use_torch_stream else None
    handle = stream.cuda_stream if stream is not None else None
    torch.cuda.synchronize()
    t = 0
    for n in (7, 5):              # two calls in a row share the fixed buffer
        got = potts.sweep_planes_noalloc(dw.data_ptr(), db.data_ptr(), L, q,
                                         seed, t, beta, n, stream=handle)
        want = ref.sweep(beta, n)
        assert np.array_equal(got, want), n
        t += n
    spins = _from_planes(dw.cpu().numpy(), db.cpu().numpy())
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
