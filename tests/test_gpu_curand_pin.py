"""Pin of the oracle's generator against NVIDIA's cuRAND (needs a GPU).

cuRAND's device-side Philox4_32_10 is an implementation of the SC'11
generator independent of the oracle's C code; with its seed, subsequence and
offset set from (seed, sweep, colour, site) it yields the counter layout the
method uses (word k & 3 of Philox((k >> 2, sweep_lo, colour, sweep_hi),
(seed_lo, seed_hi))), so every site word of the oracle must equal it.  The
sample covers full 64-bit seeds and sweep indices, both colours and the
random-start domains, and site indices up to 2^31.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from conftest import BUILD, HERE, _compile

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def curand_ref():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    src = os.path.join(HERE, "curand_philox_ref.cu")
    return _compile(src, "curand_philox_ref",
                    ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a",
                     "-O2"])


def test_oracle_site_words_equal_curand(curand_ref, tmp_path):
    rng = np.random.default_rng(20260)
    n = 20000
    seed = rng.integers(0, 2**63, size=n, dtype=np.uint64) * 2 + \
        rng.integers(0, 2, size=n, dtype=np.uint64)
    sweep = np.where(rng.random(n) < 0.5,
                     rng.integers(0, 5000, size=n, dtype=np.uint64),
                     rng.integers(0, 2**63, size=n, dtype=np.uint64))
    dom = rng.integers(0, 4, size=n, dtype=np.uint64)
    k = rng.integers(0, 2**31, size=n, dtype=np.uint64)
    seed[:4] = [0, 2**64 - 1, 11, 1]
    sweep[:4] = [0, 2**64 - 1, 2**32, 2**32 - 1]
    k[:4] = [0, 2**31 - 1, 3, 4]
    inp = np.stack([seed, sweep, dom, k], axis=1).astype(np.uint64)
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    inp.tofile(fin)
    subprocess.run([curand_ref, str(fin), str(fout)], check=True)
    ref = np.fromfile(fout, dtype=np.uint32)
    mine = np.array([oracle.site_word(int(a), int(b), int(c), int(d))
                     for a, b, c, d in inp], dtype=np.uint32)
    assert ref.shape == (n,)
    assert np.array_equal(ref, mine)
