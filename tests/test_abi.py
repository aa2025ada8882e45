"""The C-ABI library loads and exports every symbol include/*.h declares;
host-only entry points behave (CPU, no compute calls)."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from conftest import ROOT, cuda_available


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(potts_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpotts():
    from paper_1101_0876_gb300 import build, potts
    build.build()
    return potts


def test_every_declared_symbol_is_exported(libpotts):
    declared = _declared_symbols()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", libpotts.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = declared - exported
    assert not missing, missing
    lib = libpotts.lib()
    for name in declared:
        assert hasattr(lib, name)


def test_threshold_table_equals_oracle(libpotts):
    rng = np.random.default_rng(11)
    betas = [0.0, 1e-9, 0.5, np.log(4.0), np.log1p(np.sqrt(15)), 2.0, 5.0,
             22.0, 40.0] + list(rng.uniform(0, 8, 300))
    for b in betas:
        assert np.array_equal(libpotts.threshold_table(b), oracle.thresholds(b))


def test_threshold_table_rejects_bad_beta(libpotts):
    for b in (-0.1, float("nan"), float("inf")):
        with pytest.raises(libpotts.PottsError) as ei:
            libpotts.threshold_table(b)
        assert ei.value.code == libpotts.POTTS_EINVAL
        assert "beta" in libpotts.last_error()


def test_heatbath_weights_equal_oracle(libpotts):
    rng = np.random.default_rng(12)
    cases = [(b, q) for q in (2, 3, 9, 15, 24, 96, 200, 256)
             for b in [0.0, 1e-7, 0.5, np.log1p(np.sqrt(q)), 2.0, 4.0, 5.5]]
    cases += [(float(b), int(q)) for b, q in
              zip(rng.uniform(0, 5.6, 300), rng.integers(2, 257, 300))]
    for b, q in cases:
        try:
            Wo, mo = oracle.heatbath_weights(b, q)
        except ValueError:
            with pytest.raises(libpotts.PottsError) as ei:
                libpotts.heatbath_weights(b, q)
            assert ei.value.code == libpotts.POTTS_EINVAL
            continue
        W, m = libpotts.heatbath_weights(b, q)
        assert m == mo and np.array_equal(W, Wo), (b, q)


def test_create_validates_before_touching_the_device(libpotts):
    bad = [(48, 9, 0), (16, 9, 0), (64, 1, 0), (64, 257, 0), (64, 9, 2),
           (65536 + 32, 9, 0)]
    for L, q, start in bad:
        with pytest.raises(libpotts.PottsError) as ei:
            libpotts.Lattice(L, q, start, 1)
        assert ei.value.code == libpotts.POTTS_EINVAL


@pytest.mark.skipif(cuda_available(), reason="checks the no-GPU error path")
def test_create_without_gpu_reports_cuda_error(libpotts):
    with pytest.raises(libpotts.PottsError) as ei:
        libpotts.Lattice(64, 9, 0, 1)
    assert ei.value.code == libpotts.POTTS_ECUDA


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    """The product path has no fallback: a missing library is an error."""
    from paper_1101_0876_gb300 import potts
    monkeypatch.setattr(potts, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(potts, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        potts.lib()


def test_binding_constants_equal_header_enums(libpotts):
    text = open(os.path.join(ROOT, "include", "potts.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    values = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"(POTTS_\w+)\s*=\s*(\d+)", body):
            values[name] = int(val)
    assert len(values) >= 19
    for name, val in values.items():
        short = name[len("POTTS_"):]
        got = getattr(libpotts, name, getattr(libpotts, short, None))
        assert got == val, (name, got, val)
