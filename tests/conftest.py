import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _compile(src: str, out: str, cmd: list) -> str:
    os.makedirs(BUILD, exist_ok=True)
    path = os.path.join(BUILD, out)
    if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.run(cmd + ["-o", tmp, src], check=True)
        os.replace(tmp, path)
    return path


@pytest.fixture(scope="session")
def brute_force():
    """ctypes handle to tests/brute_force.c (exact enumeration)."""
    src = os.path.join(HERE, "brute_force.c")
    path = _compile(src, "libbrute.so",
                    ["gcc", "-O2", "-std=c11", "-fPIC", "-shared"])
    lib = ctypes.CDLL(path)
    lib.potts_exact_moments.argtypes = [ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double)]
    lib.potts_exact_moments.restype = ctypes.c_int

    def moments(L, q, beta):
        out = np.zeros(5, dtype=np.float64)
        rc = lib.potts_exact_moments(L, q, beta, out.ctypes.data_as(
            ctypes.POINTER(ctypes.c_double)))
        assert rc == 0
        return out
    return moments


@pytest.fixture(scope="session")
def torch_philox():
    """PyTorch's header-only CPU Philox4x32-10, compiled with g++."""
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core",
                                       "PhiloxRNGEngine.h")):
        pytest.skip("torch C++ headers not available")
    src = os.path.join(HERE, "philox_torch_ref.cpp")
    path = _compile(src, "libphilox_ref.so",
                    ["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-I", inc])
    lib = ctypes.CDLL(path)
    P32 = ctypes.POINTER(ctypes.c_uint32)
    lib.ref_philox.argtypes = [P32, P32, P32, ctypes.c_int64]
    lib.ref_philox.restype = None

    def run(ctr, key):
        c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
        k = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
        out = np.zeros_like(c)
        lib.ref_philox(c.ctypes.data_as(P32), k.ctypes.data_as(P32),
                       out.ctypes.data_as(P32), c.shape[0])
        return out
    return run


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
