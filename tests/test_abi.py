"""The C-ABI library loads on CPU and exports every symbol include/lancelot.h declares; host-only
entry points (prime generation, argument validation) work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lancelot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_06197_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 25
    for s in syms:
        assert hasattr(lib, s), s


def test_primes_agree_with_oracle_rule(lib):
    from paper_2408_06197_b300 import lancelot as LC
    log_n, q, p, dnum, _ = LC.production_primes()
    prm = O.params_production()
    assert (q, p, dnum) == (prm.q, prm.p, prm.dnum)
    log_n, q, p, dnum, _ = LC.toy_primes()
    prm = O.params_toy()
    assert (q, p, dnum) == (prm.q, prm.p, prm.dnum)


def test_invalid_arguments_are_rejected_without_gpu(lib):
    lib.lc_gen_primes.argtypes = [ctypes.c_uint32] * 4 + [ctypes.c_void_p]
    out = np.zeros(4, dtype=np.uint64)
    assert lib.lc_gen_primes(15, 70, 0, 1, out.ctypes.data) == -1   # bits out of range
    assert lib.lc_gen_primes(15, 60, 0, 1, None) == -1
    lib.lc_ctx_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.lc_ctx_create(None, 0, None, None, None) == -1
    lib.lc_distances.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_uint32] * 2 + [ctypes.c_double] + \
        [ctypes.c_uint32] * 2 + [ctypes.c_void_p] * 3
    assert lib.lc_distances(None, None, None, 0, 0, 1.0, 0, 0, None, None, None) == -1
