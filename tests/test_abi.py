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


def test_tuning_entry_points_reject_bad_arguments_without_gpu(lib):
    lib.lc_set_tuning.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32]
    lib.lc_get_tuning.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
    v = ctypes.c_int32()
    assert lib.lc_set_tuning(None, 1, 5) == -1
    assert lib.lc_get_tuning(None, 1, ctypes.byref(v)) == -1
    lib.lc_alu_probe.argtypes = [ctypes.c_void_p] + [ctypes.c_uint32] * 3 + [ctypes.c_void_p] * 2
    ms, ops = ctypes.c_double(), ctypes.c_double()
    assert lib.lc_alu_probe(None, 0, 64, 2, ctypes.byref(ms), ctypes.byref(ops)) == -1
    lib.lc_wait_selftest.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32]
    assert lib.lc_wait_selftest(None, 0, 16) == -1
    lib.lc_wire_bytes.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p]
    nb = ctypes.c_uint64()
    assert lib.lc_wire_bytes(None, 2, 0, ctypes.byref(nb)) == -1
    lib.lc_pack.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_uint32] * 3 + [ctypes.c_void_p]
    lib.lc_unpack.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_uint32] * 3 + [ctypes.c_void_p]
    assert lib.lc_pack(None, None, 1, 2, 0, None) == -1
    assert lib.lc_unpack(None, None, 1, 2, 0, None) == -1


def test_autotune_candidate_schedules_cover_every_rotation_bit():
    """Each candidate hoisting schedule sums to log2(N/2) and needs exactly the keys of its
    groups (2^g - 1 per group)."""
    from paper_2408_06197_b300 import autotune
    from paper_2408_06197_b300 import lancelot as LC
    for log_n in (12, 15, 16):
        for name, sched in autotune.candidate_schedules(log_n).items():
            assert sum(sched) == log_n - 1
            assert len(LC.rotations_of_schedule(sched)) == sum((1 << g) - 1 for g in sched)
    assert autotune.candidate_schedules(15)["g3qp"] == [3, 3, 3, 3, 2]


def test_handle_entry_points_reject_null_handles_without_gpu(lib):
    """The handle layer validates its arguments on the host before any device work: a missing
    context, handle or output is LC_EINVAL, and freeing a null handle is a no-op."""
    vp, u32 = ctypes.c_void_p, ctypes.c_uint32
    lib.lc_ct_info.argtypes = [vp] * 5
    lib.lc_ct_export.argtypes = [vp] * 4
    lib.lc_ct_view.argtypes = [vp, u32, u32, vp]
    lib.lc_ct_create.argtypes = [vp, u32, u32, u32, ctypes.c_double, vp]
    lib.lc_ct_import.argtypes = [vp, vp, u32, u32, u32, ctypes.c_double, vp]
    lib.lc_keygen.argtypes = [vp, vp, vp, vp, u32, vp, vp, vp]
    lib.lc_encrypt_plain.argtypes = [vp, vp, vp, u32, ctypes.c_double, vp, vp]
    lib.lc_ct_distances.argtypes = [vp, vp, vp, u32, u32, u32, vp, vp]
    lib.lc_ct_masked_aggregate.argtypes = [vp, vp, vp, u32, vp, u32, vp]
    lib.lc_batch_run.argtypes = [vp, vp, u32, u32, u32, vp]
    lib.lc_decrypt_values.argtypes = [vp, vp, vp, vp, ctypes.c_size_t]
    lib.lc_ct_data.argtypes = [vp]
    lib.lc_ct_data.restype = vp
    for f in ("lc_ct_free", "lc_sk_free", "lc_pk_free"):
        getattr(lib, f).argtypes = [vp]
        getattr(lib, f).restype = None
    out = vp()
    assert lib.lc_ct_info(None, None, None, None, None) == -1
    assert lib.lc_ct_export(None, None, None, None) == -1
    assert lib.lc_ct_view(None, 0, 1, ctypes.byref(out)) == -1
    assert lib.lc_ct_create(None, 1, 2, 0, 1.0, ctypes.byref(out)) == -1
    assert lib.lc_ct_import(None, None, 1, 2, 0, 1.0, ctypes.byref(out)) == -1
    assert lib.lc_keygen(None, None, None, None, 0, None, None, None) == -1
    assert lib.lc_encrypt_plain(None, None, None, 1, 1.0, None, ctypes.byref(out)) == -1
    assert lib.lc_ct_distances(None, None, None, 2, 1, 0, None, ctypes.byref(out)) == -1
    assert lib.lc_ct_masked_aggregate(None, None, None, 2, None, 1, ctypes.byref(out)) == -1
    assert lib.lc_batch_run(None, None, 1, 0, 0, None) == -1
    assert lib.lc_decrypt_values(None, None, None, None, 0) == -1
    assert lib.lc_ct_data(None) is None
    lib.lc_ct_free(None)
    lib.lc_sk_free(None)
    lib.lc_pk_free(None)
