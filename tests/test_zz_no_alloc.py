"""lc_rescale_noalloc -- the rescale for callers that cannot allocate device memory when they
call it -- against lc_rescale, through the C ABI.  Kept in its own file, collected last."""
import ctypes
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _residues(g, rng, count, deg, nl):
    a = np.empty((count, deg, nl, g.N), dtype=np.uint64)
    for i in range(nl):
        a[:, :, i] = rng.integers(0, g.q[i], size=(count, deg, g.N), dtype=np.uint64)
    return a


def test_rescale_noalloc_matches_rescale_on_two_calls():
    from paper_2408_06197_b300 import lancelot as LC
    lib = LC.lib()
    g = LC.Context.production()
    rng = np.random.default_rng(2024)
    for _ in range(2):  # two calls in a row reuse the shared static scratch
        ct = LC.u64_to_torch(_residues(g, rng, 1, 2, g.nq))
        ref = g.rescale(ct, g.L)
        out = torch.full_like(ref, -1)
        st = lib.lc_rescale_noalloc(g.h, ctypes.c_void_p(ct.data_ptr()), 1, 2, g.L,
                                    ctypes.c_void_p(out.data_ptr()))
        assert st == 0, lib.lc_last_error(g.h)
        g.sync()
        assert torch.equal(out, ref)  # exact integer arithmetic: bit-exact


def test_rescale_noalloc_allocates_nothing_in_a_debug_context():
    """A context whose allocator counts every call, created with LC_DEBUG (every launch checked):
    the entry point must not reach the allocator at all -- not for its scratch, not by growing
    the context's scratch arena (which would also go through the allocator) -- and must still
    return the same bits as lc_rescale."""
    from paper_2408_06197_b300 import lancelot as LC
    lib = LC.lib()
    g = LC.Context.production()
    calls = {"alloc": 0, "free": 0}
    stream = torch.cuda.current_stream()

    def _a(nbytes, user):
        calls["alloc"] += 1
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream)
        except RuntimeError:
            return None

    def _f(ptr, user):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    afn, ffn = LC._ALLOC_FN(_a), LC._FREE_FN(_f)
    alloc = LC._Allocator(afn, ffn, None)
    prm = LC._Params(g.log_n, g.nq, g.np_, g.dnum, g._qa.ctypes.data, g._pa.ctypes.data)
    h = ctypes.c_void_p()
    old = os.environ.get("LC_DEBUG")
    os.environ["LC_DEBUG"] = "1"
    try:
        st = lib.lc_ctx_create(ctypes.byref(prm), 0, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(alloc),
                               ctypes.byref(h))
    finally:
        if old is None:
            del os.environ["LC_DEBUG"]
        else:
            os.environ["LC_DEBUG"] = old
    assert st == 0
    try:
        rng = np.random.default_rng(7)
        before = dict(calls)
        for _ in range(2):
            ct = LC.u64_to_torch(_residues(g, rng, 1, 2, g.nq))
            ref = g.rescale(ct, g.L)
            out = torch.full_like(ref, -1)
            # the reference above may allocate (through g's own allocator); the counted context
            # below must not
            n0 = dict(calls)
            st = lib.lc_rescale_noalloc(h, ctypes.c_void_p(ct.data_ptr()), 1, 2, g.L, ctypes.c_void_p(out.data_ptr()))
            assert st == 0, lib.lc_last_error(h)
            assert lib.lc_sync(h) == 0, lib.lc_last_error(h)
            assert calls == n0
            assert torch.equal(out, ref)
        assert calls == before
    finally:
        lib.lc_ctx_destroy(h)


def test_rescale_noalloc_rejects_oversized_requests():
    from paper_2408_06197_b300 import lancelot as LC
    lib = LC.lib()
    g = LC.Context.production()
    ct = torch.zeros((3, 2, g.nq, g.N), dtype=torch.int64, device="cuda")
    out = torch.zeros((3, 2, g.L, g.N), dtype=torch.int64, device="cuda")
    st = lib.lc_rescale_noalloc(g.h, ctypes.c_void_p(ct.data_ptr()), 3, 2, g.L, ctypes.c_void_p(out.data_ptr()))
    assert st == -1  # LC_EINVAL
    assert b"static buffer holds" in lib.lc_last_error(g.h)
