"""lc_rescale_noalloc -- the rescale for callers that cannot allocate device memory when they
call it -- against lc_rescale, through the C ABI.  Kept in its own file, collected last."""
import ctypes

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


def test_rescale_noalloc_rejects_oversized_requests():
    from paper_2408_06197_b300 import lancelot as LC
    lib = LC.lib()
    g = LC.Context.production()
    ct = torch.zeros((3, 2, g.nq, g.N), dtype=torch.int64, device="cuda")
    out = torch.zeros((3, 2, g.L, g.N), dtype=torch.int64, device="cuda")
    st = lib.lc_rescale_noalloc(g.h, ctypes.c_void_p(ct.data_ptr()), 3, 2, g.L, ctypes.c_void_p(out.data_ptr()))
    assert st == -1  # LC_EINVAL
    assert b"static buffer holds" in lib.lc_last_error(g.h)
