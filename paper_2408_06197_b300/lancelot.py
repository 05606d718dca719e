"""Thin Python binding of liblancelot.so (include/lancelot.h).

Argument marshalling only: every step of the evaluation runs in the library's CUDA kernels.
PyTorch provides device memory (its caching allocator is handed to the library) and the CUDA
stream.  Ciphertext arrays are torch.int64 tensors on the GPU holding the library's uint64
words ([count][poly][limb][N], evaluation domain).  The library is loaded on first use; if it
is missing or cannot be loaded the call raises -- there is no CPU path.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import sys
import weakref
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblancelot.so")

LC_OK = 0
LC_MODE_PER_OP = 0
LC_MODE_BATCHED = 1
LC_HOIST_QP_SUM = 2
LC_H2D = 0
LC_D2H = 1
# tile-shape knobs (lc_set_tuning); options listed default first
LC_TUNE_NTT_ROW_MINB = 1
LC_TUNE_NTT_COL_MINB = 2
LC_TUNE_GROUP_SPLIT_ITEMS = 3
LC_TUNE_GROUP_WIDE_ITEMS = 4
LC_TUNE_TENSOR_WARPS = 5
LC_TUNE_NTT_ROW_TMA = 6
LC_TUNE_GROUP_KARATSUBA = 7
LC_PROBE_IMAD, LC_PROBE_IMAD_WIDE, LC_PROBE_NTT_BFLY = 0, 1, 2
TUNING_OPTIONS = {
    LC_TUNE_NTT_ROW_MINB: (5, 4, 6),
    LC_TUNE_NTT_COL_MINB: (8, 1, 6, 7),
    LC_TUNE_GROUP_SPLIT_ITEMS: (1, 2),
    LC_TUNE_GROUP_WIDE_ITEMS: (1, 2),
    LC_TUNE_TENSOR_WARPS: (16, 8, 12),
    LC_TUNE_NTT_ROW_TMA: (0, 1),
    LC_TUNE_GROUP_KARATSUBA: (1, 0),
}
TUNING_NAMES = {LC_TUNE_NTT_ROW_MINB: "ntt_row_minb", LC_TUNE_NTT_COL_MINB: "ntt_col_minb",
                LC_TUNE_GROUP_SPLIT_ITEMS: "group_split_items", LC_TUNE_GROUP_WIDE_ITEMS: "group_wide_items",
                LC_TUNE_TENSOR_WARPS: "tensor_warps", LC_TUNE_NTT_ROW_TMA: "ntt_row_tma",
                LC_TUNE_GROUP_KARATSUBA: "group_karatsuba"}
_ERRS = {-1: "LC_EINVAL", -2: "LC_ELEVEL", -3: "LC_ESCALE", -4: "LC_ENOMEM", -5: "LC_ECUDA",
         -6: "LC_ETIMEOUT", -7: "LC_EBUSY", -8: "LC_EKEY"}

_lib = None
vp = ctypes.c_void_p
u32 = ctypes.c_uint32


class LancelotError(RuntimeError):
    pass


class _Params(ctypes.Structure):
    _fields_ = [("log_n", u32), ("n_q", u32), ("n_p", u32), ("dnum", u32), ("q", vp), ("p", vp)]


_LIVE = weakref.WeakSet()  # contexts, key sets and graphs still holding library handles


def _close_all():
    """Releases every live handle at interpreter exit, while torch and CUDA are still up."""
    objs = list(_LIVE)
    for kind in (Graph, KgcKey, EvalKeys, Context):
        for o in objs:
            if isinstance(o, kind):
                try:
                    o.close()
                except Exception:
                    pass


atexit.register(_close_all)

_ALLOC_FN = ctypes.CFUNCTYPE(vp, ctypes.c_size_t, vp)
_FREE_FN = ctypes.CFUNCTYPE(None, vp, vp)


class _Job(ctypes.Structure):
    _fields_ = [("evk", vp), ("cts", vp), ("n", u32), ("chunks", u32), ("masks", vp), ("out_dist", vp),
                ("out_agg", vp)]


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", vp)]


class _KeygenRand(ctypes.Structure):
    _fields_ = [("pk_a", vp), ("pk_e", vp), ("swk_a", vp), ("swk_e", vp)]


class _EncRand(ctypes.Structure):
    _fields_ = [("r", vp), ("e0", vp), ("e1", vp)]


class _CtJob(ctypes.Structure):
    _fields_ = [("evk", vp), ("clients", vp), ("n", u32), ("masks", vp), ("want_dist", u32), ("dist", vp),
                ("agg", vp)]


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LancelotError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "lc_gen_primes": [u32, u32, u32, u32, vp],
            "lc_ctx_create": [vp, ctypes.c_int, vp, vp, vp],
            "lc_ctx_destroy": [vp],
            "lc_set_stream": [vp, vp],
            "lc_sync": [vp],
            "lc_counters": [vp, vp, ctypes.c_int],
            "lc_pk_gen": [vp, vp, vp, vp, vp],
            "lc_evk_create": [vp, vp],
            "lc_evk_free": [vp],
            "lc_evk_add": [vp, vp, vp, ctypes.c_int32, vp, vp],
            "lc_evk_export": [vp, vp, ctypes.c_int32, vp],
            "lc_evk_import": [vp, vp, ctypes.c_int32, vp],
            "lc_encode": [vp, vp, ctypes.c_size_t, ctypes.c_double, vp],
            "lc_decode": [vp, vp, ctypes.c_double, vp],
            "lc_encrypt": [vp, vp, vp, vp, vp, vp, u32, vp],
            "lc_decrypt": [vp, vp, vp, u32, u32, vp],
            "lc_crt_to_double": [vp, vp, u32, vp],
            "lc_to_coeff": [vp, vp, u32, u32],
            "lc_to_eval": [vp, vp, u32, u32],
            "lc_add": [vp, vp, vp, u32, u32, vp],
            "lc_sub": [vp, vp, vp, u32, u32, vp],
            "lc_tensor": [vp, vp, vp, u32, vp],
            "lc_relin": [vp, vp, vp, u32, u32, vp],
            "lc_rescale": [vp, vp, u32, u32, u32, vp],
            "lc_rescale_noalloc": [vp, vp, u32, u32, u32, vp],
            "lc_rotate": [vp, vp, vp, u32, u32, vp, vp],
            "lc_rotate_sum": [vp, vp, vp, u32, u32, u32, vp, u32],
            "lc_distances": [vp, vp, vp, u32, u32, ctypes.c_double, u32, u32, vp, vp, vp],
            "lc_masked_aggregate": [vp, vp, vp, u32, u32, ctypes.c_double, vp, ctypes.c_double, u32, vp, vp],
            "lc_memcpy_h2d": [vp, vp, vp, ctypes.c_size_t],
            "lc_memcpy_d2h": [vp, vp, vp, ctypes.c_size_t],
            "lc_launches": [vp],
            "lc_profile": [vp, ctypes.c_int, vp, vp, vp],
            "lc_set_max_batch": [vp, u32],
            "lc_set_tuning": [vp, u32, ctypes.c_int32],
            "lc_copy_async": [vp, vp, vp, ctypes.c_size_t, ctypes.c_int, vp],
            "lc_copy_wait": [vp, ctypes.c_uint64],
            "lc_get_tuning": [vp, u32, vp],
            "lc_alu_probe": [vp, u32, u32, u32, vp, vp],
            "lc_wait_selftest": [vp, ctypes.c_int, u32],
            "lc_wire_bytes": [vp, u32, u32, vp],
            "lc_pack": [vp, vp, u32, u32, u32, vp],
            "lc_unpack": [vp, vp, u32, u32, u32, vp],
            "lc_graph_begin": [vp],
            "lc_graph_end": [vp, vp],
            "lc_graph_launch": [vp, vp],
            "lc_graph_free": [vp],
            "lc_batch_distances": [vp, vp, u32, u32, u32, vp],
            "lc_batch_aggregate": [vp, vp, u32],
            "lc_decrypt_const": [vp, vp, vp, u32, u32, ctypes.c_double, vp],
            "lc_sample_enc": [vp, ctypes.c_uint64, ctypes.c_uint64, u32, vp, vp, vp],
            "lc_encode_dev": [vp, vp, u32, ctypes.c_double, vp],
            "lc_encode_encrypt_seeded": [vp, vp, vp, u32, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, vp],
            "lc_encrypt_seeded": [vp, vp, vp, u32, ctypes.c_uint64, ctypes.c_uint64, vp],
            "lc_encrypt_const_seeded": [vp, vp, vp, u32, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, vp],
            "lc_kgc_create": [vp, vp, vp],
            "lc_kgc_free": [vp],
            "lc_kgc_readout": [vp, vp, vp, u32, u32, ctypes.c_double, vp],
            "lc_kgc_krum": [vp, vp, u32, u32, u32, ctypes.c_int, vp, vp],
            "lc_ct_create": [vp, u32, u32, u32, ctypes.c_double, vp],
            "lc_ct_import": [vp, vp, u32, u32, u32, ctypes.c_double, vp],
            "lc_ct_export": [vp, vp, vp, vp],
            "lc_ct_info": [vp, vp, vp, vp, vp],
            "lc_ct_view": [vp, u32, u32, vp],
            "lc_ct_free": [vp],
            "lc_keygen": [vp, vp, vp, vp, u32, vp, vp, vp],
            "lc_sk_free": [vp],
            "lc_pk_free": [vp],
            "lc_encrypt_plain": [vp, vp, vp, u32, ctypes.c_double, vp, vp],
            "lc_encrypt_values": [vp, vp, vp, ctypes.c_size_t, ctypes.c_double, vp, vp],
            "lc_decrypt_values": [vp, vp, vp, vp, ctypes.c_size_t],
            "lc_ct_distances": [vp, vp, vp, u32, u32, u32, vp, vp],
            "lc_ct_masked_aggregate": [vp, vp, vp, u32, vp, u32, vp],
            "lc_batch_run": [vp, vp, u32, u32, u32, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name in ("lc_ctx_destroy", "lc_evk_free", "lc_graph_free", "lc_ct_free",
                                         "lc_sk_free", "lc_pk_free") else ctypes.c_int
        L.lc_ct_data.argtypes = [vp]
        L.lc_ct_data.restype = vp
        L.lc_last_error.argtypes = [vp]
        L.lc_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _np_ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return ctypes.c_void_p(a.ctypes.data)


def _t_ptr(t: torch.Tensor):
    assert t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def _need(buf, words: int, what: str, host_ok: bool = False):
    """The library trusts raw pointers; check every caller buffer here so that a wrong shape raises
    instead of letting a kernel read or write past its end."""
    if isinstance(buf, torch.Tensor):
        if buf.dtype not in (torch.int64, torch.uint64) or not buf.is_cuda or not buf.is_contiguous():
            raise LancelotError(f"{what}: needs a contiguous 64-bit CUDA tensor")
        n = buf.numel()
    elif isinstance(buf, np.ndarray) and host_ok:
        if buf.dtype != np.uint64 or not buf.flags.c_contiguous:
            raise LancelotError(f"{what}: needs a C-contiguous uint64 array")
        n = buf.size
    else:
        raise LancelotError(f"{what}: unsupported buffer type {type(buf).__name__}")
    if n != words:
        raise LancelotError(f"{what}: has {n} words, expected {words}")
    return buf


def _whole(buf, unit: int, what: str) -> int:
    n = buf.numel()
    if unit <= 0 or n == 0 or n % unit:
        raise LancelotError(f"{what}: {n} words is not a whole number of {unit}-word items")
    return n // unit


def rotate_at_level(level: int) -> int:
    """Mode bits of lc_distances that drop the rescaled pairs to `level` before the
    rotate-and-sum (LC_ROTATE_AT_LEVEL)."""
    return (int(level) + 1) << 8


def launches() -> int:
    out = np.zeros(1, dtype=np.uint64)
    lib().lc_launches(_np_ptr(out))
    return int(out[0])


class PinnedArray(np.ndarray):
    """numpy view of page-locked torch storage (keeps the storage alive)."""
    _owner = None


def pinned_empty(shape, dtype=np.uint64) -> np.ndarray:
    """Page-locked host array (torch pinned memory viewed as numpy)."""
    n = int(np.prod(shape)) * np.dtype(dtype).itemsize
    t = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    a = t.numpy().view(dtype).reshape(shape).view(PinnedArray)
    a._owner = t
    return a


def gen_primes(log_n: int, bits: int, skip: int, count: int) -> List[int]:
    out = np.zeros(max(1, count), dtype=np.uint64)
    st = lib().lc_gen_primes(log_n, bits, skip, count, _np_ptr(out))
    if st != LC_OK:
        raise LancelotError(f"lc_gen_primes: {_ERRS.get(st, st)}")
    return [int(x) for x in out[:count]]


def production_primes(log_n: int = 15):
    """N = 2^log_n (2^15 by default): q0 = largest 60-bit prime = 1 mod 2N, p = the next four
    60-bit ones, q1..q14 = the largest 40-bit ones (descending); dnum 4, scale 2^40."""
    q0 = gen_primes(log_n, 60, 0, 1)
    p = gen_primes(log_n, 60, 1, 4)
    return log_n, q0 + gen_primes(log_n, 40, 0, 14), p, 4, float(2 ** 40)


def toy_primes():
    """N = 2^12: q0 50-bit, q1..q2 30-bit, one 50-bit special prime; dnum = 3 (alpha = 1)."""
    q0 = gen_primes(12, 50, 0, 1)
    p = gen_primes(12, 50, 1, 1)
    return 12, q0 + gen_primes(12, 30, 0, 2), p, 3, float(2 ** 30)


def u64_to_torch(a: np.ndarray, device="cuda") -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)


def torch_to_u64(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


class Context:
    """One GPU context: parameters, device tables, the torch stream, scratch."""

    def __init__(self, log_n: int, q: Sequence[int], p: Sequence[int], dnum: int, scale: float,
                 device: int = 0, stream: Optional[torch.cuda.Stream] = None, use_torch_allocator: bool = True):
        L = lib()
        self.log_n, self.N = log_n, 1 << log_n
        self.q, self.p, self.dnum, self.scale = list(q), list(p), dnum, scale
        self.nq, self.np_ = len(q), len(p)
        self.alpha = -(-self.nq // dnum)
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        self._qa = np.array(q, dtype=np.uint64)
        self._pa = np.array(p, dtype=np.uint64)
        prm = _Params(log_n, len(q), len(p), dnum, self._qa.ctypes.data, self._pa.ctypes.data)
        self._alloc = None
        if use_torch_allocator:
            dev, st = device, self.stream

            def _a(nbytes, user):
                if sys.is_finalizing():
                    return None
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except RuntimeError:
                    return None

            def _f(ptr, user):
                if sys.is_finalizing():
                    return  # the process is exiting: leave the memory to the driver
                try:
                    torch.cuda.caching_allocator_delete(ptr)
                except Exception:
                    pass

            self._afn, self._ffn = _ALLOC_FN(_a), _FREE_FN(_f)
            self._alloc = _Allocator(self._afn, self._ffn, None)
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            st = L.lc_ctx_create(ctypes.byref(prm), device, ctypes.c_void_p(self.stream.cuda_stream),
                                 ctypes.byref(self._alloc) if self._alloc else None, ctypes.byref(h))
        if st != LC_OK:
            raise LancelotError(f"lc_ctx_create: {_ERRS.get(st, st)}")
        self.h = h
        self._deps = weakref.WeakSet()  # key sets and graphs made on this context
        _LIVE.add(self)

    @classmethod
    def production(cls, log_n: int = 15, **kw):
        """The production modulus chain (60 + 14 x 40 bits, 4 x 60-bit special primes) at
        N = 2^log_n (the packing-size sweep varies log_n; 15 is the evaluated setting)."""
        log_n, q, p, dnum, scale = production_primes(log_n)
        return cls(log_n, q, p, dnum, scale, **kw)

    @classmethod
    def toy(cls, **kw):
        log_n, q, p, dnum, scale = toy_primes()
        return cls(log_n, q, p, dnum, scale, **kw)

    def close(self):
        if getattr(self, "h", None):
            for dep in list(getattr(self, "_deps", ())):
                try:
                    dep.close()
                except Exception:
                    pass
            lib().lc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def L(self) -> int:
        return self.nq - 1

    @property
    def slots(self) -> int:
        return self.N // 2

    def _check(self, st: int, what: str):
        if st != LC_OK:
            msg = lib().lc_last_error(self.h)
            raise LancelotError(f"{what}: {_ERRS.get(st, st)} {msg.decode() if msg else ''}")

    def capture(self, fn) -> "Graph":
        """Captures the library calls made by fn() on this context's stream into a CUDA graph.
        Run fn() once before capturing so that every scratch buffer is already sized."""
        self._check(lib().lc_graph_begin(self.h), "lc_graph_begin")
        try:
            fn()
        finally:
            h = ctypes.c_void_p()
            st = lib().lc_graph_end(self.h, ctypes.byref(h))
        self._check(st, "lc_graph_end")
        return Graph(self, h)

    def set_max_batch(self, max_items: int):
        self._check(lib().lc_set_max_batch(self.h, int(max_items)), "lc_set_max_batch")

    def set_tuning(self, knob: int, value: int):
        """Select a tile-shape option (LC_TUNE_*; see TUNING_OPTIONS).  Results do not change."""
        self._check(lib().lc_set_tuning(self.h, int(knob), int(value)), "lc_set_tuning")

    def get_tuning(self, knob: int) -> int:
        v = ctypes.c_int32()
        self._check(lib().lc_get_tuning(self.h, int(knob), ctypes.byref(v)), "lc_get_tuning")
        return int(v.value)

    def tuning(self) -> Dict[str, int]:
        return {TUNING_NAMES[k]: self.get_tuning(k) for k in TUNING_OPTIONS}

    def alu_probe(self, kind: int, iters: int = 4096, blocks_per_sm: int = 8) -> Dict[str, float]:
        """Register-resident integer-pipe probe (LC_PROBE_*): {"ms", "ops", "ops_per_s"}."""
        ms, ops = ctypes.c_double(), ctypes.c_double()
        self._check(lib().lc_alu_probe(self.h, int(kind), int(iters), int(blocks_per_sm), ctypes.byref(ms),
                                       ctypes.byref(ops)), "lc_alu_probe")
        return {"ms": ms.value, "ops": ops.value, "ops_per_s": ops.value / (ms.value * 1e-3)}

    # ------------------------------------------------------------------ wire form
    def wire_bytes(self, deg: int, level: int) -> int:
        """Bytes of one wire-form record of `deg` polynomials at `level` (lc_wire_bytes)."""
        v = ctypes.c_uint64()
        self._check(lib().lc_wire_bytes(self.h, int(deg), int(level), ctypes.byref(v)), "lc_wire_bytes")
        return int(v.value)

    def pack(self, data: torch.Tensor, deg: int, level: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Word layout [count][deg][level+1][N] -> wire form (uint8 CUDA tensor [count][bytes])."""
        count = _whole(data, deg * (level + 1) * self.N, "pack")
        _need(data, count * deg * (level + 1) * self.N, "pack")
        rb = self.wire_bytes(deg, level)
        if out is None:
            out = torch.empty((count, rb), dtype=torch.uint8, device=data.device)
        if out.dtype != torch.uint8 or not out.is_cuda or not out.is_contiguous() or out.numel() < count * rb:
            raise LancelotError("pack: out must be a contiguous uint8 CUDA tensor of count x wire_bytes")
        self._check(lib().lc_pack(self.h, _t_ptr(data), count, int(deg), int(level), _t_ptr(out)), "lc_pack")
        return out

    def unpack(self, wire: torch.Tensor, count: int, deg: int, level: int,
               out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Wire form -> word layout [count][deg][level+1][N]; a residue not below its prime makes
        the next sync raise (LC_EINVAL)."""
        rb = self.wire_bytes(deg, level)
        if wire.dtype != torch.uint8 or not wire.is_cuda or not wire.is_contiguous() or wire.numel() < count * rb:
            raise LancelotError("unpack: wire must be a contiguous uint8 CUDA tensor of count x wire_bytes")
        if out is None:
            out = self.empty(count, deg, level + 1, self.N)
        _need(out, count * deg * (level + 1) * self.N, "unpack: out")
        self._check(lib().lc_unpack(self.h, _t_ptr(wire), int(count), int(deg), int(level), _t_ptr(out)), "lc_unpack")
        return out

    def wait_selftest(self, never_arrive: bool = False, max_polls: int = 1 << 16) -> int:
        """Bounded-wait self-test: LC_OK, or -6 (LC_ETIMEOUT) when a wait ran out (no exception)."""
        return int(lib().lc_wait_selftest(self.h, int(bool(never_arrive)), int(max_polls)))

    def sync(self):
        self._check(lib().lc_sync(self.h), "lc_sync")

    def counters(self, reset: bool = False):
        out = np.zeros(2, dtype=np.uint64)
        self._check(lib().lc_counters(self.h, _np_ptr(out), int(reset)), "lc_counters")
        return int(out[0]), int(out[1])

    PROF_CLASSES = ("ntt", "modup", "inner", "moddown", "tensor", "rescale", "automorphism", "other")

    def profile_start(self):
        self._check(lib().lc_profile(self.h, 1, None, None, None), "lc_profile")

    def profile_stop(self) -> Dict[str, dict]:
        ms = np.zeros(8)
        by = np.zeros(8)
        ln = np.zeros(8, dtype=np.uint64)
        self._check(lib().lc_profile(self.h, 0, _np_ptr(ms), _np_ptr(by), _np_ptr(ln)), "lc_profile")
        return {k: {"ms": float(ms[i]), "bytes": float(by[i]), "launches": int(ln[i])}
                for i, k in enumerate(self.PROF_CLASSES)}

    def h2d(self, dst: torch.Tensor, src: np.ndarray):
        """Stream-ordered host->device copy through the C ABI (src pinned or pageable)."""
        if not (isinstance(dst, torch.Tensor) and dst.is_cuda and dst.is_contiguous()
                and dst.numel() * dst.element_size() == src.nbytes):
            raise LancelotError("h2d: destination must be a contiguous CUDA tensor of the same byte size")
        self._check(lib().lc_memcpy_h2d(self.h, _t_ptr(dst), ctypes.c_void_p(src.ctypes.data), src.nbytes),
                    "lc_memcpy_h2d")

    def d2h(self, dst: np.ndarray, src: torch.Tensor):
        if not (isinstance(src, torch.Tensor) and src.is_cuda and src.is_contiguous()
                and src.numel() * src.element_size() == dst.nbytes and dst.flags.c_contiguous):
            raise LancelotError("d2h: source must be a contiguous CUDA tensor of the same byte size")
        self._check(lib().lc_memcpy_d2h(self.h, ctypes.c_void_p(dst.ctypes.data), _t_ptr(src), dst.nbytes),
                    "lc_memcpy_d2h")

    def copy_async(self, dst, src) -> int:
        """Overlapped copy between a device tensor and a pinned host array (either direction),
        ordered after the work enqueued so far; returns a ticket for copy_wait."""
        t = ctypes.c_uint64()

        def dev_ok(x, nbytes):
            return (x.is_cuda and x.is_contiguous() and x.dtype in (torch.int64, torch.uint64, torch.uint8)
                    and x.numel() * x.element_size() >= nbytes)
        if isinstance(dst, torch.Tensor) and isinstance(src, np.ndarray):
            if not dev_ok(dst, src.nbytes):
                raise LancelotError("copy_async: dst must be a contiguous 64-bit or byte CUDA tensor of src's size")
            args = (_t_ptr(dst), _np_ptr(src), src.nbytes, LC_H2D)
        elif isinstance(dst, np.ndarray) and isinstance(src, torch.Tensor):
            if not dev_ok(src, dst.nbytes):
                raise LancelotError("copy_async: src must be a contiguous 64-bit or byte CUDA tensor of dst's size")
            args = (_np_ptr(dst), _t_ptr(src), dst.nbytes, LC_D2H)
        else:
            raise LancelotError("copy_async: one side must be a device tensor and the other a host array")
        self._check(lib().lc_copy_async(self.h, *args, ctypes.byref(t)), "lc_copy_async")
        return int(t.value)

    def copy_wait(self, ticket: int):
        """The context's stream waits for the copy `ticket`."""
        self._check(lib().lc_copy_wait(self.h, int(ticket)), "lc_copy_wait")

    def empty(self, *shape) -> torch.Tensor:
        return torch.empty(shape, dtype=torch.int64, device=f"cuda:{self.device}")

    def ct_shape(self, count: int, deg: int, level: int):
        return (count, deg, level + 1, self.N)

    # ------------------------------------------------------------------ keys
    def pk_gen(self, s: np.ndarray, a: np.ndarray, e: np.ndarray) -> torch.Tensor:
        pk = self.empty(2, self.nq, self.N)
        self._check(lib().lc_pk_gen(self.h, _np_ptr(np.ascontiguousarray(s, np.int8)),
                                    _np_ptr(np.ascontiguousarray(a, np.uint64)),
                                    _np_ptr(np.ascontiguousarray(e, np.int32)), _t_ptr(pk)), "lc_pk_gen")
        return pk

    def evk(self) -> "EvalKeys":
        return EvalKeys(self)

    # ------------------------------------------------------------------ handles (lc_ct, lc_keygen, ...)
    def keygen(self, s: np.ndarray, pk_a: np.ndarray, pk_e: np.ndarray, rlk_rand, rot_rand: Dict[int, tuple]):
        """lc_keygen: (SecretKey, PublicKey, EvalKeys) from the secret and the caller's randomness;
        rlk_rand = (a, e) of the relinearisation key, rot_rand = {step: (a, e)}."""
        steps = [int(r) for r in rot_rand]
        sw_a = np.ascontiguousarray(np.stack([rlk_rand[0]] + [rot_rand[r][0] for r in steps]), np.uint64)
        sw_e = np.ascontiguousarray(np.stack([rlk_rand[1]] + [rot_rand[r][1] for r in steps]), np.int32)
        pa, pe = np.ascontiguousarray(pk_a, np.uint64), np.ascontiguousarray(pk_e, np.int32)
        if sw_a.shape != (1 + len(steps), self.dnum, self.nq + self.np_, self.N) or pa.shape != (self.nq, self.N):
            raise LancelotError("keygen: randomness of the wrong shape")
        s8 = np.ascontiguousarray(s, np.int8)
        if s8.size != self.N:
            raise LancelotError("keygen: the secret must hold N values")
        rnd = _KeygenRand(pa.ctypes.data, pe.ctypes.data, sw_a.ctypes.data, sw_e.ctypes.data)
        rs = (ctypes.c_int32 * max(1, len(steps)))(*steps)
        hs, hp, he = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        self._check(lib().lc_keygen(self.h, _np_ptr(s8), ctypes.byref(rnd), rs, len(steps), ctypes.byref(hs),
                                    ctypes.byref(hp), ctypes.byref(he)), "lc_keygen")
        evk = EvalKeys.__new__(EvalKeys)
        evk.ctx, evk.h, evk.rotations = self, he, steps
        self._deps.add(evk)
        _LIVE.add(evk)
        return SecretKey(self, hs), PublicKey(self, hp), evk

    def ct_create(self, count: int, deg: int, level: int, scale: float) -> "Ciphertext":
        h = ctypes.c_void_p()
        self._check(lib().lc_ct_create(self.h, int(count), int(deg), int(level), float(scale), ctypes.byref(h)),
                    "lc_ct_create")
        return Ciphertext(self, h)

    def ct_import(self, coeffs: np.ndarray, deg: int, level: int, scale: float) -> "Ciphertext":
        """Ciphertexts in the canonical interchange form (coefficient domain, [count][deg][level+1][N])."""
        a = np.ascontiguousarray(coeffs, np.uint64)
        unit = deg * (level + 1) * self.N
        if a.size == 0 or a.size % unit:
            raise LancelotError(f"ct_import: {a.size} words is not a whole number of {unit}-word ciphertexts")
        count = a.size // unit
        h = ctypes.c_void_p()
        self._check(lib().lc_ct_import(self.h, _np_ptr(a), count, int(deg), int(level), float(scale),
                                       ctypes.byref(h)), "lc_ct_import")
        return Ciphertext(self, h)

    @staticmethod
    def _enc_rand(count: int, N: int, r, e0, e1):
        arrs = (np.ascontiguousarray(r, np.int8), np.ascontiguousarray(e0, np.int32), np.ascontiguousarray(e1, np.int32))
        if any(x.size != count * N for x in arrs):
            raise LancelotError(f"encryption randomness must hold {count} x N values each")
        return arrs, _EncRand(*(x.ctypes.data for x in arrs))

    def encrypt_plain(self, pk: "PublicKey", m: np.ndarray, scale: float, r, e0, e1) -> "Ciphertext":
        mm = np.ascontiguousarray(m, np.int64).reshape(-1, self.N)
        keep, rnd = self._enc_rand(mm.shape[0], self.N, r, e0, e1)
        h = ctypes.c_void_p()
        self._check(lib().lc_encrypt_plain(self.h, pk.h, _np_ptr(mm), mm.shape[0], float(scale), ctypes.byref(rnd),
                                           ctypes.byref(h)), "lc_encrypt_plain")
        return Ciphertext(self, h)

    def encrypt_values(self, pk: "PublicKey", values: np.ndarray, scale: float, r, e0, e1) -> "Ciphertext":
        v = np.ascontiguousarray(values, np.float64).reshape(-1)
        count = -(-v.size // self.slots)
        keep, rnd = self._enc_rand(count, self.N, r, e0, e1)
        h = ctypes.c_void_p()
        self._check(lib().lc_encrypt_values(self.h, pk.h, _np_ptr(v), v.size, float(scale), ctypes.byref(rnd),
                                            ctypes.byref(h)), "lc_encrypt_values")
        return Ciphertext(self, h)

    def decrypt_values(self, sk: "SecretKey", ct: "Ciphertext", length: Optional[int] = None) -> np.ndarray:
        n = ct.count * self.slots if length is None else int(length)
        out = np.zeros(n, dtype=np.float64)
        self._check(lib().lc_decrypt_values(self.h, sk.h, ct.h, _np_ptr(out), n), "lc_decrypt_values")
        return out

    @staticmethod
    def _handles(cts: Sequence["Ciphertext"]):
        return (ctypes.c_void_p * len(cts))(*[c.h.value if c is not None else None for c in cts])

    def ct_distances(self, evk: "EvalKeys", clients: Sequence["Ciphertext"], mode: int = 1,
                     groups: Optional[Sequence[int]] = None) -> "Ciphertext":
        arr = self._handles(clients)
        g = np.ascontiguousarray(groups if groups is not None else [], np.uint32)
        h = ctypes.c_void_p()
        self._check(lib().lc_ct_distances(self.h, evk.h, arr, len(clients), int(mode), g.size,
                                          _np_ptr(g) if g.size else None, ctypes.byref(h)), "lc_ct_distances")
        return Ciphertext(self, h)

    def ct_masked_aggregate(self, evk: "EvalKeys", clients: Sequence["Ciphertext"], masks: Sequence["Ciphertext"],
                            mode: int = 1) -> "Ciphertext":
        arr, marr = self._handles(clients), self._handles(masks)
        h = ctypes.c_void_p()
        self._check(lib().lc_ct_masked_aggregate(self.h, evk.h, arr, len(clients), marr, int(mode), ctypes.byref(h)),
                    "lc_ct_masked_aggregate")
        return Ciphertext(self, h)

    def batch_run(self, jobs: Sequence[dict], flags: int = 0, groups: Optional[Sequence[int]] = None):
        """lc_batch_run over jobs {"evk", "clients", "masks" (optional), "distances" (bool)}:
        returns [(dist Ciphertext or None, agg Ciphertext or None)] in job order."""
        keep = []
        cj = (_CtJob * max(1, len(jobs)))()
        for k, j in enumerate(jobs):
            arr = self._handles(j["clients"])
            marr = self._handles(j["masks"]) if j.get("masks") is not None else None
            keep.append((arr, marr))
            cj[k] = _CtJob(j["evk"].h, ctypes.cast(arr, vp), len(j["clients"]),
                           ctypes.cast(marr, vp) if marr is not None else None, int(bool(j.get("distances", True))),
                           None, None)
        g = np.ascontiguousarray(groups if groups is not None else [], np.uint32)
        self._check(lib().lc_batch_run(self.h, cj, len(jobs), int(flags), g.size, _np_ptr(g) if g.size else None),
                    "lc_batch_run")
        return [(Ciphertext(self, ctypes.c_void_p(cj[k].dist)) if cj[k].dist else None,
                 Ciphertext(self, ctypes.c_void_p(cj[k].agg)) if cj[k].agg else None) for k in range(len(jobs))]

    # ------------------------------------------------------------------ encode / encrypt / decrypt
    def encode(self, z: np.ndarray, scale: float) -> np.ndarray:
        z = np.ascontiguousarray(z, dtype=np.float64)
        m = np.zeros(self.N, dtype=np.int64)
        self._check(lib().lc_encode(self.h, _np_ptr(z), z.shape[0], scale, _np_ptr(m)), "lc_encode")
        return m

    def decode(self, m: np.ndarray, scale: float) -> np.ndarray:
        m = np.ascontiguousarray(m, dtype=np.float64)
        z = np.zeros(self.N // 2, dtype=np.float64)
        self._check(lib().lc_decode(self.h, _np_ptr(m), scale, _np_ptr(z)), "lc_decode")
        return z

    def encrypt(self, pk: torch.Tensor, m: np.ndarray, r: np.ndarray, e0: np.ndarray, e1: np.ndarray,
                out: Optional[torch.Tensor] = None) -> torch.Tensor:
        m = np.ascontiguousarray(m, np.int64).reshape(-1, self.N)
        count = m.shape[0]
        for name, arr in (("r", r), ("e0", e0), ("e1", e1)):
            if np.asarray(arr).size != count * self.N:
                raise LancelotError(f"encrypt: {name} must hold {count} x N values")
        _need(pk, 2 * self.nq * self.N, "encrypt: pk")
        if out is None:
            out = self.empty(count, 2, self.nq, self.N)
        _need(out, count * 2 * self.nq * self.N, "encrypt: out")
        self._check(lib().lc_encrypt(self.h, _t_ptr(pk), _np_ptr(m), _np_ptr(np.ascontiguousarray(r, np.int8)),
                                     _np_ptr(np.ascontiguousarray(e0, np.int32)),
                                     _np_ptr(np.ascontiguousarray(e1, np.int32)), count, _t_ptr(out)), "lc_encrypt")
        return out

    def decrypt_residues(self, s: np.ndarray, ct: torch.Tensor, level: int) -> np.ndarray:
        ct = ct.contiguous()
        deg = ct.shape[-3] if ct.dim() >= 3 else 2
        _need(ct, deg * (level + 1) * self.N, "decrypt: ct")
        res = np.zeros((level + 1, self.N), dtype=np.uint64)
        self._check(lib().lc_decrypt(self.h, _np_ptr(np.ascontiguousarray(s, np.int8)), _t_ptr(ct), deg, level,
                                     _np_ptr(res)), "lc_decrypt")
        return res

    def decrypt_const(self, s: np.ndarray, cts: torch.Tensor, level: int, scale: float) -> np.ndarray:
        """Slot average of each ciphertext holding one value in every slot (KGC read-out)."""
        if cts.numel() == 0:
            return np.zeros(0, dtype=np.float64)
        count = _whole(cts, 2 * (level + 1) * self.N, "decrypt_const")
        out = np.zeros(count, dtype=np.float64)
        self._check(lib().lc_decrypt_const(self.h, _np_ptr(np.ascontiguousarray(s, np.int8)), _t_ptr(cts), count,
                                           level, scale, _np_ptr(out)), "lc_decrypt_const")
        return out

    # ------------------------------------------------------------------ device randomness
    def sample_enc(self, seed: int, first: int, count: int):
        """The device-randomness draws (r int8, e0 int32, e1 int32; [count][N]) of ciphertexts
        first .. first+count-1."""
        r = np.zeros((count, self.N), dtype=np.int8)
        e0 = np.zeros((count, self.N), dtype=np.int32)
        e1 = np.zeros((count, self.N), dtype=np.int32)
        self._check(lib().lc_sample_enc(self.h, int(seed), int(first), int(count), _np_ptr(r), _np_ptr(e0),
                                        _np_ptr(e1)), "lc_sample_enc")
        return r, e0, e1

    def encrypt_seeded(self, pk: torch.Tensor, m: torch.Tensor, seed: int, first: int,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Encrypt device plaintexts m ([count][N] int64 tensor) with device randomness."""
        count = _whole(m, self.N, "encrypt_seeded: m")
        _need(pk, 2 * self.nq * self.N, "encrypt_seeded: pk")
        if out is None:
            out = self.empty(count, 2, self.nq, self.N)
        _need(out, count * 2 * self.nq * self.N, "encrypt_seeded: out")
        self._check(lib().lc_encrypt_seeded(self.h, _t_ptr(pk), _t_ptr(m), count, int(seed), int(first),
                                            _t_ptr(out)), "lc_encrypt_seeded")
        return out

    def _slots_arg(self, z: torch.Tensor, what: str) -> int:
        if z.dtype != torch.float64 or not z.is_cuda or not z.is_contiguous() or z.numel() % self.slots:
            raise LancelotError(f"{what}: z must be a contiguous float64 CUDA tensor of whole slot vectors")
        return z.numel() // self.slots

    def encode_dev(self, z: torch.Tensor, scale: float, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """GPU encode of real slot vectors z ([count][N/2] float64 CUDA tensor) -> int64 [count][N]."""
        count = self._slots_arg(z, "encode_dev")
        if out is None:
            out = torch.empty(count, self.N, dtype=torch.int64, device=z.device)
        _need(out, count * self.N, "encode_dev: out")
        self._check(lib().lc_encode_dev(self.h, ctypes.c_void_p(z.data_ptr()), count, float(scale), _t_ptr(out)),
                    "lc_encode_dev")
        return out

    def encode_encrypt_seeded(self, pk: torch.Tensor, z: torch.Tensor, scale: float, seed: int, first: int,
                              out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Encode on the GPU and encrypt with device randomness (the clients' batched step)."""
        count = self._slots_arg(z, "encode_encrypt_seeded")
        _need(pk, 2 * self.nq * self.N, "encode_encrypt_seeded: pk")
        if out is None:
            out = self.empty(count, 2, self.nq, self.N)
        _need(out, count * 2 * self.nq * self.N, "encode_encrypt_seeded: out")
        self._check(lib().lc_encode_encrypt_seeded(self.h, _t_ptr(pk), ctypes.c_void_p(z.data_ptr()), count,
                                                   float(scale), int(seed), int(first), _t_ptr(out)),
                    "lc_encode_encrypt_seeded")
        return out

    def encrypt_const_seeded(self, pk: torch.Tensor, w: torch.Tensor, scale: float, seed: int, first: int,
                             out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Constant-slot ciphertexts (coefficient 0 = round(w[b] scale)) from device doubles w."""
        if w.dtype != torch.float64 or not w.is_cuda or not w.is_contiguous():
            raise LancelotError("encrypt_const_seeded: w must be a contiguous float64 CUDA tensor")
        count = w.numel()
        _need(pk, 2 * self.nq * self.N, "encrypt_const_seeded: pk")
        if out is None:
            out = self.empty(count, 2, self.nq, self.N)
        _need(out, count * 2 * self.nq * self.N, "encrypt_const_seeded: out")
        self._check(lib().lc_encrypt_const_seeded(self.h, _t_ptr(pk), ctypes.c_void_p(w.data_ptr()), count,
                                                  float(scale), int(seed), int(first), _t_ptr(out)),
                    "lc_encrypt_const_seeded")
        return out

    def decrypt(self, s: np.ndarray, ct: torch.Tensor, level: int, scale: float) -> np.ndarray:
        res = self.decrypt_residues(s, ct, level)
        m = np.zeros(self.N, dtype=np.float64)
        self._check(lib().lc_crt_to_double(self.h, _np_ptr(res), level, _np_ptr(m)), "lc_crt_to_double")
        return self.decode(m, scale)

    # ------------------------------------------------------------------ interchange
    def to_coeff(self, data: torch.Tensor, level: int, inplace: bool = False) -> torch.Tensor:
        """Evaluation -> coefficient domain; a copy unless `inplace` (then `data` must be contiguous)."""
        x = data if inplace else data.clone().contiguous()
        n_polys = _whole(x, (level + 1) * self.N, "to_coeff")
        _need(x, n_polys * (level + 1) * self.N, "to_coeff")
        self._check(lib().lc_to_coeff(self.h, _t_ptr(x), n_polys, level), "lc_to_coeff")
        return x

    def to_eval(self, data: torch.Tensor, level: int, inplace: bool = False) -> torch.Tensor:
        """Coefficient -> evaluation domain; a copy unless `inplace` (then `data` must be contiguous)."""
        x = data if inplace else data.clone().contiguous()
        n_polys = _whole(x, (level + 1) * self.N, "to_eval")
        _need(x, n_polys * (level + 1) * self.N, "to_eval")
        self._check(lib().lc_to_eval(self.h, _t_ptr(x), n_polys, level), "lc_to_eval")
        return x

    # ------------------------------------------------------------------ primitives
    def add(self, a, b, level):
        _whole(a, (level + 1) * self.N, "add")
        _need(b, a.numel(), "add: b")
        out = torch.empty_like(a)
        self._check(lib().lc_add(self.h, _t_ptr(a), _t_ptr(b), a.numel() // ((level + 1) * self.N), level,
                                 _t_ptr(out)), "lc_add")
        return out

    def sub(self, a, b, level):
        _whole(a, (level + 1) * self.N, "sub")
        _need(b, a.numel(), "sub: b")
        out = torch.empty_like(a)
        self._check(lib().lc_sub(self.h, _t_ptr(a), _t_ptr(b), a.numel() // ((level + 1) * self.N), level,
                                 _t_ptr(out)), "lc_sub")
        return out

    def tensor(self, a, b, level):
        _need(a, 2 * (level + 1) * self.N, "tensor: a")
        _need(b, 2 * (level + 1) * self.N, "tensor: b")
        out = self.empty(3, level + 1, self.N)
        self._check(lib().lc_tensor(self.h, _t_ptr(a), _t_ptr(b), level, _t_ptr(out)), "lc_tensor")
        return out

    def relin(self, evk: "EvalKeys", ct3: torch.Tensor, level: int) -> torch.Tensor:
        count = _whole(ct3, 3 * (level + 1) * self.N, "relin")
        out = self.empty(count, 2, level + 1, self.N)
        self._check(lib().lc_relin(self.h, evk.h, _t_ptr(ct3), count, level, _t_ptr(out)), "lc_relin")
        return out

    def rescale(self, ct: torch.Tensor, level: int, deg: int = 2) -> torch.Tensor:
        count = _whole(ct, deg * (level + 1) * self.N, "rescale")
        out = self.empty(count, deg, level, self.N)
        self._check(lib().lc_rescale(self.h, _t_ptr(ct), count, deg, level, _t_ptr(out)), "lc_rescale")
        return out

    def rescale_noalloc(self, ct: torch.Tensor, level: int, deg: int = 2,
                        out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Rescale through the entry point that allocates nothing (fixed 16 MiB library scratch);
        pass a preallocated `out` when no allocation may happen at all."""
        count = _whole(ct, deg * (level + 1) * self.N, "rescale_noalloc")
        if out is None:
            out = self.empty(count, deg, level, self.N)
        _need(out, count * deg * level * self.N, "rescale_noalloc: out")
        self._check(lib().lc_rescale_noalloc(self.h, _t_ptr(ct), count, deg, level, _t_ptr(out)),
                    "lc_rescale_noalloc")
        return out

    def rotate(self, evk: "EvalKeys", ct: torch.Tensor, level: int, rots: Sequence[int]) -> torch.Tensor:
        r = np.array(list(rots), dtype=np.int32)
        _need(ct, 2 * (level + 1) * self.N, "rotate: ct")
        out = self.empty(len(r), 2, level + 1, self.N)
        self._check(lib().lc_rotate(self.h, evk.h, _t_ptr(ct), level, len(r), _np_ptr(r), _t_ptr(out)), "lc_rotate")
        return out

    def rotate_sum(self, evk: "EvalKeys", ct: torch.Tensor, level: int, groups: Sequence[int],
                   qp_sum: bool = False) -> torch.Tensor:
        y = ct.clone().contiguous()
        g = np.array(list(groups), dtype=np.uint32)
        count = _whole(y, 2 * (level + 1) * self.N, "rotate_sum")
        self._check(lib().lc_rotate_sum(self.h, evk.h, _t_ptr(y), count, level, len(g), _np_ptr(g),
                                        LC_HOIST_QP_SUM if qp_sum else 0), "lc_rotate_sum")
        return y

    # ------------------------------------------------------------------ the method
    def distances(self, evk: "EvalKeys", cts, n: int, chunks: int, scale: float, mode: int = LC_MODE_BATCHED,
                  groups: Optional[Sequence[int]] = None, out=None, rot_level: Optional[int] = None):
        """cts: [n][chunks][2][nq][N] (torch GPU tensor, or numpy uint64 in host memory).
        rot_level: drop each rescaled pair to that level before the rotate-and-sum (outputs
        [n_pairs][2][rot_level+1][N]); None keeps level L-1."""
        npairs = n * (n - 1) // 2
        nl_out = self.L if rot_level is None else int(rot_level) + 1
        if rot_level is not None:
            mode = int(mode) | rotate_at_level(int(rot_level))
        host = isinstance(cts, np.ndarray)
        if out is None:
            out = (np.empty((npairs, 2, nl_out, self.N), dtype=np.uint64) if host
                   else self.empty(npairs, 2, nl_out, self.N))
        _need(cts, n * chunks * 2 * self.nq * self.N, "distances: cts", host_ok=True)
        _need(out, npairs * 2 * nl_out * self.N, "distances: out", host_ok=True)
        g = np.array(list(groups) if groups else [], dtype=np.uint32)
        sc = ctypes.c_double()
        pin = _np_ptr(cts) if host else _t_ptr(cts)
        pout = _np_ptr(out) if isinstance(out, np.ndarray) else _t_ptr(out)
        self._check(lib().lc_distances(self.h, evk.h, pin, n, chunks, scale, mode, len(g),
                                       _np_ptr(g) if len(g) else None, pout, ctypes.byref(sc)), "lc_distances")
        return out, sc.value

    def masked_aggregate(self, evk: "EvalKeys", cts, n: int, chunks: int, scale: float, masks, mask_scale: float,
                         mode: int = LC_MODE_BATCHED, out=None):
        host = isinstance(cts, np.ndarray)
        if out is None:
            out = (np.empty((chunks, 2, self.L, self.N), dtype=np.uint64) if host
                   else self.empty(chunks, 2, self.L, self.N))
        _need(cts, n * chunks * 2 * self.nq * self.N, "masked_aggregate: cts", host_ok=True)
        _need(masks, n * 2 * self.nq * self.N, "masked_aggregate: masks", host_ok=True)
        _need(out, chunks * 2 * self.L * self.N, "masked_aggregate: out", host_ok=True)
        sc = ctypes.c_double()
        pin = _np_ptr(cts) if host else _t_ptr(cts)
        pm = _np_ptr(masks) if isinstance(masks, np.ndarray) else _t_ptr(masks)
        pout = _np_ptr(out) if isinstance(out, np.ndarray) else _t_ptr(out)
        self._check(lib().lc_masked_aggregate(self.h, evk.h, pin, n, chunks, scale, pm, mask_scale, mode, pout,
                                              ctypes.byref(sc)), "lc_masked_aggregate")
        return out, sc.value


class Job:
    """One aggregation round: its tenant's keys, client ciphertexts [n][chunks][2][nq][N] and,
    for the aggregate, masks [n][2][nq][N].  Outputs are allocated on demand."""

    def __init__(self, evk: "EvalKeys", cts: torch.Tensor, n: int, chunks: int, masks: Optional[torch.Tensor] = None):
        ctx = evk.ctx
        _need(cts, n * chunks * 2 * ctx.nq * ctx.N, "Job: cts")
        if masks is not None:
            _need(masks, n * 2 * ctx.nq * ctx.N, "Job: masks")
        self.evk, self.cts, self.n, self.chunks, self.masks = evk, cts, n, chunks, masks
        self.out_dist: Optional[torch.Tensor] = None
        self.out_agg: Optional[torch.Tensor] = None

    def _c(self) -> _Job:
        return _Job(self.evk.h.value, self.cts.data_ptr(), self.n, self.chunks,
                    self.masks.data_ptr() if self.masks is not None else None,
                    self.out_dist.data_ptr() if self.out_dist is not None else None,
                    self.out_agg.data_ptr() if self.out_agg is not None else None)


def batch_distances(ctx: "Context", jobs: Sequence[Job], mode_flags: int = 0,
                    groups: Optional[Sequence[int]] = None):
    """Distances of several rounds (different n, model sizes, tenants) in shared batched waves."""
    for j in jobs:
        if j.out_dist is None:
            j.out_dist = ctx.empty(j.n * (j.n - 1) // 2, 2, ctx.L, ctx.N)
        _need(j.out_dist, j.n * (j.n - 1) // 2 * 2 * ctx.L * ctx.N, "batch_distances: out")
    arr = (_Job * max(1, len(jobs)))(*[j._c() for j in jobs])
    g = np.array(list(groups) if groups else [], dtype=np.uint32)
    ctx._check(lib().lc_batch_distances(ctx.h, arr, len(jobs), int(mode_flags) & LC_HOIST_QP_SUM, len(g),
                                        _np_ptr(g) if len(g) else None), "lc_batch_distances")


def batch_aggregate(ctx: "Context", jobs: Sequence[Job]):
    """Masked aggregates of several rounds in shared batched waves."""
    for j in jobs:
        if j.masks is None:
            raise LancelotError("batch_aggregate: job without masks")
        if j.out_agg is None:
            j.out_agg = ctx.empty(j.chunks, 2, ctx.L, ctx.N)
        _need(j.out_agg, j.chunks * 2 * ctx.L * ctx.N, "batch_aggregate: out")
    arr = (_Job * max(1, len(jobs)))(*[j._c() for j in jobs])
    ctx._check(lib().lc_batch_aggregate(ctx.h, arr, len(jobs)), "lc_batch_aggregate")


class Graph:
    """A captured sequence of library calls; launch() replays it on the context's stream."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        ctx._deps.add(self)
        _LIVE.add(self)

    def launch(self):
        self.ctx._check(lib().lc_graph_launch(self.ctx.h, self.h), "lc_graph_launch")

    def close(self):
        if getattr(self, "h", None):
            lib().lc_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Handle:
    """A library handle freed through its (live) context."""
    _free = None

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        ctx._deps.add(self)
        _LIVE.add(self)

    def close(self):
        if getattr(self, "h", None):
            if getattr(self.ctx, "h", None) and self.h.value:
                getattr(lib(), self._free)(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SecretKey(_Handle):
    """lc_sk: the KGC's secret key."""
    _free = "lc_sk_free"


class PublicKey(_Handle):
    """lc_pk: the public key the clients encrypt with."""
    _free = "lc_pk_free"


class Ciphertext(_Handle):
    """lc_ct: a device-resident array of ciphertexts that carries its degree, level and scale."""
    _free = "lc_ct_free"

    def info(self):
        c, d, l, sc = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
        self.ctx._check(lib().lc_ct_info(self.h, ctypes.byref(c), ctypes.byref(d), ctypes.byref(l), ctypes.byref(sc)),
                        "lc_ct_info")
        return int(c.value), int(d.value), int(l.value), float(sc.value)

    @property
    def count(self) -> int:
        return self.info()[0]

    @property
    def level(self) -> int:
        return self.info()[2]

    @property
    def scale(self) -> float:
        return self.info()[3]

    def export(self) -> np.ndarray:
        """[count][deg][level+1][N] in the coefficient domain (canonical interchange form)."""
        count, deg, level, _ = self.info()
        out = np.zeros((count, deg, level + 1, self.ctx.N), dtype=np.uint64)
        self.ctx._check(lib().lc_ct_export(self.h, _np_ptr(out), None, None), "lc_ct_export")
        return out

    def view(self, first: int, count: int) -> "Ciphertext":
        h = ctypes.c_void_p()
        self.ctx._check(lib().lc_ct_view(self.h, int(first), int(count), ctypes.byref(h)), "lc_ct_view")
        return Ciphertext(self.ctx, h)

    def tensor(self) -> torch.Tensor:
        """A torch view of the device words [count][deg][level+1][N] (evaluation domain) that
        keeps this handle alive."""
        count, deg, level, _ = self.info()
        n = count * deg * (level + 1) * self.ctx.N
        ptr = lib().lc_ct_data(self.h)

        class _Arr:  # __cuda_array_interface__ over the handle's memory
            __cuda_array_interface__ = {"shape": (n,), "typestr": "<i8", "data": (ptr, False), "version": 2,
                                        "strides": None}
        t = torch.as_tensor(_Arr(), device=f"cuda:{self.ctx.device}")
        t._lc_owner = self
        return t.view(count, deg, level + 1, self.ctx.N)


class EvalKeys:
    """Device-resident switching keys (relinearisation + rotations): the server's evk."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx._check(lib().lc_evk_create(ctx.h, ctypes.byref(h)), "lc_evk_create")
        self.h = h
        ctx._deps.add(self)
        _LIVE.add(self)
        self.rotations: List[int] = []

    def add(self, s: np.ndarray, rotation: Optional[int], a: np.ndarray, e: np.ndarray):
        rot = -1 if rotation is None else int(rotation)
        self.ctx._check(lib().lc_evk_add(self.ctx.h, self.h, _np_ptr(np.ascontiguousarray(s, np.int8)), rot,
                                         _np_ptr(np.ascontiguousarray(a, np.uint64)),
                                         _np_ptr(np.ascontiguousarray(e, np.int32))), "lc_evk_add")
        if rotation is not None:
            self.rotations.append(int(rotation))

    def export(self, rotation: Optional[int]) -> np.ndarray:
        c = self.ctx
        out = np.zeros((c.dnum, 2, c.nq + c.np_, c.N), dtype=np.uint64)
        rot = -1 if rotation is None else int(rotation)
        c._check(lib().lc_evk_export(c.h, self.h, rot, _np_ptr(out)), "lc_evk_export")
        return out

    def import_key(self, rotation: Optional[int], key: np.ndarray):
        """Adds a key from its canonical form (as `export` returns it): a key set restored without
        the secret."""
        c = self.ctx
        k = np.ascontiguousarray(key, np.uint64)
        if k.shape != (c.dnum, 2, c.nq + c.np_, c.N):
            raise LancelotError(f"import_key: expected shape {(c.dnum, 2, c.nq + c.np_, c.N)}, got {k.shape}")
        rot = -1 if rotation is None else int(rotation)
        c._check(lib().lc_evk_import(c.h, self.h, rot, _np_ptr(k)), "lc_evk_import")
        if rotation is not None:
            self.rotations.append(int(rotation))

    def close(self):
        if getattr(self, "h", None):
            if getattr(self.ctx, "h", None):  # the keys are freed through their (live) context
                lib().lc_evk_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KgcKey:
    """The KGC's secret resident on the device (mod q0) for the device-side KGC step: read-out
    of the distance ciphertexts and Krum / Multi-Krum selection, without host round trips."""

    def __init__(self, ctx: Context, s: np.ndarray):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx._check(lib().lc_kgc_create(ctx.h, _np_ptr(np.ascontiguousarray(s, np.int8)), ctypes.byref(h)),
                   "lc_kgc_create")
        self.h = h
        ctx._deps.add(self)
        _LIVE.add(self)

    def readout(self, cts: torch.Tensor, level: int, scale: float,
                out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Slot value of each constant-slot ciphertext, into a device float64 tensor."""
        c = self.ctx
        count = _whole(cts, 2 * (level + 1) * c.N, "kgc readout")
        if out is None:
            out = torch.empty(count, dtype=torch.float64, device=cts.device)
        if out.dtype != torch.float64 or out.numel() != count or not out.is_contiguous():
            raise LancelotError("kgc readout: out must be a contiguous float64 tensor of one value per ciphertext")
        c._check(lib().lc_kgc_readout(c.h, self.h, _t_ptr(cts), count, level, float(scale),
                                      ctypes.c_void_p(out.data_ptr())), "lc_kgc_readout")
        return out

    def krum(self, dist: torch.Tensor, n: int, f: int, n_select: int, average: bool = True,
             w: Optional[torch.Tensor] = None, sel: Optional[torch.Tensor] = None):
        """(weights [n] float64, kept indices [n_select] int32), both on the device (pass w and
        sel to reuse buffers, e.g. inside a graph capture)."""
        c = self.ctx
        if dist.dtype != torch.float64 or dist.numel() != n * (n - 1) // 2 or not dist.is_contiguous():
            raise LancelotError("kgc krum: dist must hold n(n-1)/2 contiguous float64 values")
        if w is None:
            w = torch.empty(n, dtype=torch.float64, device=dist.device)
        if sel is None:
            sel = torch.empty(n_select, dtype=torch.int32, device=dist.device)
        if w.dtype != torch.float64 or w.numel() != n or sel.dtype != torch.int32 or sel.numel() != n_select:
            raise LancelotError("kgc krum: w must hold n float64 values and sel n_select int32 values")
        c._check(lib().lc_kgc_krum(c.h, ctypes.c_void_p(dist.data_ptr()), n, f, n_select, 1 if average else 0,
                                   ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(sel.data_ptr())), "lc_kgc_krum")
        return w, sel

    def close(self):
        if getattr(self, "h", None):
            if getattr(self.ctx, "h", None):
                lib().lc_kgc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rotations_of_schedule(groups: Sequence[int]) -> List[int]:
    out, stride = [], 1
    for g in groups:
        for t in range(1, 1 << g):
            out.append(t * stride)
        stride <<= g
    return out
