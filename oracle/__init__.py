"""TEST INFRASTRUCTURE ONLY: plain CPU RNS-CKKS oracle for the Lancelot server evaluation.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import
this package.  It shares no code with the CUDA library (paper_2408_06197_b300) and never
imports it.  Heavy arithmetic lives in ckks_oracle.cpp (unsigned __int128, `%`, textbook
NTT); this file adds FP64 encode/decode (numpy FFT as a library step), big-integer CRT for
decryption, and scale bookkeeping.

Parity status of each function is pinned in tests/test_oracle_pins.py; nothing here is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

_u64p = ctypes.POINTER(ctypes.c_uint64)
_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        L.or_gen_primes.argtypes = [ctypes.c_int] * 4 + [vp]
        L.or_philox4x64.argtypes = [vp, vp, vp]
        L.or_sample_enc.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.or_ctx_new.restype = vp
        L.or_ctx_new.argtypes = [ctypes.c_int] * 4 + [vp, vp]
        L.or_ctx_free.argtypes = [vp]
        L.or_alpha.argtypes = [vp]
        L.or_psi.restype = ctypes.c_uint64
        L.or_psi.argtypes = [vp, ctypes.c_int]
        L.or_galois.restype = ctypes.c_uint64
        L.or_galois.argtypes = [vp, ctypes.c_long]
        L.or_counters.argtypes = [vp, vp]
        L.or_reset_counters.argtypes = [vp]
        L.or_set_threads.argtypes = [ctypes.c_int]
        for f in ("or_ntt_fwd", "or_ntt_inv"):
            getattr(L, f).argtypes = [vp, ctypes.c_int, vp]
        for f in ("or_to_coeff", "or_to_eval"):
            getattr(L, f).argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
        L.or_key_to_coeff.argtypes = [vp, vp]
        L.or_poly_mul.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        L.or_automorph_coeff.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_uint64, vp]
        L.or_modup_coeff.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp]
        L.or_moddown_coeff.argtypes = [vp, vp, ctypes.c_int, vp]
        L.or_pk_gen.argtypes = [vp, vp, vp, vp, vp]
        L.or_swk_gen.argtypes = [vp, vp, ctypes.c_uint64, vp, vp, vp]
        L.or_encrypt.argtypes = [vp] * 7
        L.or_decrypt.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
        for f in ("or_add", "or_sub"):
            getattr(L, f).argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
        L.or_tensor.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.or_relin.argtypes = [vp, vp, ctypes.c_int, vp, vp]
        L.or_rescale.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp]
        L.or_keyswitch.argtypes = [vp, vp, ctypes.c_int, vp, vp]
        L.or_rotate_hoisted.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.or_rotate_sum.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp, ctypes.c_int]
        L.or_distances.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp,
                                   ctypes.c_int, vp, vp, ctypes.c_int, vp, ctypes.c_int, vp]
        L.or_distances_dropped.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp,
                                           ctypes.c_int, vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp]
        L.or_masked_aggregate.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _ptr_array(arrs: Sequence[np.ndarray]):
    t = (ctypes.c_void_p * max(1, len(arrs)))()
    for i, a in enumerate(arrs):
        t[i] = a.ctypes.data
    return t


def set_threads(n: int) -> int:
    return lib().or_set_threads(int(n))


# ----------------------------------------------------------------------------- parameters

def gen_primes(log_n: int, bits: int, skip: int, count: int) -> List[int]:
    """The `count` largest `bits`-bit primes q = 1 mod 2N, after skipping `skip`, descending."""
    out = np.zeros(max(1, count), dtype=np.uint64)
    if lib().or_gen_primes(log_n, bits, skip, count, _p(out)) != 0:
        raise ValueError("not enough primes")
    return [int(x) for x in out[:count]]


def philox4x64(ctr: Sequence[int], key: Sequence[int]) -> List[int]:
    """One Philox4x64-10 block (four 64-bit words) for a 256-bit counter and 128-bit key."""
    c = np.array(ctr, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64(_p(c), _p(k), _p(o))
    return [int(x) for x in o]


def sample_enc(seed: int, first: int, count: int, n: int):
    """Device-randomness mode: (r int8, e0 int32, e1 int32), each [count][n], of ciphertexts
    first .. first+count-1 (Philox4x64-10; ternary r by multiply-shift, centred-binomial errors
    with eta = 21)."""
    r = np.zeros((count, n), dtype=np.int8)
    e0 = np.zeros((count, n), dtype=np.int32)
    e1 = np.zeros((count, n), dtype=np.int32)
    lib().or_sample_enc(seed, first, count, n, _p(r), _p(e0), _p(e1))
    return r, e0, e1


@dataclasses.dataclass
class Params:
    log_n: int
    q: List[int]
    p: List[int]
    dnum: int
    scale: float

    @property
    def N(self) -> int:
        return 1 << self.log_n

    @property
    def L(self) -> int:
        return len(self.q) - 1

    @property
    def alpha(self) -> int:
        return -(-len(self.q) // self.dnum)

    @property
    def slots(self) -> int:
        return self.N // 2


def params_production(log_n: int = 15) -> Params:
    """N=2^log_n (2^15 by default); q0 largest 60-bit prime = 1 mod 2N, p the next four, q1..q14
    the largest 40-bit."""
    q0 = gen_primes(log_n, 60, 0, 1)
    p = gen_primes(log_n, 60, 1, 4)
    q = q0 + gen_primes(log_n, 40, 0, 14)
    return Params(log_n, q, p, 4, float(2 ** 40))


def params_toy() -> Params:
    """N=2^12; q0 50-bit, q1..q2 30-bit, one 50-bit special prime; alpha=1, dnum=3."""
    q0 = gen_primes(12, 50, 0, 1)
    p = gen_primes(12, 50, 1, 1)
    q = q0 + gen_primes(12, 30, 0, 2)
    return Params(12, q, p, 3, float(2 ** 30))


class Context:
    def __init__(self, prm: Params):
        self.prm = prm
        q = np.array(prm.q, dtype=np.uint64)
        p = np.array(prm.p, dtype=np.uint64)
        self.h = lib().or_ctx_new(prm.log_n, len(prm.q), len(prm.p), prm.dnum, _p(q), _p(p))
        self.N = prm.N
        self.alpha = lib().or_alpha(self.h)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_ctx_free(self.h)
            self.h = None

    # ---------------------------------------------------------------- low level
    def psi(self, mi: int) -> int:
        return int(lib().or_psi(self.h, mi))

    def galois(self, r: int) -> int:
        return int(lib().or_galois(self.h, r))

    def counters(self):
        out = np.zeros(2, dtype=np.int64)
        lib().or_counters(self.h, _p(out))
        return int(out[0]), int(out[1])

    def reset_counters(self):
        lib().or_reset_counters(self.h)

    def ntt(self, mi: int, a: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib().or_ntt_fwd(self.h, mi, _p(x))
        return x

    def intt(self, mi: int, a: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib().or_ntt_inv(self.h, mi, _p(x))
        return x

    def poly_mul(self, mi: int, a, b) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.uint64)
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        lib().or_poly_mul(self.h, mi, _p(a), _p(b), _p(out))
        return out

    def to_coeff(self, data: np.ndarray) -> np.ndarray:
        """[..., rows, N] evaluation -> coefficient (rows are q_0.. q_{rows-1})."""
        x = np.ascontiguousarray(data, dtype=np.uint64).copy()
        rows = x.shape[-2]
        cnt = int(np.prod(x.shape[:-2])) if x.ndim > 2 else 1
        lib().or_to_coeff(self.h, _p(x), cnt, rows)
        return x

    def to_eval(self, data: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(data, dtype=np.uint64).copy()
        rows = x.shape[-2]
        cnt = int(np.prod(x.shape[:-2])) if x.ndim > 2 else 1
        lib().or_to_eval(self.h, _p(x), cnt, rows)
        return x

    def key_to_coeff(self, key: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(key, dtype=np.uint64).copy()
        lib().or_key_to_coeff(self.h, _p(x))
        return x

    def automorph_coeff(self, a: np.ndarray, mods: Sequence[int], g: int) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.zeros_like(a)
        m = np.array(mods, dtype=np.int32)
        lib().or_automorph_coeff(self.h, _p(a), a.shape[0], _p(m), g, _p(out))
        return out

    def modup_coeff(self, c_coef: np.ndarray, level: int, j: int) -> np.ndarray:
        c_coef = np.ascontiguousarray(c_coef, dtype=np.uint64)
        out = np.zeros((level + 1 + len(self.prm.p), self.N), dtype=np.uint64)
        lib().or_modup_coeff(self.h, _p(c_coef), level, j, _p(out))
        return out

    def moddown_coeff(self, u_coef: np.ndarray, level: int) -> np.ndarray:
        u_coef = np.ascontiguousarray(u_coef, dtype=np.uint64)
        out = np.zeros((level + 1, self.N), dtype=np.uint64)
        lib().or_moddown_coeff(self.h, _p(u_coef), level, _p(out))
        return out

    # ---------------------------------------------------------------- encode / decode
    def encode(self, z: np.ndarray, scale: float) -> np.ndarray:
        """Encode (paper: Batch Encoding): m_k = rint((2/N) Re sum_j scale z_j xi^(-k 5^j)), xi = e^(i pi/N).
        The sum over j is one length-2N FFT of the vector with scale*z_j placed at 5^j mod 2N."""
        N = self.N
        z = np.asarray(z, dtype=np.complex128)
        assert z.shape[-1] <= N // 2
        zz = np.zeros(N // 2, dtype=np.complex128)
        zz[: z.shape[-1]] = z
        e = rot_group(N)
        A = np.zeros(2 * N, dtype=np.complex128)
        A[e] = scale * zz
        F = np.fft.fft(A)  # F[k] = sum_e A[e] exp(-2 pi i k e / 2N) = sum_j w_j xi^{-k e_j}
        return np.rint((2.0 / N) * F[:N].real).astype(np.int64)

    def decode(self, m: np.ndarray, scale: float) -> np.ndarray:
        """Decode: z_j = m(xi^(5^j)) / scale (complex), m given as float coefficients."""
        N = self.N
        A = np.zeros(2 * N, dtype=np.complex128)
        A[:N] = np.asarray(m, dtype=np.float64)
        F = np.fft.ifft(A) * (2 * N)  # F[e] = sum_k m_k exp(+2 pi i k e / 2N)
        return F[rot_group(N)] / scale

    # ---------------------------------------------------------------- keys / enc / dec
    def pk_gen(self, s: np.ndarray, a: np.ndarray, e: np.ndarray) -> np.ndarray:
        out = np.zeros((2, len(self.prm.q), self.N), dtype=np.uint64)
        lib().or_pk_gen(self.h, _p(np.ascontiguousarray(s, np.int8)), _p(np.ascontiguousarray(a, np.uint64)),
                        _p(np.ascontiguousarray(e, np.int32)), _p(out))
        return out

    def swk_gen(self, s: np.ndarray, galois: int, a: np.ndarray, e: np.ndarray) -> np.ndarray:
        """galois = 0: relinearisation key (s~ = s^2); else rotation key (s~ = phi_galois(s))."""
        rows = len(self.prm.q) + len(self.prm.p)
        out = np.zeros((self.prm.dnum, 2, rows, self.N), dtype=np.uint64)
        lib().or_swk_gen(self.h, _p(np.ascontiguousarray(s, np.int8)), galois, _p(np.ascontiguousarray(a, np.uint64)),
                         _p(np.ascontiguousarray(e, np.int32)), _p(out))
        return out

    def encrypt(self, pk: np.ndarray, m: np.ndarray, r, e0, e1) -> np.ndarray:
        out = np.zeros((2, len(self.prm.q), self.N), dtype=np.uint64)
        lib().or_encrypt(self.h, _p(pk), _p(np.ascontiguousarray(m, np.int64)), _p(np.ascontiguousarray(r, np.int8)),
                         _p(np.ascontiguousarray(e0, np.int32)), _p(np.ascontiguousarray(e1, np.int32)), _p(out))
        return out

    def decrypt_residues(self, s: np.ndarray, ct: np.ndarray, level: int) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint64)
        out = np.zeros((level + 1, self.N), dtype=np.uint64)
        lib().or_decrypt(self.h, _p(np.ascontiguousarray(s, np.int8)), _p(ct), ct.shape[0], level, _p(out))
        return out

    def crt_centered(self, res: np.ndarray) -> List[int]:
        """Exact centred CRT of residues [l+1][N] (Python big integers)."""
        mods = self.prm.q[: res.shape[0]]
        Q = 1
        for q in mods:
            Q *= q
        terms = []
        for i, q in enumerate(mods):
            Qi = Q // q
            terms.append((Qi * pow(Qi % q, -1, q)) % Q)
        out = []
        cols = [res[i].tolist() for i in range(len(mods))]
        for x in range(res.shape[1]):
            v = 0
            for i in range(len(mods)):
                v += cols[i][x] * terms[i]
            v %= Q
            if v > Q // 2:
                v -= Q
            out.append(v)
        return out

    def decrypt(self, s: np.ndarray, ct: np.ndarray, level: int, scale: float) -> np.ndarray:
        """Decrypt + decode to real slot values (paper: Decryption, Batch Decoding)."""
        res = self.decrypt_residues(s, ct, level)
        m = np.array([float(v) for v in self.crt_centered(res)], dtype=np.float64)
        return self.decode(m, scale).real

    # ---------------------------------------------------------------- evaluation
    def sub(self, a, b, level):
        out = np.zeros_like(a)
        lib().or_sub(self.h, _p(a), _p(b), a.shape[0], level, _p(out))
        return out

    def add(self, a, b, level):
        out = np.zeros_like(a)
        lib().or_add(self.h, _p(a), _p(b), a.shape[0], level, _p(out))
        return out

    def tensor(self, a, b, level):
        out = np.zeros((3,) + a.shape[1:], dtype=np.uint64)
        lib().or_tensor(self.h, _p(a), _p(b), level, _p(out))
        return out

    def relin(self, ct3, level, rlk):
        out = np.zeros((2,) + ct3.shape[1:], dtype=np.uint64)
        lib().or_relin(self.h, _p(ct3), level, _p(rlk), _p(out))
        return out

    def rescale(self, ct, level):
        out = np.zeros((ct.shape[0], level, self.N), dtype=np.uint64)
        lib().or_rescale(self.h, _p(ct), ct.shape[0], level, _p(out))
        return out

    def keyswitch(self, poly_eval, level, key):
        out = np.zeros((2, level + 1, self.N), dtype=np.uint64)
        lib().or_keyswitch(self.h, _p(np.ascontiguousarray(poly_eval)), level, _p(key), _p(out))
        return out

    def rotate_hoisted(self, ct, level, rots: Sequence[int], keys: Sequence[np.ndarray]):
        outs = [np.zeros_like(ct) for _ in rots]
        r = (ctypes.c_long * len(rots))(*rots)
        lib().or_rotate_hoisted(self.h, _p(ct), level, len(rots), r, _ptr_array(keys), _ptr_array(outs))
        return outs

    def rotate_sum(self, ct, level, groups: Sequence[int], rot_keys: dict, qp_sum: bool = False):
        """Rotate-and-sum with hoisting groups; qp_sum sums each group's inner products in Q U P
        and switches down once (the one-ModDown hoisting variant)."""
        x = np.ascontiguousarray(ct).copy()
        g = np.array(groups, dtype=np.int32)
        kr = np.array(list(rot_keys.keys()), dtype=np.int32)
        ks = [rot_keys[k] for k in rot_keys]
        st = lib().or_rotate_sum(self.h, _p(x), level, len(g), _p(g), len(kr), _p(kr), _ptr_array(ks),
                                 int(qp_sum))
        if st:
            raise KeyError("missing rotation key")
        return x

    def distances(self, cts: np.ndarray, rlk, groups, rot_keys: dict, pairs=None, qp_sum: bool = False,
                  rot_level: int | None = None) -> np.ndarray:
        """cts [n][chunks][2][L+1][N] -> [n_pairs][2][L][N] (i<j lexicographic, or `pairs`).
        rot_level: reduce each rescaled pair to that level (keep its limbs 0..rot_level) before the
        rotate-and-sum; the output is then [n_pairs][2][rot_level+1][N]."""
        n, chunks = cts.shape[0], cts.shape[1]
        L = len(self.prm.q) - 1
        if rot_level is not None:
            return self._distances_dropped(cts, rlk, groups, rot_keys, pairs, qp_sum, rot_level)
        g = np.array(groups, dtype=np.int32)
        kr = np.array(list(rot_keys.keys()), dtype=np.int32)
        ks = [rot_keys[k] for k in rot_keys]
        if pairs is None:
            pl = np.zeros(2, dtype=np.int32)
            nsel = 0
            npairs = n * (n - 1) // 2
        else:
            pl = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1))
            nsel = len(pairs)
            npairs = nsel
        out = np.zeros((npairs, 2, L, self.N), dtype=np.uint64)
        st = lib().or_distances(self.h, _p(np.ascontiguousarray(cts)), n, chunks, _p(rlk), len(g), _p(g),
                                len(kr), _p(kr), _ptr_array(ks), nsel, _p(pl), int(qp_sum), _p(out))
        if st:
            raise KeyError("missing rotation key")
        return out

    def _distances_dropped(self, cts, rlk, groups, rot_keys, pairs, qp_sum, rot_level):
        n, chunks = cts.shape[0], cts.shape[1]
        g = np.array(groups, dtype=np.int32)
        kr = np.array(list(rot_keys.keys()), dtype=np.int32)
        ks = [rot_keys[k] for k in rot_keys]
        if pairs is None:
            pl = np.zeros(2, dtype=np.int32)
            nsel, npairs = 0, n * (n - 1) // 2
        else:
            pl = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1))
            nsel = npairs = len(pairs)
        out = np.zeros((npairs, 2, rot_level + 1, self.N), dtype=np.uint64)
        st = lib().or_distances_dropped(self.h, _p(np.ascontiguousarray(cts)), n, chunks, _p(rlk), len(g), _p(g),
                                        len(kr), _p(kr), _ptr_array(ks), nsel, _p(pl), int(qp_sum), int(rot_level),
                                        _p(out))
        if st == -2:
            raise ValueError("rot_level outside [0, L-1]")
        if st:
            raise KeyError("missing rotation key")
        return out

    def masked_aggregate(self, cts: np.ndarray, masks: np.ndarray, rlk) -> np.ndarray:
        n, chunks = cts.shape[0], cts.shape[1]
        L = len(self.prm.q) - 1
        out = np.zeros((chunks, 2, L, self.N), dtype=np.uint64)
        lib().or_masked_aggregate(self.h, _p(np.ascontiguousarray(cts)), n, chunks, _p(np.ascontiguousarray(masks)),
                                  _p(rlk), _p(out))
        return out


def rot_group(N: int) -> np.ndarray:
    """Exponents 5^j mod 2N for j < N/2 (the slot order, subgroup T = <5>)."""
    e = np.empty(N // 2, dtype=np.int64)
    v = 1
    for j in range(N // 2):
        e[j] = v
        v = (v * 5) % (2 * N)
    return e


def default_schedule(slots: int) -> List[int]:
    """Log-step rotate-and-sum: one rotation per group (g = 1), log2(slots) groups."""
    return [1] * int(round(math.log2(slots)))


def rotations_of_schedule(groups: Sequence[int]) -> List[int]:
    out, stride = [], 1
    for g in groups:
        for t in range(1, 1 << g):
            out.append(t * stride)
        stride <<= g
    return out
