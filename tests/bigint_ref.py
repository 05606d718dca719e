"""Independent big-integer reference for tiny ring sizes (pins the oracle, not the GPU path).

Everything here is written directly from textbook definitions with Python integers:
negacyclic schoolbook multiplication in Z_q[X]/(X^N+1), evaluation at powers of a 2N-th root,
CRT composition, and substitution X -> X^g.  It shares nothing with oracle/ or the CUDA path.
"""
from __future__ import annotations

from typing import List, Sequence


def negacyclic_mul(a: Sequence[int], b: Sequence[int], q: int) -> List[int]:
    N = len(a)
    out = [0] * N
    for i in range(N):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += ai * int(b[j])
            else:
                out[k - N] -= ai * int(b[j])
    return [x % q for x in out]


def negacyclic_mul_int(a: Sequence[int], b: Sequence[int]) -> List[int]:
    """Exact product over Z[X]/(X^N+1) (no modulus)."""
    N = len(a)
    out = [0] * N
    for i in range(N):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += ai * int(b[j])
            else:
                out[k - N] -= ai * int(b[j])
    return out


def eval_at(a: Sequence[int], point: int, q: int) -> int:
    acc = 0
    for c in reversed([int(x) for x in a]):
        acc = (acc * point + c) % q
    return acc


def substitute(a: Sequence[int], g: int) -> List[int]:
    """a(X^g) mod X^N+1 over the integers."""
    N = len(a)
    out = [0] * N
    for i, c in enumerate(a):
        k = (i * g) % (2 * N)
        if k < N:
            out[k] += int(c)
        else:
            out[k - N] -= int(c)
    return out


def crt(residues: Sequence[int], moduli: Sequence[int]) -> int:
    """Value in [0, prod) with the given residues."""
    M = 1
    for m in moduli:
        M *= m
    x = 0
    for r, m in zip(residues, moduli):
        Mi = M // m
        x += int(r) * Mi * pow(Mi % m, -1, m)
    return x % M


def centred(x: int, M: int) -> int:
    x %= M
    return x - M if x > M // 2 else x


def prod(xs: Sequence[int]) -> int:
    p = 1
    for x in xs:
        p *= int(x)
    return p


def round_div(x: int, d: int) -> int:
    """round(x/d) for odd d > 0 (no ties)."""
    return (2 * x + d) // (2 * d)
