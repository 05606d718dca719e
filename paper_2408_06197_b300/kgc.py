"""Key-generation-center side of masked-based encrypted sorting (host, plaintext).

The KGC holds sk, decrypts the pair distances, sorts the clients and returns an encrypted
mask (paper: Section "Masked-based Encrypted Sorting", Algorithm 2; aggregation rules in the
appendix "Descriptions of Aggregation Rules").  This module is the plaintext part: scores,
selection and the mask matrix P_pi.  Encrypting the mask uses the library's encrypt call.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def krum_scores(dist: np.ndarray, f: int) -> np.ndarray:
    """s_i = sum of the n - f - 2 smallest squared distances from W_i to the other updates."""
    d = np.asarray(dist, dtype=np.float64)
    n = d.shape[0]
    k = max(0, n - f - 2)
    out = np.empty(n)
    for i in range(n):
        others = np.sort(np.delete(d[i], i), kind="stable")
        out[i] = others[:k].sum()
    return out


def krum_select(dist: np.ndarray, f: int, n_select: int) -> List[int]:
    """Krum (n_select = 1) / Multi-Krum: the n_select lowest Krum scores, stable order, ties to
    the lower index (Algorithm 2's ArgSort-then-take-first loop).  The loop's extra condition
    n - |psi| > 2c + 2 is not applied: the workload's l wins where the two disagree."""
    s = krum_scores(dist, f)
    order = np.argsort(s, kind="stable")
    return [int(i) for i in order[:n_select]]


def median_select(dist: np.ndarray) -> int:
    """Distance median (Algorithm 2, Median branch): the client at the middle of the ArgSort of
    the per-client distance sums, positions read 1-based ((n+1)/2 odd, n/2 even)."""
    sums = np.asarray(dist, dtype=np.float64).sum(axis=1)
    order = np.argsort(sums, kind="stable")
    return int(order[(len(sums) - 1) // 2])


def permutation_mask(n: int, selected: Sequence[int]) -> np.ndarray:
    """P_pi restricted to the kept clients: row r is e_{selected[r]}, remaining rows are o."""
    P = np.zeros((n, n), dtype=np.int64)
    for r, c in enumerate(selected):
        P[r, c] = 1
    return P


def mask_weights(n: int, selected: Sequence[int], average: bool) -> np.ndarray:
    """Per-client weight folded into the mask ciphertext: the column sums of P_pi, divided by
    l for Multi-Krum averaging (the (c/n) factor of ServerUpdate folded into the mask)."""
    w = permutation_mask(n, selected).sum(axis=0).astype(np.float64)
    if average and len(selected):
        w /= len(selected)
    return w
