"""Shared builders for the parity tests: the same seeded randomness goes to the oracle and to
the CUDA library; nothing the CUDA path computes is ever fed to the oracle."""
from __future__ import annotations

import numpy as np

import oracle as O
import synth as S


def oracle_params(kind: str) -> O.Params:
    return O.params_toy() if kind == "toy" else O.params_production()


def gpu_context(kind: str):
    from paper_2408_06197_b300 import lancelot as LC
    return LC.Context.toy() if kind == "toy" else LC.Context.production()


class KeySet:
    """Secret, public-key and switching-key randomness for one (seed, config)."""

    def __init__(self, prm: O.Params, seed: int, config: int, rotations):
        N = prm.N
        self.prm = prm
        self.s = S.secret_key(seed, config, N)
        self.pk_a, self.pk_e = S.pk_rand(seed, config, prm.q, N)
        qp = prm.q + prm.p
        self.rlk = S.swk_rand(seed, config, qp, prm.dnum, N, None)
        self.rot = {r: S.swk_rand(seed, config, qp, prm.dnum, N, r) for r in rotations}

    def oracle_keys(self, ctx: O.Context):
        pk = ctx.pk_gen(self.s, self.pk_a, self.pk_e)
        rlk = ctx.swk_gen(self.s, 0, *self.rlk)
        rk = {r: ctx.swk_gen(self.s, ctx.galois(r), *v) for r, v in self.rot.items()}
        return pk, rlk, rk

    def gpu_keys(self, g):
        pk = g.pk_gen(self.s, self.pk_a, self.pk_e)
        evk = g.evk()
        evk.add(self.s, None, *self.rlk)
        for r, v in self.rot.items():
            evk.add(self.s, r, *v)
        return pk, evk


def plaintexts(ctx: O.Context, prm: O.Params, X: np.ndarray) -> np.ndarray:
    """Oracle-encoded integer plaintexts for values X [..., slots] -> int64 [..., N]."""
    flat = X.reshape(-1, X.shape[-1])
    return np.stack([ctx.encode(z, prm.scale) for z in flat]).reshape(X.shape[:-1] + (prm.N,))


def enc_rand_for(seed, config, clients, chunks, N):
    return S.enc_rand_batch(seed, config, clients, chunks, N)
