"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module draws random numbers and builds workload shapes; it holds none of the
method's arithmetic (no encoding, no modular reduction beyond drawing a uniform residue
below a given modulus, no NTT).  Both implementations receive exactly the same draws,
so encryption and key-generation randomness is an *input* to each of them.

Generator: numpy PCG64 seeded by SeedSequence([seed, config, job, client, chunk, purpose]).

Distributions (the paper only names X_key and X_err, Section "CKKS Scheme Description"):
  * secret / encryption ephemeral r: uniform ternary {-1, 0, +1}, each with probability 1/3;
  * error e: N(0, 3.2^2) rounded half-to-even, redrawn where |e| > 19 (about 6 sigma);
  * "a" polynomials: independent uniform residues in [0, q) per RNS limb, given in the
    coefficient domain (uniform over R_QP by CRT).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Iterable, Sequence

import numpy as np

# purpose tags for SeedSequence (stable numbers; never reorder)
P_UPDATE = 1
P_SK = 2
P_PK_A = 3
P_PK_E = 4
P_SWK_A = 5
P_SWK_E = 6
P_ENC_R = 7
P_ENC_E0 = 8
P_ENC_E1 = 9
P_BYZ = 10
P_JOB = 11
P_ARRIVAL = 12

# chunk index used for the per-client mask ciphertext's encryption randomness
MASK_CHUNK = 1 << 20

# configuration numbers used in the seed sequence
CFG_TOY = 1
CFG_PLAIN = 2
CFG_BATCHED = 3
CFG_UNEVEN = 4
CFG_SERVING = 5

SIGMA = 3.2
ERR_BOUND = 19


def rng(seed: int, config: int, job: int, client: int, chunk: int, purpose: int) -> np.random.Generator:
    ss = np.random.SeedSequence([int(seed), int(config), int(job), int(client), int(chunk), int(purpose)])
    return np.random.Generator(np.random.PCG64(ss))


def ternary(g: np.random.Generator, n: int) -> np.ndarray:
    """Uniform ternary vector in {-1, 0, 1} (int8)."""
    return (g.integers(0, 3, size=n, dtype=np.int64) - 1).astype(np.int8)


def gaussian_error(g: np.random.Generator, n: int, sigma: float = SIGMA, bound: int = ERR_BOUND) -> np.ndarray:
    """Rounded Gaussian (ties to even), redrawn beyond |e| > bound (int32)."""
    out = np.rint(g.normal(0.0, sigma, size=n))
    bad = np.abs(out) > bound
    while bad.any():
        out[bad] = np.rint(g.normal(0.0, sigma, size=int(bad.sum())))
        bad = np.abs(out) > bound
    return out.astype(np.int32)


def uniform_residues(g: np.random.Generator, moduli: Sequence[int], n: int) -> np.ndarray:
    """[len(moduli)][n] uint64, row i uniform in [0, moduli[i])."""
    out = np.empty((len(moduli), n), dtype=np.uint64)
    for i, q in enumerate(moduli):
        out[i] = g.integers(0, int(q), size=n, dtype=np.uint64)
    return out


# ---------------------------------------------------------------------------------------
# key / encryption randomness bundles
# ---------------------------------------------------------------------------------------

def secret_key(seed: int, config: int, n: int, job: int = 0) -> np.ndarray:
    return ternary(rng(seed, config, job, 0, 0, P_SK), n)


def pk_rand(seed: int, config: int, q_moduli: Sequence[int], n: int, job: int = 0):
    a = uniform_residues(rng(seed, config, job, 0, 0, P_PK_A), q_moduli, n)
    e = gaussian_error(rng(seed, config, job, 0, 0, P_PK_E), n)
    return a, e


def key_id(rotation: int | None) -> int:
    """0 for the relinearisation key, r+1 for the rotation key of left-rotation r."""
    return 0 if rotation is None else int(rotation) + 1


def swk_rand(seed: int, config: int, qp_moduli: Sequence[int], dnum: int, n: int,
             rotation: int | None, job: int = 0):
    """Randomness of one switching key: a [dnum][len(qp)][n] (coefficient domain), e [dnum][n]."""
    kid = key_id(rotation)
    a = np.stack([uniform_residues(rng(seed, config, job, kid, j, P_SWK_A), qp_moduli, n) for j in range(dnum)])
    e = np.stack([gaussian_error(rng(seed, config, job, kid, j, P_SWK_E), n) for j in range(dnum)])
    return a, e


def enc_rand(seed: int, config: int, client: int, chunk: int, n: int, job: int = 0):
    """(r, e0, e1) for one encryption: r ternary int8, e0/e1 int32."""
    r = ternary(rng(seed, config, job, client, chunk, P_ENC_R), n)
    e0 = gaussian_error(rng(seed, config, job, client, chunk, P_ENC_E0), n)
    e1 = gaussian_error(rng(seed, config, job, client, chunk, P_ENC_E1), n)
    return r, e0, e1


def enc_rand_batch(seed: int, config: int, clients: Iterable[int], chunks: Iterable[int], n: int, job: int = 0):
    """Stacked (r [B][n] int8, e0 [B][n] int32, e1 [B][n] int32) in (client, chunk) row-major order."""
    rs, e0s, e1s = [], [], []
    chunks = list(chunks)
    for c in clients:
        for k in chunks:
            r, e0, e1 = enc_rand(seed, config, c, k, n, job)
            rs.append(r); e0s.append(e0); e1s.append(e1)
    return np.stack(rs), np.stack(e0s), np.stack(e1s)


# ---------------------------------------------------------------------------------------
# workloads (shapes from the paper's evaluation setup; values synthetic)
# ---------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    config: int
    log_n: int            # ring degree N = 2^log_n; slots = N/2
    n_clients: int
    d: int                # model length (fp64 values per client)
    seed: int
    byzantine: tuple      # client indices
    byz_rule: str         # "scale10", "flip5", "noise0.1", "scale5"
    n_select: int         # clients the KGC keeps (Krum: 1; Multi-Krum: l)
    f: int                # assumed Byzantine count for Krum scores
    job: int = 0

    @property
    def slots(self) -> int:
        return 1 << (self.log_n - 1)

    @property
    def chunks(self) -> int:
        return max(1, math.ceil(self.d / self.slots))

    @property
    def n_pairs(self) -> int:
        return self.n_clients * (self.n_clients - 1) // 2


TOY = Workload("toy_N4096_n4", CFG_TOY, 12, 4, 2048, 0, (3,), "scale10", 1, 1)
PLAIN = Workload("plain_N32768_n10_d2^20", CFG_PLAIN, 15, 10, 1 << 20, 0, (8, 9), "flip5", 6, 2)
BATCHED = Workload("batched_N32768_n50_d2^22", CFG_BATCHED, 15, 50, 1 << 22, 1,
                   tuple(range(40, 50)), "noise0.1", 6, 10)


def client_updates(w: Workload, clients: Iterable[int] | None = None) -> np.ndarray:
    """[len(clients)][d] float64 updates ~ N(0, 0.01^2) with the workload's Byzantine rule."""
    clients = list(range(w.n_clients)) if clients is None else list(clients)
    out = np.empty((len(clients), w.d), dtype=np.float64)
    for row, c in enumerate(clients):
        x = rng(w.seed, w.config, w.job, c, 0, P_UPDATE).normal(0.0, 0.01, size=w.d)
        if c in w.byzantine:
            if w.byz_rule == "scale10":
                x = x * 10.0
            elif w.byz_rule == "flip5":
                x = x * -5.0
            elif w.byz_rule == "scale5":
                x = x * 5.0
            elif w.byz_rule == "noise0.1":
                x = x + rng(w.seed, w.config, w.job, c, 0, P_BYZ).normal(0.0, 0.1, size=w.d)
            else:
                raise ValueError(w.byz_rule)
        out[row] = x
    return out


def uneven_jobs(seed: int = 2, n_jobs: int = 8):
    """Job list of the uneven batch: n ~ U{5,10,20,40}, d ~ U{2^16,2^18,2^20,2^22}, 20% Byzantine x5."""
    g = rng(seed, CFG_UNEVEN, 0, 0, 0, P_JOB)
    jobs = []
    for j in range(n_jobs):
        n = int(g.choice([5, 10, 20, 40]))
        d = int(g.choice([1 << 16, 1 << 18, 1 << 20, 1 << 22]))
        nb = n // 5
        jobs.append(Workload(f"uneven_job{j}_n{n}_d{d}", CFG_UNEVEN, 15, n, d, seed,
                             tuple(range(n - nb, n)), "scale5", max(1, n - 2 * nb - 3), nb, job=j))
    return jobs


def split_chunks(x: np.ndarray, slots: int) -> np.ndarray:
    """[d] -> [chunks][slots], zero padded."""
    chunks = max(1, math.ceil(x.shape[-1] / slots))
    out = np.zeros(x.shape[:-1] + (chunks * slots,), dtype=np.float64)
    out[..., : x.shape[-1]] = x
    return out.reshape(x.shape[:-1] + (chunks, slots))


@dataclasses.dataclass(frozen=True)
class ServingRound:
    rid: int
    arrival: float        # seconds from the start of the run
    tenant: int
    n_clients: int
    d: int


def serving_rounds(seed: int = 3, n_rounds: int = 1000, rate: float = 1.0, tenants: int = 4,
                   sizes=(5, 10, 20, 40), lengths=(1 << 16, 1 << 18, 1 << 20, 1 << 22)):
    """Round stream of the serving workload: Poisson arrivals at `rate` per second, tenant
    uniform over `tenants`, n uniform over `sizes`, d uniform over `lengths` (the uneven-batch
    size distribution).  The draws depend on (seed, n_rounds index) only, not on the rate:
    inter-arrival gaps are unit exponentials divided by the rate."""
    g = rng(seed, CFG_SERVING, 0, 0, 0, P_ARRIVAL)
    gaps = g.exponential(1.0, size=n_rounds)
    ten = g.integers(0, tenants, size=n_rounds)
    ns = g.choice(np.asarray(sizes), size=n_rounds)
    ds = g.choice(np.asarray(lengths), size=n_rounds)
    t = np.cumsum(gaps) / rate
    return [ServingRound(i, float(t[i]), int(ten[i]), int(ns[i]), int(ds[i])) for i in range(n_rounds)]
