"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle, bit for bit in the
coefficient domain, plus decrypted accuracy against FP64.  Every oracle input is built from
the shared seeded generators and the oracle's own encoder/encryptor."""
import math

import numpy as np
import pytest

import oracle as O
import synth as S
from common import KeySet, plaintexts

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(kind):
    from paper_2408_06197_b300 import lancelot as LC
    return LC.Context.toy() if kind == "toy" else LC.Context.production()


class Env:
    def __init__(self, kind, seed, config, extra_rot=()):
        from paper_2408_06197_b300 import lancelot as LC
        self.LC = LC
        self.kind = kind
        self.prm = O.params_toy() if kind == "toy" else O.params_production()
        self.o = O.Context(self.prm)
        self.g = _ctx(kind)
        self.sched = O.default_schedule(self.prm.slots)
        rots = sorted(set(O.rotations_of_schedule(self.sched)) | set(extra_rot))
        self.keys = KeySet(self.prm, seed, config, rots)
        self.opk, self.orlk, self.ork = self.keys.oracle_keys(self.o)
        self.gpk, self.gevk = self.keys.gpu_keys(self.g)
        self.seed, self.config = seed, config
        self.N, self.L = self.prm.N, self.prm.L

    def g_coeff(self, t, level):
        return self.LC.torch_to_u64(self.g.to_coeff(t, level))

    def o_coeff(self, a):
        return self.o.to_coeff(a)

    def encrypt_both(self, X, clients, chunks):
        """X [n][chunks][slots] -> (oracle cts, gpu cts) of the same integer plaintexts."""
        m = plaintexts(self.o, self.prm, X)
        r, e0, e1 = S.enc_rand_batch(self.seed, self.config, clients, chunks, self.N)
        flat_m = m.reshape(-1, self.N)
        ocs = np.stack([self.o.encrypt(self.opk, flat_m[k], r[k], e0[k], e1[k]) for k in range(flat_m.shape[0])])
        gcs = self.g.encrypt(self.gpk, flat_m, r, e0, e1)
        shape = X.shape[:-1] + (2, self.prm.L + 1, self.N)
        return ocs.reshape(shape), gcs.reshape(shape)


@pytest.fixture(scope="module")
def toy():
    return Env("toy", S.TOY.seed, S.TOY.config, extra_rot=(3, 6, 12))


@pytest.fixture(scope="module")
def prod():
    return Env("prod", 0, S.CFG_PLAIN)


@pytest.fixture(params=["toy", "prod"])
def env(request, toy, prod):
    return toy if request.param == "toy" else prod


# ------------------------------------------------------------------------------- transforms

def test_ntt_roundtrip_and_negacyclic_product(env):
    rng = np.random.default_rng(1)
    nl = env.L + 1
    a = np.stack([rng.integers(0, q, size=env.N, dtype=np.uint64) for q in env.prm.q])
    b = np.stack([rng.integers(0, q, size=env.N, dtype=np.uint64) for q in env.prm.q])
    ga, gb = env.LC.u64_to_torch(a), env.LC.u64_to_torch(b)
    ea, eb = env.g.to_eval(ga, env.L), env.g.to_eval(gb, env.L)
    assert np.array_equal(env.g_coeff(ea, env.L), a)
    # tensor of (a, 0) and (b, 0): first output is a*b in Z_q[X]/(X^N+1)
    z = torch.zeros_like(ea)
    t = env.g.tensor(torch.stack([ea, z]).contiguous(), torch.stack([eb, z]).contiguous(), env.L)
    prod_coef = env.g_coeff(t[0].contiguous(), env.L)
    for i in (0, nl - 1):
        assert np.array_equal(prod_coef[i], env.o.poly_mul(i, a[i], b[i]))


def _extreme_polys(prm, N):
    """Inputs at the edges of the residue range: all q - 1, alternating 0 / q - 1, a single
    spike, and values in the top 2^10 of [0, q) -- the largest intermediate values a lazy
    transform sees, where a quotient estimate that falls short matters most."""
    rng = np.random.default_rng(11)
    out = []
    for kind in range(4):
        rows = []
        for q in prm.q:
            q = np.uint64(q)
            if kind == 0:
                v = np.full(N, q - np.uint64(1), dtype=np.uint64)
            elif kind == 1:
                v = np.where(np.arange(N) % 2 == 0, np.uint64(0), q - np.uint64(1)).astype(np.uint64)
            elif kind == 2:
                v = np.zeros(N, dtype=np.uint64)
                v[N // 3] = q - np.uint64(1)
            else:
                v = q - np.uint64(1) - rng.integers(0, 1 << 10, size=N, dtype=np.uint64)
            rows.append(v)
        out.append(np.stack(rows))
    return out


def _check_extreme_transforms(LC, g, o, prm):
    L = len(prm.q) - 1
    polys = _extreme_polys(prm, prm.N)
    evals = []
    for a in polys:
        e = g.to_eval(LC.u64_to_torch(a), L)
        eh = LC.torch_to_u64(e)
        assert all((eh[i] < np.uint64(q)).all() for i, q in enumerate(prm.q))
        assert np.array_equal(LC.torch_to_u64(g.to_coeff(e, L)), a)
        # the same words read as an evaluation vector: inverse, then forward, returns them
        v = LC.u64_to_torch(a)
        assert np.array_equal(LC.torch_to_u64(g.to_eval(g.to_coeff(v, L), L)), a)
        evals.append(e)
    z = torch.zeros_like(evals[0])
    for ia, ib in ((0, 0), (0, 1), (1, 3), (2, 3)):
        t = g.tensor(torch.stack([evals[ia], z]).contiguous(), torch.stack([evals[ib], z]).contiguous(), L)
        prod = LC.torch_to_u64(g.to_coeff(t[0].contiguous(), L))
        for i in range(L + 1):
            assert np.array_equal(prod[i], o.poly_mul(i, polys[ia][i], polys[ib][i])), (ia, ib, i)


def test_ntt_extreme_inputs(env):
    """Transforms of extreme vectors, where the lazy ranges are widest: forward outputs are
    canonical and invert exactly; extreme evaluation vectors survive inverse-then-forward; and
    the negacyclic product of two extreme polynomials (forward, pointwise, inverse) equals the
    oracle's product in every limb.  (The two sides' evaluation orders and roots differ, so
    evaluation vectors are not compared across them.)"""
    _check_extreme_transforms(env.LC, env.g, env.o, env.prm)


@pytest.mark.parametrize("log_n", [15, 16])
def test_ntt_extreme_inputs_at_the_lazy_limit(log_n):
    """The same checks with 46-bit primes, the largest that the transforms run without in-network
    reductions and with the three-product quotient (forward values up to 68q before the final
    reduction), at N = 2^15 and 2^16 (16 stages, the widest ranges)."""
    from paper_2408_06197_b300 import lancelot as LC
    q = O.gen_primes(log_n, 60, 0, 1) + O.gen_primes(log_n, 46, 0, 3)
    p = O.gen_primes(log_n, 60, 1, 1)
    assert all((1 << 45) < x < (1 << 46) for x in q[1:])
    prm = O.Params(log_n, q, p, 4, float(2 ** 40))
    _check_extreme_transforms(LC, LC.Context(log_n, q, p, 4, float(2 ** 40)), O.Context(prm), prm)


def test_encoder_matches_oracle(env):
    z = np.random.default_rng(2).normal(0, 0.01, env.prm.slots)
    mg = env.g.encode(z, env.prm.scale)
    mo = env.o.encode(z, env.prm.scale)
    diff = np.abs(mg - mo)
    assert diff.max() <= 1 and np.count_nonzero(diff) <= 2
    back = env.g.decode(mo.astype(np.float64), env.prm.scale)
    assert np.abs(back - z).max() <= 0.5 * env.N / env.prm.scale


# ------------------------------------------------------------------------------- keys, enc, dec

def test_keys_bit_exact(env):
    assert np.array_equal(env.g_coeff(env.gpk, env.L), env.o_coeff(env.opk))
    assert np.array_equal(env.gevk.export(None), env.o.key_to_coeff(env.orlk))
    r = env.sched and O.rotations_of_schedule(env.sched)[3]
    assert np.array_equal(env.gevk.export(r), env.o.key_to_coeff(env.ork[r]))


def test_key_set_restored_from_export_gives_identical_distances(toy):
    """Checkpoint / restore of a key set without the secret: every key exported in canonical form
    and imported into a fresh set exports the same words and gives bit-identical distances with
    the one-ModDown schedule; a non-canonical residue is rejected."""
    LC, g = toy.LC, toy.g
    fresh = g.evk()
    fresh.import_key(None, toy.gevk.export(None))
    for r in toy.gevk.rotations:
        fresh.import_key(r, toy.gevk.export(r))
    r0 = toy.gevk.rotations[0]
    assert np.array_equal(fresh.export(r0), toy.gevk.export(r0))
    X = S.split_chunks(S.client_updates(S.Workload("ck", S.CFG_TOY, 12, 3, toy.prm.slots, 9, (2,), "scale10", 1, 1)),
                       toy.prm.slots)
    _, gcs = toy.encrypt_both(X, range(3), range(1))
    sched = [2] + [1] * (len(toy.sched) - 2)
    mode = LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM
    a, _ = g.distances(toy.gevk, gcs, 3, 1, toy.prm.scale, mode=mode, groups=sched)
    b, _ = g.distances(fresh, gcs, 3, 1, toy.prm.scale, mode=mode, groups=sched)
    assert torch.equal(a, b)
    bad = toy.gevk.export(None)
    bad[0, 1, 0, 5] = toy.prm.q[0]
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):
        g.evk().import_key(None, bad)


def test_encrypt_decrypt_bit_exact(env):
    X = np.random.default_rng(3).normal(0, 0.01, (2, 1, env.prm.slots))
    ocs, gcs = env.encrypt_both(X, [0, 1], [0])
    for i in range(2):
        assert np.array_equal(env.g_coeff(gcs[i, 0].contiguous(), env.L), env.o_coeff(ocs[i, 0]))
    res_g = env.g.decrypt_residues(env.keys.s, gcs[0, 0].contiguous(), env.L)
    res_o = env.o.decrypt_residues(env.keys.s, ocs[0, 0], env.L)
    assert np.array_equal(res_g, res_o)
    zg = env.g.decrypt(env.keys.s, gcs[0, 0].contiguous(), env.L, env.prm.scale)
    # fresh noise: about 1e-7 per slot (production), 1e-5 (toy); max over all slots ~5 sigma
    assert np.abs(zg - X[0, 0]).max() < (1e-4 if env.kind == "toy" else 1e-6)


# ------------------------------------------------------------------------------- primitives

def test_sub_tensor_relin_rescale_bit_exact(env):
    X = np.random.default_rng(4).normal(0, 0.01, (2, 1, env.prm.slots))
    ocs, gcs = env.encrypt_both(X, [0, 1], [0])
    L = env.L
    od = env.o.sub(ocs[0, 0], ocs[1, 0], L)
    gd = env.g.sub(gcs[0, 0].contiguous(), gcs[1, 0].contiguous(), L)
    assert np.array_equal(env.g_coeff(gd, L), env.o_coeff(od))
    o3 = env.o.tensor(od, od, L)
    g3 = env.g.tensor(gd, gd, L)
    assert np.array_equal(env.g_coeff(g3, L), env.o_coeff(o3))
    o2 = env.o.relin(o3, L, env.orlk)
    g2 = env.g.relin(env.gevk, g3, L)[0]
    assert np.array_equal(env.g_coeff(g2, L), env.o_coeff(o2))
    orr = env.o.rescale(o2, L)
    grr = env.g.rescale(g2.contiguous(), L)[0]
    assert np.array_equal(env.g_coeff(grr, L - 1), env.o_coeff(orr))
    sc = env.prm.scale ** 2 / env.prm.q[L]
    dz = X[0, 0] - X[1, 0]
    assert np.abs(env.g.decrypt(env.keys.s, grr, L - 1, sc) - dz * dz).max() < (1e-4 if env.kind == "toy" else 5e-7)


def test_hoisted_rotations_and_rotate_sum_bit_exact(env):
    X = np.random.default_rng(5).normal(0, 0.01, (1, 1, env.prm.slots))
    ocs, gcs = env.encrypt_both(X, [0], [0])
    L = env.L
    rots = [1, 2, 4] if env.kind == "prod" else [1, 3, 6, 12]
    outs_o = env.o.rotate_hoisted(ocs[0, 0], L, rots, [env.ork[r] for r in rots])
    outs_g = env.g.rotate(env.gevk, gcs[0, 0].contiguous(), L, rots)
    for k, r in enumerate(rots):
        assert np.array_equal(env.g_coeff(outs_g[k].contiguous(), L), env.o_coeff(outs_o[k]))
    z = env.g.decrypt(env.keys.s, outs_g[0].contiguous(), L, env.prm.scale)
    assert np.abs(z - np.roll(X[0, 0], -rots[0])).max() < (2e-4 if env.kind == "toy" else 2e-6)
    # rotate-and-sum: log-step, and (toy) a hoisted group of size 2
    scheds = [env.sched] + ([[2] + [1] * (len(env.sched) - 2)] if env.kind == "toy" else [])
    for sched in scheds:
        need = O.rotations_of_schedule(sched)
        yo = env.o.rotate_sum(ocs[0, 0], L, sched, {r: env.ork[r] for r in need})
        yg = env.g.rotate_sum(env.gevk, gcs[0, 0].contiguous(), L, sched)
        assert np.array_equal(env.g_coeff(yg, L), env.o_coeff(yo))


def test_qp_sum_hoisting_bit_exact_toy(toy):
    X = np.random.default_rng(6).normal(0, 0.01, (1, 1, toy.prm.slots))
    ocs, gcs = toy.encrypt_both(X, [0], [0])
    sched = [2] + [1] * (len(toy.sched) - 2)
    need = O.rotations_of_schedule(sched)
    yo = toy.o.rotate_sum(ocs[0, 0], toy.L, sched, {r: toy.ork[r] for r in need}, qp_sum=True)
    yg = toy.g.rotate_sum(toy.gevk, gcs[0, 0].contiguous(), toy.L, sched, qp_sum=True)
    assert np.array_equal(toy.g_coeff(yg, toy.L), toy.o_coeff(yo))


def test_qp_sum_groups_of_seven_bit_exact_toy():
    """One-ModDown groups of 7 rotations ([3, 3, 3, 2] at 2^11 slots): the fused group kernel at
    its largest size, against the oracle, for a single ciphertext and for batched distances."""
    sched = [3, 3, 3, 2]
    e = Env("toy", 11, S.CFG_TOY, extra_rot=O.rotations_of_schedule(sched))
    X = np.random.default_rng(8).normal(0, 0.01, (1, 1, e.prm.slots))
    ocs, gcs = e.encrypt_both(X, [0], [0])
    need = O.rotations_of_schedule(sched)
    yo = e.o.rotate_sum(ocs[0, 0], e.L, sched, {r: e.ork[r] for r in need}, qp_sum=True)
    yg = e.g.rotate_sum(e.gevk, gcs[0, 0].contiguous(), e.L, sched, qp_sum=True)
    assert np.array_equal(e.g_coeff(yg, e.L), e.o_coeff(yo))
    w = S.Workload("t5g3", S.CFG_TOY, 12, 5, 2 * e.prm.slots - 9, 11, (4,), "scale10", 1, 1)
    W = S.client_updates(w)
    ocs, gcs = e.encrypt_both(S.split_chunks(W, e.prm.slots), range(5), range(2))
    Dg, _ = e.g.distances(e.gevk, gcs, 5, 2, e.prm.scale, mode=e.LC.LC_MODE_BATCHED | e.LC.LC_HOIST_QP_SUM,
                          groups=sched)
    Do = e.o.distances(ocs, e.orlk, sched, e.ork, qp_sum=True)
    assert np.array_equal(e.g_coeff(Dg, e.L - 1), e.o_coeff(Do))


def test_qp_sum_groups_of_fifteen_bit_exact_toy():
    """One-ModDown groups of 15 rotations ([4, 4, 3] at 2^11 slots; the largest group the fused
    kernel takes), against the oracle: a rotate-and-sum, batched distances, and the uneven
    multi-job path with per-item key tables."""
    sched = [4, 4, 3]
    e = Env("toy", 13, S.CFG_TOY, extra_rot=O.rotations_of_schedule(sched))
    LC = e.LC
    X = np.random.default_rng(9).normal(0, 0.01, (1, 1, e.prm.slots))
    ocs, gcs = e.encrypt_both(X, [0], [0])
    need = O.rotations_of_schedule(sched)
    yo = e.o.rotate_sum(ocs[0, 0], e.L, sched, {r: e.ork[r] for r in need}, qp_sum=True)
    yg = e.g.rotate_sum(e.gevk, gcs[0, 0].contiguous(), e.L, sched, qp_sum=True)
    assert np.array_equal(e.g_coeff(yg, e.L), e.o_coeff(yo))
    w = S.Workload("t4g4", S.CFG_TOY, 12, 4, 2 * e.prm.slots - 9, 13, (3,), "scale10", 1, 1)
    W = S.client_updates(w)
    ocs, gcs = e.encrypt_both(S.split_chunks(W, e.prm.slots), range(4), range(2))
    mode = LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM
    Dg, sc = e.g.distances(e.gevk, gcs, 4, 2, e.prm.scale, mode=mode, groups=sched)
    Do = e.o.distances(ocs, e.orlk, sched, e.ork, qp_sum=True)
    assert np.array_equal(e.g_coeff(Dg, e.L - 1), e.o_coeff(Do))
    from test_oracle_pins import toy_distance_tolerance
    v = e.g.decrypt(e.keys.s, Dg[0].contiguous(), e.L - 1, sc)
    assert np.abs(v - np.sum((W[0] - W[1]) ** 2)).max() <= toy_distance_tolerance(e.prm)
    job = LC.Job(e.gevk, gcs, 4, 2)
    LC.batch_distances(e.g, [job, LC.Job(e.gevk, gcs[:3].contiguous(), 3, 2)], LC.LC_HOIST_QP_SUM, sched)
    assert torch.equal(job.out_dist, Dg)
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):  # 5-bit one-ModDown groups: not supported
        e.g.rotate_sum(e.gevk, gcs[0, 0].contiguous(), e.L, [5, 4, 2], qp_sum=True)


@pytest.mark.slow
def test_qp_sum_groups_of_fifteen_production_bit_exact():
    """A schedule with groups of 4 rotation bits at N = 2^15 ([4,4,4,2], 48 rotation keys): the
    rotate-and-sum of a fresh ciphertext and the distances of 3 clients bit-exact against the
    oracle's one-ModDown groups, and the distances within 1e-5 of FP64."""
    sched = [4, 4, 4, 2]
    e = Env("prod", 6, S.CFG_PLAIN, extra_rot=O.rotations_of_schedule(sched))
    LC = e.LC
    X = np.random.default_rng(10).normal(0, 0.01, (1, 1, e.prm.slots))
    ocs, gcs = e.encrypt_both(X, [0], [0])
    need = O.rotations_of_schedule(sched)
    yo = e.o.rotate_sum(ocs[0, 0], e.L, sched, {r: e.ork[r] for r in need}, qp_sum=True)
    yg = e.g.rotate_sum(e.gevk, gcs[0, 0].contiguous(), e.L, sched, qp_sum=True)
    assert np.array_equal(e.g_coeff(yg, e.L), e.o_coeff(yo))
    w = S.Workload("p3g4", S.CFG_PLAIN, 15, 3, e.prm.slots + 5, 6, (2,), "flip5", 1, 0)
    W = S.client_updates(w)
    ocs, gcs = e.encrypt_both(S.split_chunks(W, e.prm.slots), range(3), range(w.chunks))
    Dg, sc = e.g.distances(e.gevk, gcs, 3, w.chunks, e.prm.scale, mode=LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM,
                           groups=sched)
    Do = e.o.distances(ocs, e.orlk, sched, e.ork, qp_sum=True)
    assert np.array_equal(e.g_coeff(Dg, e.L - 1), e.o_coeff(Do))
    k = 0
    for i in range(3):
        for j in range(i + 1, 3):
            ref = np.sum((W[i] - W[j]) ** 2)
            assert abs(e.g.decrypt(e.keys.s, Dg[k].contiguous(), e.L - 1, sc)[0] - ref) / ref < 1e-5
            k += 1


@pytest.fixture(scope="module")
def prod_g2():
    """Production parameters with the rotation keys of the hoisting schedule [2]*7 (21 keys)."""
    e = Env.__new__(Env)
    from paper_2408_06197_b300 import lancelot as LC
    e.LC, e.kind = LC, "prod"
    e.prm = O.params_production()
    e.o = O.Context(e.prm)
    e.g = _ctx("prod")
    e.sched = [2] * 7
    e.keys = KeySet(e.prm, 4, S.CFG_PLAIN, O.rotations_of_schedule(e.sched))
    e.opk, e.orlk, e.ork = e.keys.oracle_keys(e.o)
    e.gpk, e.gevk = e.keys.gpu_keys(e.g)
    e.seed, e.config = 4, S.CFG_PLAIN
    e.N, e.L = e.prm.N, e.prm.L
    return e


G3QP = [3, 3, 3, 3, 2]  # the benchmark's rotation schedule at N = 2^15 (autotuner's pick)


@pytest.fixture(scope="module")
def prod_g3():
    """Production parameters with the keys of the benchmark's schedule [3,3,3,3,2] (31 keys, a
    superset of the 14 log-step keys)."""
    e = Env.__new__(Env)
    from paper_2408_06197_b300 import lancelot as LC
    e.LC, e.kind = LC, "prod"
    e.prm = O.params_production()
    e.o = O.Context(e.prm)
    e.g = _ctx("prod")
    e.sched = G3QP
    e.keys = KeySet(e.prm, 0, S.CFG_PLAIN, O.rotations_of_schedule(G3QP))
    e.opk, e.orlk, e.ork = e.keys.oracle_keys(e.o)
    e.gpk, e.gevk = e.keys.gpu_keys(e.g)
    e.seed, e.config = 0, S.CFG_PLAIN
    e.N, e.L = e.prm.N, e.prm.L
    return e


def test_level_drop_distances_bit_exact_toy(toy):
    """LC_ROTATE_AT_LEVEL(0): the rescaled pairs dropped to limb q_0 before the rotate-and-sum, in
    both modes, bit-exact against the oracle's dropped distances; LC_ELEVEL above L - 1."""
    LC = toy.LC
    w, W, X, ocs, gcs = _toy_inputs(toy)
    Do = toy.o.distances(ocs, toy.orlk, toy.sched, toy.ork, rot_level=0)
    for mode in (LC.LC_MODE_BATCHED, LC.LC_MODE_PER_OP):
        Dg, sc = toy.g.distances(toy.gevk, gcs, w.n_clients, w.chunks, toy.prm.scale, mode=mode, rot_level=0)
        assert Dg.shape == (w.n_pairs, 2, 1, toy.N)
        assert np.array_equal(toy.g_coeff(Dg, 0), toy.o_coeff(Do))
    with pytest.raises(LC.LancelotError, match="LC_ELEVEL"):
        toy.g.distances(toy.gevk, gcs, w.n_clients, w.chunks, toy.prm.scale, rot_level=toy.L)


def test_level_drop_distances_production_bit_exact(prod_g2):
    """At N = 2^15: pairs rescaled to level 13 and dropped to level 1 (q_0 q_1, 100 bits) before
    one-ModDown groups [2]*7, bit-exact against the oracle, every distance within 1e-5 of FP64."""
    e = prod_g2
    LC = e.LC
    w = S.Workload("p3drop", S.CFG_PLAIN, 15, 3, 2 * e.prm.slots - 50, 4, (2,), "flip5", 1, 0)
    W = S.client_updates(w)
    X = S.split_chunks(W, e.prm.slots)
    ocs, gcs = e.encrypt_both(X, range(3), range(w.chunks))
    mode = LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM
    Dg, sc = e.g.distances(e.gevk, gcs, 3, w.chunks, e.prm.scale, mode=mode, groups=e.sched, rot_level=1)
    Do = e.o.distances(ocs, e.orlk, e.sched, e.ork, qp_sum=True, rot_level=1)
    assert np.array_equal(e.g_coeff(Dg, 1), e.o_coeff(Do))
    k = 0
    for i in range(3):
        for j in range(i + 1, 3):
            ref = np.sum((W[i] - W[j]) ** 2)
            v = e.g.decrypt(e.keys.s, Dg[k].contiguous(), 1, sc)
            assert np.abs(v - ref).max() / ref < 1e-5
            assert abs(e.g.decrypt_const(e.keys.s, Dg[k:k + 1].contiguous(), 1, sc)[0] - ref) / ref < 1e-5
            k += 1


def test_qp_sum_distances_production_bit_exact(prod_g2):
    e = prod_g2
    w = S.Workload("p3g2", S.CFG_PLAIN, 15, 3, e.prm.slots, 4, (2,), "flip5", 1, 0)
    W = S.client_updates(w)
    X = S.split_chunks(W, e.prm.slots)
    ocs, gcs = e.encrypt_both(X, range(3), range(1))
    mode = e.LC.LC_MODE_BATCHED | e.LC.LC_HOIST_QP_SUM
    Dg, sc = e.g.distances(e.gevk, gcs, 3, 1, e.prm.scale, mode=mode, groups=e.sched)
    Do = e.o.distances(ocs, e.orlk, e.sched, e.ork, qp_sum=True)
    assert np.array_equal(e.g_coeff(Dg, e.L - 1), e.o_coeff(Do))
    Dp, _ = e.g.distances(e.gevk, gcs, 3, 1, e.prm.scale, mode=e.LC.LC_MODE_PER_OP | e.LC.LC_HOIST_QP_SUM,
                          groups=e.sched)
    assert torch.equal(Dg, Dp)
    k = 0
    for i in range(3):
        for j in range(i + 1, 3):
            ref = np.sum((W[i] - W[j]) ** 2)
            v = e.g.decrypt(e.keys.s, Dg[k].contiguous(), e.L - 1, sc)
            assert np.abs(v - ref).max() / ref < 1e-5
            k += 1


# ------------------------------------------------------------------------------- the method (toy)

def _toy_inputs(toy):
    w = S.TOY
    W = S.client_updates(w)
    X = S.split_chunks(W, toy.prm.slots)
    ocs, gcs = toy.encrypt_both(X, range(w.n_clients), range(w.chunks))
    return w, W, X, ocs, gcs


def test_toy_distances_bit_exact_both_modes_and_fp64(toy):
    from paper_2408_06197_b300 import kgc
    from test_oracle_pins import toy_distance_tolerance
    w, W, X, ocs, gcs = _toy_inputs(toy)
    toy.g.counters(reset=True)
    Dg, sc = toy.g.distances(toy.gevk, gcs, w.n_clients, w.chunks, toy.prm.scale, mode=toy.LC.LC_MODE_BATCHED)
    ks, mu = toy.g.counters(reset=True)
    assert ks == w.n_pairs * (1 + len(toy.sched)) and mu == ks
    Dp, _ = toy.g.distances(toy.gevk, gcs, w.n_clients, w.chunks, toy.prm.scale, mode=toy.LC.LC_MODE_PER_OP)
    assert torch.equal(Dg, Dp)
    Do = toy.o.distances(ocs, toy.orlk, toy.sched, toy.ork)
    assert np.array_equal(toy.g_coeff(Dg, toy.L - 1), toy.o_coeff(Do))
    tol = toy_distance_tolerance(toy.prm)
    dist = np.zeros((w.n_clients, w.n_clients))
    k = 0
    for i in range(w.n_clients):
        for j in range(i + 1, w.n_clients):
            v = toy.g.decrypt(toy.keys.s, Dg[k].contiguous(), toy.L - 1, sc)
            assert np.abs(v - np.sum((W[i] - W[j]) ** 2)).max() <= tol
            dist[i, j] = dist[j, i] = v[0]
            k += 1
    ref = np.array([[np.sum((W[i] - W[j]) ** 2) for j in range(w.n_clients)] for i in range(w.n_clients)])
    assert kgc.krum_select(dist, w.f, w.n_select) == kgc.krum_select(ref, w.f, w.n_select)


def test_toy_masked_aggregate_bit_exact(toy):
    from paper_2408_06197_b300 import kgc
    w, W, X, ocs, gcs = _toy_inputs(toy)
    sel = [0]
    wts = kgc.mask_weights(w.n_clients, sel, average=False)
    MX = np.stack([np.full((1, toy.prm.slots), wts[i]) for i in range(w.n_clients)])
    m = plaintexts(toy.o, toy.prm, MX)[:, 0]
    r, e0, e1 = S.enc_rand_batch(w.seed, w.config, range(w.n_clients), [S.MASK_CHUNK], toy.N)
    om = np.stack([toy.o.encrypt(toy.opk, m[i], r[i], e0[i], e1[i]) for i in range(w.n_clients)])
    gm = toy.g.encrypt(toy.gpk, m, r, e0, e1)
    for mode in (toy.LC.LC_MODE_BATCHED, toy.LC.LC_MODE_PER_OP):
        ag, sc = toy.g.masked_aggregate(toy.gevk, gcs, w.n_clients, w.chunks, toy.prm.scale, gm, toy.prm.scale,
                                        mode=mode)
        ao = toy.o.masked_aggregate(ocs, om, toy.orlk)
        assert np.array_equal(toy.g_coeff(ag, toy.L - 1), toy.o_coeff(ao))
    got = toy.g.decrypt(toy.keys.s, ag[0].contiguous(), toy.L - 1, sc)
    assert np.linalg.norm(got - X[0, 0]) / np.linalg.norm(X[0, 0]) < 1e-3


def test_batched_waves_match_single_wave(toy):
    w, W, X, ocs, gcs = _toy_inputs(toy)
    D1, _ = toy.g.distances(toy.gevk, gcs, w.n_clients, w.chunks, toy.prm.scale)
    toy.g.set_max_batch(4)  # 6 pairs -> waves of 4 and 2
    try:
        D2, _ = toy.g.distances(toy.gevk, gcs, w.n_clients, w.chunks, toy.prm.scale)
    finally:
        toy.g.set_max_batch(0)
    assert torch.equal(D1, D2)


def test_graph_replay_matches_direct_calls(toy):
    """A captured distances + aggregate step replays on new inputs written into the same buffers."""
    w, W, X, ocs, gcs = _toy_inputs(toy)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    from paper_2408_06197_b300 import lancelot as LC
    with torch.cuda.stream(stream):
        g = LC.Context.toy(stream=stream)
        pk, evk = toy.keys.gpu_keys(g)
        cts = gcs.clone()
        out_d = g.empty(w.n_pairs, 2, toy.L, toy.N)  # level L-1 ciphertexts have L limbs
        out_a = g.empty(w.chunks, 2, toy.L, toy.N)
        masks = gcs[:, 0].contiguous()

    def step():
        g.distances(evk, cts, w.n_clients, w.chunks, toy.prm.scale, out=out_d)
        g.masked_aggregate(evk, cts, w.n_clients, w.chunks, toy.prm.scale, masks, toy.prm.scale, out=out_a)

    with torch.cuda.stream(stream):
        step()
        graph = g.capture(step)
        cts.copy_(torch.flip(gcs, dims=[0]))  # new inputs in the captured buffer
        graph.launch()
        g.sync()
        got_d, got_a = out_d.clone(), out_a.clone()
        step()
        g.sync()
    assert torch.equal(got_d, out_d) and torch.equal(got_a, out_a)
    graph.close()


def test_host_buffers_match_device_buffers(toy):
    w, W, X, ocs, gcs = _toy_inputs(toy)
    host = toy.LC.torch_to_u64(gcs.contiguous())
    Dh, _ = toy.g.distances(toy.gevk, host, w.n_clients, w.chunks, toy.prm.scale)
    Dd, _ = toy.g.distances(toy.gevk, gcs, w.n_clients, w.chunks, toy.prm.scale)
    assert np.array_equal(Dh, toy.LC.torch_to_u64(Dd))


def test_edge_cases(toy):
    LC = toy.LC
    w, W, X, ocs, gcs = _toy_inputs(toy)
    # two clients: exactly one pair
    D2, _ = toy.g.distances(toy.gevk, gcs[:2].contiguous(), 2, 1, toy.prm.scale)
    D4, _ = toy.g.distances(toy.gevk, gcs, 4, 1, toy.prm.scale)
    assert torch.equal(D2[0], D4[0])
    with pytest.raises(LC.LancelotError):
        toy.g.distances(toy.gevk, gcs[:1].contiguous(), 1, 1, toy.prm.scale)
    empty = toy.g.evk()
    with pytest.raises(LC.LancelotError, match="LC_EKEY"):
        toy.g.distances(empty, gcs, 4, 1, toy.prm.scale)
    with pytest.raises(LC.LancelotError):
        toy.g.distances(toy.gevk, gcs, 4, 1, toy.prm.scale, groups=[1, 1])  # does not cover all slots
    for bad in (0.0, -1.0, float("nan"), float("inf")):  # malformed scale
        with pytest.raises(LC.LancelotError, match="LC_ESCALE"):
            toy.g.distances(toy.gevk, gcs, 4, 1, bad)
        with pytest.raises(LC.LancelotError, match="LC_ESCALE"):
            toy.g.masked_aggregate(toy.gevk, gcs, 4, 1, toy.prm.scale, gcs[:, 0].contiguous(), bad)


def _job_inputs(env, keys, w, seed_client0):
    W = S.client_updates(w)
    X = S.split_chunks(W, env.prm.slots)
    m = plaintexts(env.o, env.prm, X).reshape(-1, env.N)
    r, e0, e1 = S.enc_rand_batch(w.seed, w.config, range(w.n_clients), range(w.chunks), env.N, job=w.job)
    return W, X, m, r, e0, e1


def test_uneven_batch_matches_each_job_alone(toy):
    """Jobs with different client counts, chunk counts and tenants (key sets) batched together give
    each job exactly the results it gets alone (distances with the log-step and the one-ModDown
    schedules, and masked aggregates)."""
    LC = toy.LC
    g = toy.g
    keys_b = KeySet(toy.prm, 7, S.CFG_UNEVEN, O.rotations_of_schedule(toy.sched) + [3])
    _, evk_b = keys_b.gpu_keys(g)
    pk_b = g.pk_gen(keys_b.s, keys_b.pk_a, keys_b.pk_e)
    specs = [(3, 1, toy.gevk, toy.gpk, 0), (5, 3, evk_b, pk_b, 1), (2, 2, toy.gevk, toy.gpk, 2), (4, 2, evk_b, pk_b, 3),
             (2, 1, evk_b, pk_b, 4), (2, 3, toy.gevk, toy.gpk, 5), (2, 1, toy.gevk, toy.gpk, 6), (2, 2, evk_b, pk_b, 7)]
    jobs = []
    for n, chunks, evk, pk, jid in specs:
        w = S.Workload(f"u{jid}", S.CFG_UNEVEN, 12, n, chunks * toy.prm.slots - 7, 2, (n - 1,), "scale5", 1, 1, job=jid)
        W, X, m, r, e0, e1 = _job_inputs(toy, None, w, 0)
        cts = g.encrypt(pk, m, r, e0, e1).reshape(n, chunks, 2, toy.L + 1, toy.N)
        masks = g.encrypt(pk, m.reshape(n, chunks, -1)[:, 0].copy(), r.reshape(n, chunks, -1)[:, 0].copy(),
                          e0.reshape(n, chunks, -1)[:, 0].copy(), e1.reshape(n, chunks, -1)[:, 0].copy())
        jobs.append(LC.Job(evk, cts, n, chunks, masks))
    for sched, flags in ((None, 0), ([2] + [1] * (len(toy.sched) - 2), LC.LC_HOIST_QP_SUM)):
        for j in jobs:
            j.out_dist = None
        LC.batch_distances(g, jobs, LC.LC_MODE_BATCHED | flags, sched)
        for j in jobs:
            alone, _ = g.distances(j.evk, j.cts, j.n, j.chunks, toy.prm.scale, mode=LC.LC_MODE_BATCHED | flags,
                                   groups=sched)
            assert torch.equal(alone, j.out_dist)
    LC.batch_aggregate(g, jobs)
    for j in jobs:
        alone, _ = g.masked_aggregate(j.evk, j.cts, j.n, j.chunks, toy.prm.scale, j.masks, toy.prm.scale)
        assert torch.equal(alone, j.out_agg)
    # smaller waves: jobs with at least half a wave of pairs (chunks) run on their own, the others
    # share waves -- 4: the five single-pair jobs in two shared waves (and the single-chunk jobs'
    # aggregates in one), the rest alone; 8: the jobs of at most 3 pairs shared; 3: every job
    # alone.  Identical in every case.
    for cap in (4, 8, 3):
        g.set_max_batch(cap)
        try:
            for j in jobs:
                j.out_dist = j.out_agg = None
            LC.batch_distances(g, jobs)
            LC.batch_aggregate(g, jobs)
            for j in jobs:
                alone, _ = g.distances(j.evk, j.cts, j.n, j.chunks, toy.prm.scale)
                assert torch.equal(alone, j.out_dist)
                alone, _ = g.masked_aggregate(j.evk, j.cts, j.n, j.chunks, toy.prm.scale, j.masks, toy.prm.scale)
                assert torch.equal(alone, j.out_agg)
        finally:
            g.set_max_batch(0)


# ------------------------------------------------------------------------------- production sizes

def test_production_distances_small_bit_exact(prod):
    w = S.Workload("p3", S.CFG_PLAIN, 15, 3, 2 * prod.prm.slots - 100, 0, (2,), "flip5", 1, 0)
    W = S.client_updates(w)
    X = S.split_chunks(W, prod.prm.slots)   # ragged: the last chunk is zero padded
    ocs, gcs = prod.encrypt_both(X, range(3), range(w.chunks))
    Dg, sc = prod.g.distances(prod.gevk, gcs, 3, w.chunks, prod.prm.scale)
    Do = prod.o.distances(ocs, prod.orlk, prod.sched, prod.ork)
    assert np.array_equal(prod.g_coeff(Dg, prod.L - 1), prod.o_coeff(Do))
    k = 0
    for i in range(3):
        for j in range(i + 1, 3):
            ref = np.sum((W[i] - W[j]) ** 2)
            v = prod.g.decrypt(prod.keys.s, Dg[k].contiguous(), prod.L - 1, sc)
            assert abs(v[0] - ref) / ref < 1e-5
            k += 1


@pytest.mark.slow
def test_production_full_size_sampled(prod_g3):
    """Config of the benchmark in its launch configuration (n=10, d=2^20, 64 chunks, batched
    launches, one-ModDown groups [3,3,3,3,2]): every pair against FP64 and two sampled pairs + two
    sampled aggregate chunks bit-exact against the oracle."""
    from paper_2408_06197_b300 import kgc
    prod = prod_g3
    mode = prod.LC.LC_MODE_BATCHED | prod.LC.LC_HOIST_QP_SUM
    w = S.PLAIN
    W = S.client_updates(w)
    X = S.split_chunks(W, prod.prm.slots)
    m = plaintexts(prod.o, prod.prm, X)
    r, e0, e1 = S.enc_rand_batch(w.seed, w.config, range(w.n_clients), range(w.chunks), prod.N)
    gcs = prod.g.encrypt(prod.gpk, m.reshape(-1, prod.N), r, e0, e1).reshape(w.n_clients, w.chunks, 2, prod.L + 1,
                                                                               prod.N)
    Dg, sc = prod.g.distances(prod.gevk, gcs, w.n_clients, w.chunks, prod.prm.scale, mode=mode, groups=G3QP)
    dist = np.zeros((w.n_clients, w.n_clients))
    ref = np.zeros_like(dist)
    k = 0
    for i in range(w.n_clients):
        for j in range(i + 1, w.n_clients):
            v = prod.g.decrypt(prod.keys.s, Dg[k].contiguous(), prod.L - 1, sc)
            ref[i, j] = ref[j, i] = np.sum((W[i] - W[j]) ** 2)
            assert abs(v[0] - ref[i, j]) / ref[i, j] < 1e-5
            dist[i, j] = dist[j, i] = v[0]
            k += 1
    sel = kgc.krum_select(dist, w.f, w.n_select)
    assert sel == kgc.krum_select(ref, w.f, w.n_select) and not (set(sel) & set(w.byzantine))
    # sampled pairs bit-exact: (0,1) and (7,9) -> local clients
    clients = [0, 1, 7, 9]
    idx = {c: k for k, c in enumerate(clients)}
    ocs = np.stack([np.stack([prod.o.encrypt(prod.opk, m[c, k], r[c * w.chunks + k], e0[c * w.chunks + k],
                                             e1[c * w.chunks + k]) for k in range(w.chunks)]) for c in clients])
    pairs = [(0, 1), (7, 9)]
    Do = prod.o.distances(ocs, prod.orlk, G3QP, prod.ork, pairs=[(idx[i], idx[j]) for i, j in pairs], qp_sum=True)

    def pidx(i, j):
        return i * w.n_clients - i * (i + 1) // 2 + (j - i - 1)

    for t, (i, j) in enumerate(pairs):
        assert np.array_equal(prod.g_coeff(Dg[pidx(i, j)].contiguous(), prod.L - 1), prod.o_coeff(Do[t]))
    # masked aggregate of the selected clients, weights 1/l
    wts = kgc.mask_weights(w.n_clients, sel, average=True)
    mm = plaintexts(prod.o, prod.prm, np.stack([np.full((1, prod.prm.slots), wts[i]) for i in range(w.n_clients)]))[:, 0]
    rm, e0m, e1m = S.enc_rand_batch(w.seed, w.config, range(w.n_clients), [S.MASK_CHUNK], prod.N)
    gm = prod.g.encrypt(prod.gpk, mm, rm, e0m, e1m)
    Ag, asc = prod.g.masked_aggregate(prod.gevk, gcs, w.n_clients, w.chunks, prod.prm.scale, gm, prod.prm.scale)
    agg_ref = sum(wts[i] * W[i] for i in range(w.n_clients))
    got = np.concatenate([prod.g.decrypt(prod.keys.s, Ag[k].contiguous(), prod.L - 1, asc) for k in range(w.chunks)])
    assert np.linalg.norm(got - agg_ref) / np.linalg.norm(agg_ref) < 1e-5
    om = np.stack([prod.o.encrypt(prod.opk, mm[i], rm[i], e0m[i], e1m[i]) for i in range(w.n_clients)])
    for k in (0, w.chunks - 1):
        ock = np.stack([prod.o.encrypt(prod.opk, m[c, k], r[c * w.chunks + k], e0[c * w.chunks + k],
                                       e1[c * w.chunks + k]) for c in range(w.n_clients)])[:, None]
        Ao = prod.o.masked_aggregate(np.ascontiguousarray(ock), om, prod.orlk)
        assert np.array_equal(prod.g_coeff(Ag[k].contiguous(), prod.L - 1), prod.o_coeff(Ao[0]))


@pytest.mark.slow
def test_batched_config_full_size_sampled(prod_g3):
    """The batched configuration at full size (n=50, d=2^22: 256 ciphertexts per client, 94 GB
    resident, 1,225 pairs in waves) in the benchmark's launch configuration: every pair's
    read-out against FP64, Multi-Krum selection, and 18 sampled pairs bit-exact against the
    oracle (honest/honest, honest/noisy and noisy/noisy pairs)."""
    from paper_2408_06197_b300 import kgc
    e = prod_g3
    LC = e.LC
    w = S.BATCHED
    chunks, n = w.chunks, w.n_clients
    gcs = e.g.empty(n, chunks, 2, e.L + 1, e.N)
    sq = np.zeros((n, n))
    Ws = {}
    for i in range(n):
        Wi = S.client_updates(w, [i])[0]
        Ws[i] = Wi
        m = plaintexts(e.o, e.prm, S.split_chunks(Wi, e.prm.slots))
        r, e0, e1 = S.enc_rand_batch(w.seed, w.config, [i], range(chunks), e.N)
        e.g.encrypt(e.gpk, m, r, e0, e1, out=gcs[i].view(chunks, 2, e.L + 1, e.N))
    for i in range(n):
        for j in range(i + 1, n):
            sq[i, j] = sq[j, i] = np.sum((Ws[i] - Ws[j]) ** 2)
    Dg, sc = e.g.distances(e.gevk, gcs, n, chunks, e.prm.scale, mode=LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM,
                           groups=G3QP)
    got = e.g.decrypt_const(e.keys.s, Dg, e.L - 1, sc)
    dist = np.zeros((n, n))
    k = 0
    for i in range(n):
        for j in range(i + 1, n):
            assert abs(got[k] - sq[i, j]) / sq[i, j] < 1e-5
            dist[i, j] = dist[j, i] = got[k]
            k += 1
    sel = kgc.krum_select(dist, w.f, w.n_select)
    assert sel == kgc.krum_select(sq, w.f, w.n_select) and not (set(sel) & set(w.byzantine))
    # 18 sampled pairs bit-exact: every pair inside three groups of four clients, spread over the
    # client range, honest and noisy (40-49) -- a group at a time, so that the oracle holds the
    # 256-chunk ciphertexts of four clients (8 GB) at most
    compared = 0
    for group in ((0, 3, 41, 45), (17, 29, 47, 49), (5, 12, 33, 44)):
        ocs = []
        for c in group:
            m = plaintexts(e.o, e.prm, S.split_chunks(Ws[c], e.prm.slots))
            r, e0, e1 = S.enc_rand_batch(w.seed, w.config, [c], range(chunks), e.N)
            ocs.append(np.stack([e.o.encrypt(e.opk, m[k], r[k], e0[k], e1[k]) for k in range(chunks)]))
        local = [(a, b) for a in range(4) for b in range(a + 1, 4)]
        Do = e.o.distances(np.stack(ocs), e.orlk, G3QP, e.ork, pairs=local, qp_sum=True)
        del ocs
        for t, (a, b) in enumerate(local):
            i, j = group[a], group[b]
            p = i * n - i * (i + 1) // 2 + (j - i - 1)
            assert np.array_equal(e.g_coeff(Dg[p].contiguous(), e.L - 1), e.o_coeff(Do[t]))
            compared += 1
    assert compared >= 16


@pytest.fixture(scope="module")
def prod_g2_b(prod_g2):
    """A second tenant at production parameters: its own key set (seed 9) for the same [2]*7
    schedule, on the same context as prod_g2."""
    e = prod_g2
    keys = KeySet(e.prm, 9, S.CFG_UNEVEN, O.rotations_of_schedule(e.sched))
    opk, orlk, ork = keys.oracle_keys(e.o)
    gpk, gevk = keys.gpu_keys(e.g)
    return keys, opk, orlk, ork, gpk, gevk


@pytest.mark.slow
def test_uneven_batch_production_sampled_against_oracle(prod_g2, prod_g2_b):
    """The uneven multi-job batch at production parameters (N = 2^15): three jobs of different
    client counts and model sizes, two tenants with their own key sets, one-ModDown groups [2]*7,
    through lc_batch_distances / lc_batch_aggregate with a wave cap that makes two jobs share
    waves and one run on its own.  Every pair's read-out against FP64; two sampled pairs and one
    aggregate chunk per job bit-exact against the oracle run with that job's keys."""
    e = prod_g2
    LC, g = e.LC, e.g
    keys_b, opk_b, orlk_b, ork_b, gpk_b, gevk_b = prod_g2_b
    tenants = {0: (e.keys, e.opk, e.orlk, e.ork, e.gpk, e.gevk), 1: (keys_b, opk_b, orlk_b, ork_b, gpk_b, gevk_b)}
    specs = [(10, 3, 0), (5, 9, 1), (6, 2, 0)]  # (clients, chunks, tenant); d ragged
    jobs, meta = [], []
    for jid, (n, chunks, ten) in enumerate(specs):
        keys, opk, orlk, ork, gpk, gevk = tenants[ten]
        nb = max(1, n // 5)
        w = S.Workload(f"up{jid}", S.CFG_UNEVEN, 15, n, chunks * e.prm.slots - 101, 2, tuple(range(n - nb, n)),
                       "scale5", max(1, n - 2 * nb - 3), nb, job=jid)
        W = S.client_updates(w)
        X = S.split_chunks(W, e.prm.slots)
        m = plaintexts(e.o, e.prm, X).reshape(n, chunks, e.N)
        r, e0, e1 = S.enc_rand_batch(w.seed, w.config, range(n), range(chunks), e.N, job=jid)
        cts = g.encrypt(gpk, m.reshape(-1, e.N), r, e0, e1).reshape(n, chunks, 2, e.L + 1, e.N)
        wts = np.zeros(n)
        wts[: n - nb] = 1.0 / (n - nb)
        mm = plaintexts(e.o, e.prm, np.stack([np.full((1, e.prm.slots), wts[i]) for i in range(n)]))[:, 0]
        rm, e0m, e1m = S.enc_rand_batch(w.seed, w.config, range(n), [S.MASK_CHUNK], e.N, job=jid)
        masks = g.encrypt(gpk, mm, rm, e0m, e1m)
        jobs.append(LC.Job(gevk, cts, n, chunks, masks))
        meta.append((w, W, X, m, (r, e0, e1), mm, (rm, e0m, e1m), wts, ten))
    g.set_max_batch(32)  # job 0 (45 pairs) runs alone; jobs 1 and 2 (10 + 15 pairs) share a wave
    try:
        LC.batch_distances(g, jobs, LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM, e.sched)
        LC.batch_aggregate(g, jobs)
    finally:
        g.set_max_batch(0)
    sc = e.prm.scale * e.prm.scale / e.prm.q[e.L]
    for j, (w, W, X, m, (r, e0, e1), mm, (rm, e0m, e1m), wts, ten) in zip(jobs, meta):
        keys, opk, orlk, ork, gpk, gevk = tenants[ten]
        n, chunks = w.n_clients, w.chunks
        got = g.decrypt_const(keys.s, j.out_dist, e.L - 1, sc)
        k = 0
        for a in range(n):
            for b in range(a + 1, n):
                ref = np.sum((W[a] - W[b]) ** 2)
                assert abs(got[k] - ref) / ref < 1e-5
                k += 1
        sample = [(0, 1), (n - 3, n - 1)]
        clients = sorted({c for p in sample for c in p})
        idx = {c: t for t, c in enumerate(clients)}
        ocs = np.stack([np.stack([e.o.encrypt(opk, m[c, k], r[c * chunks + k], e0[c * chunks + k],
                                              e1[c * chunks + k]) for k in range(chunks)]) for c in clients])
        Do = e.o.distances(ocs, orlk, e.sched, ork, pairs=[(idx[a], idx[b]) for a, b in sample], qp_sum=True)
        for t, (a, b) in enumerate(sample):
            p = a * n - a * (a + 1) // 2 + (b - a - 1)
            assert np.array_equal(e.g_coeff(j.out_dist[p].contiguous(), e.L - 1), e.o_coeff(Do[t]))
        kk = chunks - 1
        ock = np.stack([e.o.encrypt(opk, m[c, kk], r[c * chunks + kk], e0[c * chunks + kk], e1[c * chunks + kk])
                        for c in range(n)])[:, None]
        om = np.stack([e.o.encrypt(opk, mm[i], rm[i], e0m[i], e1m[i]) for i in range(n)])
        Ao = e.o.masked_aggregate(np.ascontiguousarray(ock), om, orlk)
        assert np.array_equal(e.g_coeff(j.out_agg[kk].contiguous(), e.L - 1), e.o_coeff(Ao[0]))
        asc = e.prm.scale * e.prm.scale / e.prm.q[e.L]
        agg = np.concatenate([g.decrypt(keys.s, j.out_agg[c].contiguous(), e.L - 1, asc) for c in range(chunks)])
        ref = sum(wts[i] * X[i].reshape(-1) for i in range(n))
        assert np.linalg.norm(agg - ref) / np.linalg.norm(ref) < 1e-5


def test_overlapped_copies_match_stream_ordered_copies(toy):
    """lc_copy_async / lc_copy_wait: an input copied in on the copy stream, transformed, and
    copied out after the transform gives the same words as the stream-ordered path; a copy
    into a buffer that queued work still reads waits for that work."""
    LC = toy.LC
    g = toy.g
    rng = np.random.default_rng(21)
    a = np.stack([rng.integers(0, q, size=toy.N, dtype=np.uint64) for q in toy.prm.q])
    ha = LC.pinned_empty(a.shape)
    ha[...] = a
    d = g.empty(*a.shape)
    t = g.copy_async(d, ha)
    g.copy_wait(t)
    g.to_eval(d, toy.L, inplace=True)
    hb = LC.pinned_empty(a.shape)
    t2 = g.copy_async(hb, d)  # ordered after the transform
    # overwrite the device buffer only after the read-out above has been queued
    g.copy_wait(t2)
    zero = LC.pinned_empty(a.shape)
    zero[...] = 0
    g.copy_wait(g.copy_async(d, zero))
    g.sync()
    torch.cuda.synchronize()
    ref = LC.torch_to_u64(g.to_eval(LC.u64_to_torch(a), toy.L))
    assert np.array_equal(np.asarray(hb), ref)
    assert not LC.torch_to_u64(d).any()
    with pytest.raises(LC.LancelotError):
        g.copy_wait(10 ** 9)
    with pytest.raises(LC.LancelotError):  # a ticket is consumed by its wait
        g.copy_wait(t2)
    # slots are reused: many copies do not grow the event pool past the copies in flight
    tickets = set()
    for _ in range(50):
        tk = g.copy_async(hb, d)
        g.copy_wait(tk)
        tickets.add(tk)
    assert len(tickets) <= 2


@pytest.mark.parametrize("log_n", [13, pytest.param(16, marks=pytest.mark.slow)])
def test_other_ring_degrees_bit_exact(log_n):
    """The packing-size sweep's rings (production primes at N = 2^13 and 2^16): distances of three
    clients in one-ModDown groups of 7 rotations, bit-exact against the oracle."""
    from paper_2408_06197_b300 import autotune
    from paper_2408_06197_b300 import lancelot as LC
    prm = O.params_production(log_n)
    o = O.Context(prm)
    g = LC.Context.production(log_n)
    sched = autotune.candidate_schedules(log_n)["g3qp"]
    keys = KeySet(prm, 5, S.CFG_PLAIN, O.rotations_of_schedule(sched))
    opk, orlk, ork = keys.oracle_keys(o)
    gpk, gevk = keys.gpu_keys(g)
    w = S.Workload(f"ring{log_n}", S.CFG_PLAIN, log_n, 3, prm.slots + 11, 5, (2,), "flip5", 1, 0)
    X = S.split_chunks(S.client_updates(w), prm.slots)
    m = plaintexts(o, prm, X).reshape(-1, prm.N)
    r, e0, e1 = S.enc_rand_batch(w.seed, w.config, range(3), range(w.chunks), prm.N)
    ocs = np.stack([o.encrypt(opk, m[k], r[k], e0[k], e1[k]) for k in range(m.shape[0])]).reshape(
        3, w.chunks, 2, prm.L + 1, prm.N)
    gcs = g.encrypt(gpk, m, r, e0, e1).reshape(3, w.chunks, 2, prm.L + 1, prm.N)
    Dg, _ = g.distances(gevk, gcs, 3, w.chunks, prm.scale, mode=LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM,
                        groups=sched)
    Do = o.distances(ocs, orlk, sched, ork, qp_sum=True)
    assert np.array_equal(LC.torch_to_u64(g.to_coeff(Dg, prm.L - 1)), o.to_coeff(Do))


@pytest.mark.parametrize("n_polys", [1, 7, 53])
def test_tma_row_pass_matches_per_tile_row_pass(prod, n_polys):
    """Forward NTT with the persistent bulk-copy row pass (each block walks several tiles at 53
    polynomials x 15 limbs x 16 tiles, with a ragged last wave) equals the one-block-per-tile pass
    bit for bit, round-trips, and leaves the context's error word clear."""
    LC, g = prod.LC, prod.g
    rng = np.random.default_rng(n_polys)
    a = np.stack([np.stack([rng.integers(0, q, size=prod.N, dtype=np.uint64) for q in prod.prm.q])
                  for _ in range(n_polys)])
    ga = LC.u64_to_torch(a)
    before = g.get_tuning(LC.LC_TUNE_NTT_ROW_TMA)
    try:
        g.set_tuning(LC.LC_TUNE_NTT_ROW_TMA, 0)
        ref = LC.torch_to_u64(g.to_eval(ga, prod.L))
        g.set_tuning(LC.LC_TUNE_NTT_ROW_TMA, 1)
        ev = g.to_eval(ga, prod.L)
        assert np.array_equal(LC.torch_to_u64(ev), ref)
        assert np.array_equal(LC.torch_to_u64(g.to_coeff(ev, prod.L)), a)
        g.sync()
    finally:
        g.set_tuning(LC.LC_TUNE_NTT_ROW_TMA, before)
