"""The handle layer of the C ABI (lc_keygen, lc_ct handles with level / scale / degree,
lc_ct_import / export, lc_encrypt_plain, lc_ct_distances, lc_ct_masked_aggregate, lc_batch_run)
against the CPU oracle, bit for bit in the coefficient domain, and its rejections of
ciphertexts at the wrong level or scale."""
import numpy as np
import pytest

import oracle as O
import synth as S
from common import KeySet, plaintexts
from test_oracle_pins import toy_distance_tolerance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class HEnv:
    """Keys made by lc_keygen from the same randomness the oracle's keys are made from."""

    def __init__(self, kind, seed, config, sched):
        from paper_2408_06197_b300 import lancelot as LC
        self.LC = LC
        self.prm = O.params_toy() if kind == "toy" else O.params_production()
        self.o = O.Context(self.prm)
        self.g = LC.Context.toy() if kind == "toy" else LC.Context.production()
        self.sched = sched
        self.rots = O.rotations_of_schedule(sched)
        self.keys = KeySet(self.prm, seed, config, self.rots)
        self.opk, self.orlk, self.ork = self.keys.oracle_keys(self.o)
        k = self.keys
        self.sk, self.pk, self.evk = self.g.keygen(k.s, k.pk_a, k.pk_e, k.rlk, k.rot)
        self.seed, self.config = seed, config
        self.N, self.L = self.prm.N, self.prm.L

    def inputs(self, w):
        W = S.client_updates(w)
        X = S.split_chunks(W, self.prm.slots)
        m = plaintexts(self.o, self.prm, X).reshape(-1, self.N)
        r, e0, e1 = S.enc_rand_batch(w.seed, w.config, range(w.n_clients), range(w.chunks), self.N, job=w.job)
        ocs = np.stack([self.o.encrypt(self.opk, m[k], r[k], e0[k], e1[k]) for k in range(m.shape[0])])
        return W, X, m, (r, e0, e1), ocs.reshape(w.n_clients, w.chunks, 2, self.L + 1, self.N)

    def clients_separate(self, w, m, rnd):
        """One handle per client, each its own allocation (the library gathers them)."""
        r, e0, e1 = rnd
        c = w.chunks
        return [self.g.encrypt_plain(self.pk, m[i * c:(i + 1) * c], self.prm.scale, r[i * c:(i + 1) * c],
                                     e0[i * c:(i + 1) * c], e1[i * c:(i + 1) * c]) for i in range(w.n_clients)]

    def clients_views(self, w, m, rnd):
        """One handle holding every client's chunks, and one view per client (contiguous)."""
        whole = self.g.encrypt_plain(self.pk, m, self.prm.scale, *rnd)
        return [whole.view(i * w.chunks, w.chunks) for i in range(w.n_clients)]


@pytest.fixture(scope="module")
def htoy():
    return HEnv("toy", S.TOY.seed, S.TOY.config, O.default_schedule(O.params_toy().slots))


def _masks(e, n, weights, job=0):
    MX = np.stack([np.full((1, e.prm.slots), weights[i]) for i in range(n)])
    m = plaintexts(e.o, e.prm, MX)[:, 0]
    r, e0, e1 = S.enc_rand_batch(e.seed, e.config, range(n), [S.MASK_CHUNK], e.N, job=job)
    om = np.stack([e.o.encrypt(e.opk, m[i], r[i], e0[i], e1[i]) for i in range(n)])
    gm = [e.g.encrypt_plain(e.pk, m[i:i + 1], e.prm.scale, r[i:i + 1], e0[i:i + 1], e1[i:i + 1]) for i in range(n)]
    return om, gm


def test_keygen_matches_oracle_keys(htoy):
    e = htoy
    assert np.array_equal(e.evk.export(None), e.o.key_to_coeff(e.orlk))
    for r in (e.rots[0], e.rots[-1]):
        assert np.array_equal(e.evk.export(r), e.o.key_to_coeff(e.ork[r]))


def test_handle_distances_and_aggregate_bit_exact_toy(htoy):
    e, LC = htoy, htoy.LC
    w = S.TOY
    W, X, m, rnd, ocs = e.inputs(w)
    Do = e.o.distances(ocs, e.orlk, e.sched, e.ork)
    q_L = e.prm.q[e.L]
    for clients in (e.clients_separate(w, m, rnd), e.clients_views(w, m, rnd)):
        assert np.array_equal(clients[1].export()[:, :, :, :], e.o.to_coeff(ocs[1]))
        D = e.g.ct_distances(e.evk, clients, mode=LC.LC_MODE_BATCHED)
        count, deg, level, scale = D.info()
        assert (count, deg, level) == (w.n_pairs, 2, e.L - 1)
        assert scale == e.prm.scale * e.prm.scale / q_L
        assert np.array_equal(D.export(), e.o.to_coeff(Do))
        v = e.g.decrypt_values(e.sk, D.view(0, 1))
        assert np.abs(v - np.sum((W[0] - W[1]) ** 2)).max() <= toy_distance_tolerance(e.prm)
    # a level drop before the rotations: the output handle is at that level
    D0 = e.g.ct_distances(e.evk, e.clients_views(w, m, rnd), mode=LC.LC_MODE_BATCHED | LC.rotate_at_level(0))
    assert D0.info()[:3] == (w.n_pairs, 2, 0)
    assert np.array_equal(D0.export(), e.o.to_coeff(e.o.distances(ocs, e.orlk, e.sched, e.ork, rot_level=0)))
    om, gm = _masks(e, w.n_clients, [1.0, 0.0, 0.0, 0.0])
    Ao = e.o.masked_aggregate(ocs, om, e.orlk)
    for mode in (LC.LC_MODE_BATCHED, LC.LC_MODE_PER_OP):
        A = e.g.ct_masked_aggregate(e.evk, e.clients_separate(w, m, rnd), gm, mode=mode)
        assert A.info()[:3] == (w.chunks, 2, e.L - 1)
        assert np.array_equal(A.export(), e.o.to_coeff(Ao))


def test_import_export_round_trip_and_values(htoy):
    e = htoy
    w = S.TOY
    W, X, m, rnd, ocs = e.inputs(w)
    coeffs = np.stack([e.o.to_coeff(ocs[i, 0]) for i in range(w.n_clients)])
    h = e.g.ct_import(coeffs, 2, e.L, e.prm.scale)
    assert h.info() == (w.n_clients, 2, e.L, e.prm.scale)
    assert np.array_equal(h.export(), coeffs)
    # the handle's device words (evaluation domain) seen as a torch tensor, and a view's
    t = h.tensor()
    assert t.shape == (w.n_clients, 2, e.L + 1, e.N)
    assert torch.equal(t, e.g.to_eval(e.LC.u64_to_torch(coeffs), e.L))
    assert torch.equal(h.view(1, 2).tensor(), t[1:3])
    # values in, values out: encode + encrypt in one call, decrypt + decode in one call
    vals = X[0, 0][: e.prm.slots - 5]
    r, e0, e1 = (a[:1] for a in rnd)
    ct = e.g.encrypt_values(e.pk, vals, e.prm.scale, r, e0, e1)
    back = e.g.decrypt_values(e.sk, ct, vals.size)
    # toy parameters (scale 2^30, N = 2^12): fresh encryption noise is about 3e-5 per slot
    assert np.abs(back - vals).max() < 5e-4
    assert ct.info() == (1, 2, e.L, e.prm.scale)


def test_wrong_level_scale_degree_and_shape_are_rejected(htoy):
    e, LC = htoy, htoy.LC
    w = S.TOY
    W, X, m, rnd, ocs = e.inputs(w)
    good = e.clients_separate(w, m, rnd)
    low = e.g.ct_create(w.chunks, 2, e.L - 1, e.prm.scale)           # one level down
    other = e.g.ct_create(w.chunks, 2, e.L, e.prm.scale * 2)          # another scale
    deg3 = e.g.ct_create(w.chunks, 3, e.L, e.prm.scale)               # not relinearised
    more = e.g.ct_create(w.chunks + 1, 2, e.L, e.prm.scale)           # another chunk count
    with pytest.raises(LC.LancelotError, match="LC_ELEVEL"):
        e.g.ct_distances(e.evk, good[:2] + [low] + good[3:])
    with pytest.raises(LC.LancelotError, match="LC_ESCALE"):
        e.g.ct_distances(e.evk, good[:3] + [other])
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):
        e.g.ct_distances(e.evk, [deg3] + good[1:])
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):
        e.g.ct_distances(e.evk, good[:3] + [more])
    om, gm = _masks(e, w.n_clients, [1.0, 0.0, 0.0, 0.0])
    low_mask = e.g.ct_create(1, 2, e.L - 1, e.prm.scale)
    with pytest.raises(LC.LancelotError, match="LC_ELEVEL"):
        e.g.ct_masked_aggregate(e.evk, good, gm[:3] + [low_mask])
    odd_mask = e.g.ct_create(1, 2, e.L, e.prm.scale * 3)
    with pytest.raises(LC.LancelotError, match="LC_ESCALE"):
        e.g.ct_masked_aggregate(e.evk, good, gm[:3] + [odd_mask])
    # a distance output (level L-1) fed back as a client
    D = e.g.ct_distances(e.evk, good)
    with pytest.raises(LC.LancelotError, match="LC_ELEVEL"):
        e.g.ct_distances(e.evk, [D.view(0, 1), D.view(1, 1)])
    # import: a residue equal to its prime, a level beyond L, a bad scale
    bad = np.zeros((1, 2, e.L + 1, e.N), dtype=np.uint64)
    bad[0, 1, 2, 17] = e.prm.q[2]
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):
        e.g.ct_import(bad, 2, e.L, e.prm.scale)
    with pytest.raises(LC.LancelotError, match="LC_ELEVEL"):
        e.g.ct_create(1, 2, e.L + 1, e.prm.scale)
    with pytest.raises(LC.LancelotError, match="LC_ESCALE"):
        e.g.ct_create(1, 2, e.L, float("nan"))
    # batch run: one malformed job stops the whole call before anything runs
    with pytest.raises(LC.LancelotError, match="LC_ELEVEL"):
        e.g.batch_run([{"evk": e.evk, "clients": good}, {"evk": e.evk, "clients": good[:1] + [low]}])


def test_batch_run_two_tenants_matches_oracle(htoy):
    """Two tenants with their own key sets (lc_keygen) and uneven jobs in one lc_batch_run: each
    job's distances and aggregate equal the oracle's for that tenant's keys."""
    e, LC = htoy, htoy.LC
    e2 = HEnv.__new__(HEnv)
    e2.__dict__.update(e.__dict__)
    e2.keys = KeySet(e.prm, 11, S.CFG_UNEVEN, e.rots)
    e2.opk, e2.orlk, e2.ork = e2.keys.oracle_keys(e.o)
    k = e2.keys
    e2.sk, e2.pk, e2.evk = e.g.keygen(k.s, k.pk_a, k.pk_e, k.rlk, k.rot)
    e2.seed, e2.config = 11, S.CFG_UNEVEN
    specs = [(e, 3, 2, 0), (e2, 4, 1, 1), (e2, 2, 3, 2)]
    jobs, expect = [], []
    for env, n, chunks, jid in specs:
        w = S.Workload(f"h{jid}", env.config, 12, n, chunks * env.prm.slots - 3, env.seed, (n - 1,), "scale5", 1, 1,
                       job=jid)
        W, X, m, rnd, ocs = env.inputs(w)
        wts = [1.0 / n] * n
        om, gm = _masks(env, n, wts, job=jid)
        jobs.append({"evk": env.evk, "clients": env.clients_separate(w, m, rnd), "masks": gm})
        expect.append((env.o.distances(ocs, env.orlk, env.sched, env.ork), env.o.masked_aggregate(ocs, om, env.orlk)))
    out = e.g.batch_run(jobs)
    for (D, A), (Do, Ao) in zip(out, expect):
        assert np.array_equal(D.export(), e.o.to_coeff(Do))
        assert np.array_equal(A.export(), e.o.to_coeff(Ao))


@pytest.mark.slow
def test_handle_distances_production_bit_exact():
    """At N = 2^15 with the benchmark's one-ModDown schedule: keys from lc_keygen, clients from
    lc_encrypt_plain, distances from lc_ct_distances, all bit-exact against the oracle."""
    sched = [3, 3, 3, 3, 2]
    e = HEnv("prod", 5, S.CFG_PLAIN, sched)
    LC = e.LC
    w = S.Workload("hp", S.CFG_PLAIN, 15, 3, e.prm.slots + 11, 5, (2,), "flip5", 1, 0)
    W, X, m, rnd, ocs = e.inputs(w)
    D = e.g.ct_distances(e.evk, e.clients_views(w, m, rnd), mode=LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM,
                         groups=sched)
    Do = e.o.distances(ocs, e.orlk, sched, e.ork, qp_sum=True)
    assert np.array_equal(D.export(), e.o.to_coeff(Do))
    v = e.g.decrypt_values(e.sk, D.view(2, 1), 1)[0]
    ref = np.sum((W[1] - W[2]) ** 2)
    assert abs(v - ref) / ref < 1e-5


def test_handle_edge_cases(htoy):
    """An empty batch runs nothing; a view outside its handle, a zero-count view, a handle of no
    ciphertexts as a client, and a single client are rejected; a zero-count handle exports
    nothing and keeps its metadata."""
    e, LC = htoy, htoy.LC
    assert e.g.batch_run([]) == []
    h = e.g.ct_create(3, 2, e.L, e.prm.scale)
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):
        h.view(2, 2)
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):
        h.view(0, 0)
    empty = e.g.ct_create(0, 2, e.L, e.prm.scale)
    assert empty.info() == (0, 2, e.L, e.prm.scale)
    assert empty.export().shape == (0, 2, e.L + 1, e.N)
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):
        e.g.ct_distances(e.evk, [empty, empty])
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):
        e.g.ct_distances(e.evk, [h])
