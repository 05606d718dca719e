"""Serving loop and KGC read-out on the GPU: every round's distances, selection and aggregate are
the same whether the round runs alone or batched with other tenants' rounds, under any admission
budget; the GPU read-out of constant-slot ciphertexts equals coefficient 0 of the oracle's
decryption."""
import numpy as np
import pytest

import oracle as O
import synth as S
from common import KeySet, plaintexts
from test_gpu_parity import Env, _toy_inputs
from test_oracle_pins import toy_distance_tolerance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


SCHED = [2] * 5 + [1]  # one-ModDown groups of 3 rotations, the serving loop's schedule at N = 2^12


@pytest.fixture(scope="module")
def toy():
    return Env("toy", S.TOY.seed, S.TOY.config, extra_rot=O.rotations_of_schedule(SCHED))


def _centred(v, q):
    v = int(v)
    return v - q if v > q // 2 else v


def test_decrypt_const_matches_oracle_coefficient0(toy):
    w, W, X, ocs, gcs = _toy_inputs(toy)
    Dg, sc = toy.g.distances(toy.gevk, gcs, w.n_clients, w.chunks, toy.prm.scale)
    Do = toy.o.distances(ocs, toy.orlk, toy.sched, toy.ork)
    got = toy.g.decrypt_const(toy.keys.s, Dg, toy.L - 1, sc)
    q0 = toy.prm.q[0]
    tol = toy_distance_tolerance(toy.prm)
    k = 0
    for i in range(w.n_clients):
        for j in range(i + 1, w.n_clients):
            res = toy.o.decrypt_residues(toy.keys.s, Do[k], toy.L - 1)
            assert got[k] == _centred(res[0][0], q0) / sc
            assert abs(got[k] - np.sum((W[i] - W[j]) ** 2)) <= tol
            k += 1
    # a sub-range of the batch reads the same values
    part = toy.g.decrypt_const(toy.keys.s, Dg[2:5].contiguous(), toy.L - 1, sc)
    assert np.array_equal(part, got[2:5])
    assert toy.g.decrypt_const(toy.keys.s, Dg[:0], toy.L - 1, sc).shape == (0,)


def test_decrypt_const_production():
    env = Env("prod", 0, S.CFG_PLAIN)
    w = S.Workload("pc", S.CFG_PLAIN, 15, 3, env.prm.slots + 300, 0, (2,), "flip5", 1, 0)
    W = S.client_updates(w)
    X = S.split_chunks(W, env.prm.slots)
    _, gcs = env.encrypt_both(X, range(3), range(w.chunks))
    Dg, sc = env.g.distances(env.gevk, gcs, 3, w.chunks, env.prm.scale)
    got = env.g.decrypt_const(env.keys.s, Dg, env.L - 1, sc)
    k = 0
    for i in range(3):
        for j in range(i + 1, 3):
            ref = np.sum((W[i] - W[j]) ** 2)
            assert abs(got[k] - ref) / ref < 1e-5
            full = env.g.decrypt(env.keys.s, Dg[k].contiguous(), env.L - 1, sc)
            assert abs(got[k] - full.mean()) / ref < 1e-6
            k += 1


# ------------------------------------------------------------------------------- serving loop

class _Feed:
    """Toy rounds of two tenants; ciphertexts encrypted once, handed out at admission."""

    def __init__(self, env):
        from paper_2408_06197_b300 import serving as SV
        self.env, self.SV = env, SV
        g = env.g
        kb = KeySet(env.prm, 9, S.CFG_SERVING, O.rotations_of_schedule(SCHED))
        pk_b, evk_b = kb.gpu_keys(g)
        self.tenants = [SV.Tenant(env.gevk, env.gpk, env.keys.s), SV.Tenant(evk_b, pk_b, kb.s)]
        specs = [(0, 0, 4, 1), (1, 1, 5, 2), (2, 0, 3, 3), (3, 1, 4, 1), (4, 0, 6, 2), (5, 1, 3, 2)]
        self.W, self.cts, self.specs = {}, {}, specs
        for rid, ten, n, chunks in specs:
            w = S.Workload(f"s{rid}", S.CFG_SERVING, 12, n, chunks * env.prm.slots - 5, 3, (n - 1,), "scale5",
                           max(1, n - 3), 1, job=rid)
            W = S.client_updates(w)
            X = S.split_chunks(W, env.prm.slots)
            m = plaintexts(env.o, env.prm, X).reshape(-1, env.N)
            r, e0, e1 = S.enc_rand_batch(w.seed, w.config, range(n), range(chunks), env.N, job=rid)
            pk = self.tenants[ten].pk
            self.cts[rid] = g.encrypt(pk, m, r, e0, e1).reshape(n, chunks, 2, env.L + 1, env.N)
            self.W[rid] = W

    def rounds(self, rids=None, spacing=0.0):
        out = []
        for rid, ten, n, chunks in self.specs:
            if rids is None or rid in rids:
                out.append(self.SV.Round(rid, ten, n, chunks, arrival=rid * spacing, f=1, n_select=max(1, n - 3),
                                         average=True))
        return out

    def server(self, budget, device_kgc_seed=None):
        return self.SV.Server(self.env.g, self.tenants, budget, ingest=lambda r: self.cts[r.rid].clone(),
                              mask_rand=lambda r, i: S.enc_rand(3, S.CFG_SERVING, i, S.MASK_CHUNK, self.env.N,
                                                                job=r.rid), groups=SCHED, keep_outputs=True,
                              device_kgc_seed=device_kgc_seed)


@pytest.fixture(scope="module")
def feed(toy):
    return _Feed(toy)


def _by_rid(done):
    return {r.rid: r for r in done}


def test_serving_round_identical_alone_and_in_mix(feed):
    mix = _by_rid(feed.server(1e12).run(feed.rounds(), realtime=False))
    assert len(mix) == len(feed.specs)
    for rid, *_ in feed.specs:
        alone = _by_rid(feed.server(1e12).run(feed.rounds([rid]), realtime=False))[rid]
        got = mix[rid]
        assert torch.equal(alone.job.out_dist, got.job.out_dist)
        assert torch.equal(alone.job.masks, got.job.masks)
        assert torch.equal(alone.job.out_agg, got.job.out_agg)
        assert alone.selected == got.selected


def test_serving_budget_and_arrivals_do_not_change_results(feed):
    ref = _by_rid(feed.server(1e12).run(feed.rounds(), realtime=False))
    srv = feed.server(1.0)  # admits one round at a time
    one = _by_rid(srv.run(feed.rounds(), realtime=False))
    spaced = _by_rid(feed.server(1e12).run(feed.rounds(spacing=0.02), realtime=True))
    for rid in ref:
        for other in (one, spaced):
            assert torch.equal(ref[rid].job.out_dist, other[rid].job.out_dist)
            assert torch.equal(ref[rid].job.out_agg, other[rid].job.out_agg)
    assert srv.used == 0 and not srv.active and not srv.waiting


def test_serving_results_match_fp64(feed, toy):
    from paper_2408_06197_b300 import kgc
    done = _by_rid(feed.server(1e12).run(feed.rounds(), realtime=False))
    tol = toy_distance_tolerance(toy.prm)
    for rid, ten, n, chunks in feed.specs:
        r, W = done[rid], feed.W[rid]
        ref = np.array([[np.sum((W[i] - W[j]) ** 2) for j in range(n)] for i in range(n)])
        assert np.abs(r.distances - ref).max() <= tol
        assert r.selected == kgc.krum_select(ref, 1, max(1, n - 3))
        assert n - 1 not in r.selected  # the Byzantine client (x5) is never kept
        wts = kgc.mask_weights(n, r.selected, average=True)
        X = S.split_chunks(W, toy.prm.slots)
        sc = toy.prm.scale * toy.prm.scale / toy.prm.q[toy.L]
        s = feed.tenants[ten].s
        for k in range(chunks):
            got = toy.g.decrypt(s, r.job.out_agg[k].contiguous(), toy.L - 1, sc)
            want = np.tensordot(wts, X[:, k], axes=1)
            # toy parameters (scale 2^30): about 7e-6 rms per slot, so 1e-4 is about 14 sigma
            assert np.abs(got - want).max() < 1e-4


def test_serving_with_device_kgc(feed, toy):
    """KGC step on the device: same selections as the host KGC, every round identical alone and
    in the mix, aggregates decrypt to the weighted sums."""
    from paper_2408_06197_b300 import kgc
    host = _by_rid(feed.server(1e12).run(feed.rounds(), realtime=False))
    dev = _by_rid(feed.server(1e12, device_kgc_seed=77).run(feed.rounds(), realtime=False))
    sc = toy.prm.scale * toy.prm.scale / toy.prm.q[toy.L]
    for rid, ten, n, chunks in feed.specs:
        assert dev[rid].selected == host[rid].selected
        assert np.array_equal(dev[rid].distances, host[rid].distances)
        alone = _by_rid(feed.server(1e12, device_kgc_seed=77).run(feed.rounds([rid]), realtime=False))[rid]
        assert torch.equal(alone.job.masks, dev[rid].job.masks)
        assert torch.equal(alone.job.out_agg, dev[rid].job.out_agg)
        wts = kgc.mask_weights(n, dev[rid].selected, average=True)
        X = S.split_chunks(feed.W[rid], toy.prm.slots)
        for k in range(chunks):
            got = toy.g.decrypt(feed.tenants[ten].s, dev[rid].job.out_agg[k].contiguous(), toy.L - 1, sc)
            assert np.abs(got - np.tensordot(wts, X[:, k], axes=1)).max() < 1e-4


def test_serving_two_lanes_identical_to_one_lane(feed, toy):
    """The lane pipeline with two contexts -- rounds of at most 6 pairs on a high-priority stream,
    the others on a low-priority stream, keys shared -- gives every round the same distances,
    selection, masks and aggregate as one lane, with rounds arriving while others run."""
    from paper_2408_06197_b300 import lancelot as LC
    from paper_2408_06197_b300 import serving as SV
    one = _by_rid(feed.server(1e12, device_kgc_seed=77).run(feed.rounds(), realtime=False))
    lo, hi = torch.cuda.Stream(priority=0), torch.cuda.Stream(priority=-1)
    g_fast, g_bulk = LC.Context.toy(stream=hi), LC.Context.toy(stream=lo)
    srv = SV.Server(toy.g, feed.tenants, 1e12, ingest=lambda r: feed.cts[r.rid].clone(),
                    mask_rand=None, groups=SCHED, keep_outputs=True, device_kgc_seed=77,
                    lanes=[SV.Lane(g_fast, 6, "fast"), SV.Lane(g_bulk, None, "bulk")])
    two = _by_rid(srv.run(feed.rounds(spacing=0.005), realtime=True))
    torch.cuda.synchronize()
    assert {r.lane for r in two.values()} == {0, 1}
    for rid, *_ in feed.specs:
        a, b = one[rid], two[rid]
        assert a.selected == b.selected
        assert np.array_equal(a.distances, b.distances)
        assert torch.equal(a.job.masks, b.job.masks)
        assert torch.equal(a.job.out_agg, b.job.out_agg)
    assert srv.used == 0 and not srv.active
