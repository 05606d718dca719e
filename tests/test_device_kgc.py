"""Device randomness, seeded encryption and the device-side KGC step.

* The GPU's Philox draws equal the oracle's (which is pinned to numpy's generator).
* Seeded encryption equals the oracle's encryption of the same plaintext with the oracle's
  draws, bit for bit; constant-slot (mask) encryption likewise.
* A round whose KGC step runs on the device (read-out, Krum, masks, aggregate) selects the same
  clients as the host KGC and produces the same aggregate bits as the host path given the same
  mask randomness; captured in one CUDA graph it replays to the same bits.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from common import plaintexts
from test_gpu_parity import Env

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHED = [3, 3, 3, 2]  # one-ModDown groups of 7 rotations at N = 2^12


@pytest.fixture(scope="module")
def toy():
    return Env("toy", 13, S.CFG_TOY, extra_rot=O.rotations_of_schedule(SCHED))


def test_device_draws_equal_oracle_draws(toy):
    for seed, first, count in [(1, 0, 2), (2 ** 63 + 5, 10 ** 9, 3)]:
        gr = toy.g.sample_enc(seed, first, count)
        orr = O.sample_enc(seed, first, count, toy.N)
        for a, b in zip(gr, orr):
            assert np.array_equal(a, b)


def test_seeded_encryption_bit_exact(toy):
    X = np.random.default_rng(40).normal(0, 0.01, (3, toy.prm.slots))
    m = plaintexts(toy.o, toy.prm, X)
    seed, first = 99, 500
    g = toy.g.encrypt_seeded(toy.gpk, toy.LC.u64_to_torch(m.view(np.uint64)).view(torch.int64), seed, first)
    r, e0, e1 = O.sample_enc(seed, first, 3, toy.N)
    for b in range(3):
        o = toy.o.encrypt(toy.opk, m[b], r[b], e0[b], e1[b])
        assert np.array_equal(toy.g_coeff(g[b].contiguous(), toy.L), toy.o_coeff(o))
    # constant-slot ciphertexts (masks): coefficient 0 = round(w * scale)
    w = np.array([0.25, 0.0, 1.0 / 3.0])
    gm = toy.g.encrypt_const_seeded(toy.gpk, torch.tensor(w, dtype=torch.float64, device="cuda"), toy.prm.scale,
                                    seed, first)
    for b in range(3):
        mb = np.zeros(toy.N, dtype=np.int64)
        mb[0] = int(np.rint(w[b] * toy.prm.scale))
        o = toy.o.encrypt(toy.opk, mb, r[b], e0[b], e1[b])
        assert np.array_equal(toy.g_coeff(gm[b].contiguous(), toy.L), toy.o_coeff(o))
        z = toy.g.decrypt(toy.keys.s, gm[b].contiguous(), toy.L, toy.prm.scale)
        assert np.abs(z - w[b]).max() < 1e-4


def _round_inputs(toy, n=6, chunks=2, job=0):
    w = S.Workload("dk", S.CFG_TOY, 12, n, chunks * toy.prm.slots - 9, 13, (n - 1,), "scale10", max(1, n - 3), 1,
                   job=job)
    W = S.client_updates(w)
    X = S.split_chunks(W, toy.prm.slots)
    _, gcs = toy.encrypt_both(X, range(n), range(chunks))
    return w, W, gcs


def test_device_kgc_round_matches_host_kgc(toy):
    from paper_2408_06197_b300 import kgc, serving
    LC = toy.LC
    g = toy.g
    w, W, gcs = _round_inputs(toy)
    n, chunks = w.n_clients, w.chunks
    key = LC.KgcKey(g, toy.keys.s)
    seed, first = 2024, 7
    res = serving.round_on_device(g, toy.gevk, toy.gpk, key, gcs, n, chunks, w.f, w.n_select, seed, first,
                                  groups=SCHED)
    torch.cuda.synchronize()
    # host KGC on the same distance ciphertexts
    sc = toy.prm.scale ** 2 / toy.prm.q[toy.L]
    vals = g.decrypt_const(toy.keys.s, res["dist"], toy.L - 1, sc)
    assert np.array_equal(res["values"].cpu().numpy(), vals)
    d = np.zeros((n, n))
    k = 0
    for i in range(n):
        for j in range(i + 1, n):
            d[i, j] = d[j, i] = vals[k]
            k += 1
    sel = kgc.krum_select(d, w.f, w.n_select)
    assert res["selected"].cpu().tolist() == sel
    wts = kgc.mask_weights(n, sel, average=True)
    assert np.array_equal(res["weights"].cpu().numpy(), wts)
    # host masks with the same draws, host-path aggregate: identical bits
    r, e0, e1 = g.sample_enc(seed, first, n)
    m = np.zeros((n, toy.N), dtype=np.int64)
    m[:, 0] = np.rint(wts * toy.prm.scale).astype(np.int64)
    masks = g.encrypt(toy.gpk, m, r, e0, e1)
    assert torch.equal(masks, res["masks"])
    agg, _ = g.masked_aggregate(toy.gevk, gcs, n, chunks, toy.prm.scale, masks, toy.prm.scale)
    assert torch.equal(agg, res["agg"])
    # plaintext check: the aggregate decrypts to the weighted sum of the kept updates
    X = S.split_chunks(W, toy.prm.slots)
    for c in range(chunks):
        got = g.decrypt(toy.keys.s, res["agg"][c].contiguous(), toy.L - 1, sc)
        assert np.abs(got - np.tensordot(wts, X[:, c], axes=1)).max() < 1e-4
    assert n - 1 not in sel


def test_device_kgc_round_in_one_graph(toy):
    """The whole round captured once and replayed on new client ciphertexts written into the same
    input buffer gives the bits of a direct run on those ciphertexts."""
    from paper_2408_06197_b300 import serving
    from paper_2408_06197_b300 import lancelot as LC
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = LC.Context.toy(stream=stream)
        pk, evk = toy.keys.gpu_keys(g)
        key = LC.KgcKey(g, toy.keys.s)
        w, W, gcs_a = _round_inputs(toy, job=1)
        _, _, gcs_b = _round_inputs(toy, job=2)
        n, chunks = w.n_clients, w.chunks
        cts = gcs_a.clone()
        bufs = serving.round_on_device(g, evk, pk, key, cts, n, chunks, w.f, w.n_select, 5, 0, groups=SCHED)
        g.sync()  # every scratch size is now known
        graph = g.capture(lambda: serving.round_on_device(g, evk, pk, key, cts, n, chunks, w.f, w.n_select, 5, 0,
                                                          groups=SCHED, out=bufs))
        cts.copy_(gcs_b)
        graph.launch()
        g.sync()
        replay = {k: v.clone() for k, v in bufs.items()}
        direct = serving.round_on_device(g, evk, pk, key, gcs_b.clone(), n, chunks, w.f, w.n_select, 5, 0,
                                         groups=SCHED)
        g.sync()
        for k in ("dist", "values", "weights", "selected", "masks", "agg"):
            assert torch.equal(replay[k], direct[k]), k
        graph.close()
        key.close()
        evk.close()
        g.close()


@pytest.fixture(scope="module")
def prod():
    return Env("prod", 14, S.CFG_PLAIN)


def test_gpu_encoder_matches_oracle_encoder(prod):
    z = np.random.default_rng(41).normal(0, 0.01, (6, prod.prm.slots))
    z[0] = 0.0
    z[1, :] = np.linspace(-1, 1, prod.prm.slots)
    mg = prod.g.encode_dev(torch.tensor(z, device="cuda"), prod.prm.scale).cpu().numpy()
    mo = plaintexts(prod.o, prod.prm, z)
    diff = np.abs(mg - mo)
    assert diff.max() <= 1 and np.count_nonzero(diff) <= 12  # FP64 near-ties only
    assert not mg[0].any()


def test_gpu_encode_encrypt_decrypts_and_composes(prod):
    z = np.random.default_rng(42).normal(0, 0.01, (3, prod.prm.slots))
    zt = torch.tensor(z, device="cuda")
    ct = prod.g.encode_encrypt_seeded(prod.gpk, zt, prod.prm.scale, 8, 100)
    m = prod.g.encode_dev(zt, prod.prm.scale)
    ref = prod.g.encrypt_seeded(prod.gpk, m, 8, 100)
    assert torch.equal(ct, ref)
    for b in range(3):
        got = prod.g.decrypt(prod.keys.s, ct[b].contiguous(), prod.L, prod.prm.scale)
        assert np.abs(got - z[b]).max() < 1e-6
