"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: primality and the prime
rule (sympy), evaluation at powers of psi, schoolbook negacyclic products, exact big-integer
rounding (rescale), exact error sets of the approximate base conversions, the key-switch
phase bound, decryption against plaintext (encrypt, multiply, rotate), the hoisting and lazy
relinearisation counters, and the toy workload end to end against FP64.
"""
import math

import numpy as np
import pytest
import sympy

import oracle as O
import synth as S
from bigint_ref import centred, crt, eval_at, negacyclic_mul, negacyclic_mul_int, prod, round_div, substitute


def tiny(log_n=4, nq=4, np_=2, dnum=2, qbits=26, pbits=31):
    q = O.gen_primes(log_n, qbits, 0, nq)
    p = O.gen_primes(log_n, pbits, 0, np_)
    return O.Params(log_n, q, p, dnum, float(2 ** 16))


def rand_poly(rng, moduli, N):
    return np.stack([rng.integers(0, int(m), size=N, dtype=np.uint64) for m in moduli])


# --------------------------------------------------------------------------- primes

@pytest.mark.parametrize("maker,log_n,bits_q0,bits_q,bits_p,nq,np_", [
    (O.params_production, 15, 60, 40, 60, 15, 4),
    (O.params_toy, 12, 50, 30, 50, 3, 1),
])
def test_prime_rule(maker, log_n, bits_q0, bits_q, bits_p, nq, np_):
    prm = maker()
    M = 2 << log_n
    assert len(prm.q) == nq and len(prm.p) == np_
    for x in prm.q + prm.p:
        assert sympy.isprime(x) and x % M == 1
    assert prm.q[0].bit_length() == bits_q0 and all(x.bit_length() == bits_q for x in prm.q[1:])
    assert all(x.bit_length() == bits_p for x in prm.p)
    # q0 is the largest such prime below 2^bits; p continue the descending list without gaps
    chain60 = [prm.q[0]] + prm.p
    top = (1 << bits_q0) - 1
    cands = [c for c in range(top - top % M + 1, chain60[-1] - 1, -M) if c <= top]
    primes = [c for c in cands if sympy.isprime(c)]
    assert primes[: len(chain60)] == chain60
    top = (1 << bits_q) - 1
    cands = [c for c in range(top - top % M + 1, prm.q[-1] - 1, -M) if c <= top]
    assert [c for c in cands if sympy.isprime(c)][: nq - 1] == prm.q[1:]
    assert len(set(prm.q + prm.p)) == nq + np_


# --------------------------------------------------------------------------- NTT

def test_psi_is_primitive_2n_root():
    prm = tiny()
    ctx = O.Context(prm)
    for i, m in enumerate(prm.q + prm.p):
        psi = ctx.psi(i)
        assert pow(psi, prm.N, m) == m - 1 and pow(psi, 2 * prm.N, m) == 1


@pytest.mark.parametrize("log_n", [4, 6])
def test_ntt_is_evaluation_at_odd_powers(log_n):
    prm = tiny(log_n=log_n)
    ctx = O.Context(prm)
    rng = np.random.default_rng(5)
    for i, m in enumerate(prm.q + prm.p):
        a = rng.integers(0, m, size=prm.N, dtype=np.uint64)
        A = ctx.ntt(i, a)
        psi = ctx.psi(i)
        for k in range(prm.N):
            assert int(A[k]) == eval_at(a.tolist(), pow(psi, 2 * k + 1, m), m)


def test_ntt_spot_evaluation_production():
    prm = O.params_production()
    ctx = O.Context(prm)
    rng = np.random.default_rng(6)
    for i in (0, 7, 15):  # a 60-bit q, a 40-bit q, a special prime
        m = (prm.q + prm.p)[i]
        a = rng.integers(0, m, size=prm.N, dtype=np.uint64)
        A = ctx.ntt(i, a)
        psi = ctx.psi(i)
        for k in (0, 1, 12345, prm.N - 1):
            assert int(A[k]) == eval_at(a.tolist(), pow(psi, 2 * k + 1, m), m)
        assert np.array_equal(ctx.intt(i, A), a)


@pytest.mark.parametrize("log_n", [6, 10])
def test_transform_product_is_schoolbook(log_n):
    prm = tiny(log_n=log_n)
    ctx = O.Context(prm)
    rng = np.random.default_rng(7)
    for i, m in enumerate(prm.q[:2] + prm.p[:1]):
        idx = i if i < 2 else len(prm.q)
        a = rng.integers(0, m, size=prm.N, dtype=np.uint64)
        b = rng.integers(0, m, size=prm.N, dtype=np.uint64)
        assert ctx.poly_mul(idx, a, b).tolist() == negacyclic_mul(a.tolist(), b.tolist(), m)


def test_transform_product_spot_n4096():
    prm = O.params_toy()
    ctx = O.Context(prm)
    rng = np.random.default_rng(8)
    m, N = prm.q[0], prm.N
    a = rng.integers(0, m, size=N, dtype=np.uint64).tolist()
    b = rng.integers(0, m, size=N, dtype=np.uint64).tolist()
    out = ctx.poly_mul(0, np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64))
    for k in (0, 1, 2047, 4095):
        v = sum(a[i] * b[k - i] for i in range(k + 1)) - sum(a[i] * b[N + k - i] for i in range(k + 1, N))
        assert int(out[k]) == v % m


# --------------------------------------------------------------------------- encode / automorphism

def test_encode_matches_naive_sum_and_roundtrips():
    prm = tiny(log_n=8)
    ctx = O.Context(prm)
    N, scale = prm.N, 2.0 ** 30
    rng = np.random.default_rng(9)
    z = rng.normal(0, 1, N // 2)
    m = ctx.encode(z, scale)
    e = O.rot_group(N)
    k = np.arange(N)[:, None]
    xi = np.exp(-1j * np.pi * (k * e[None, :] % (2 * N)) / N)
    naive = np.rint((2.0 / N) * (xi @ (scale * z)).real).astype(np.int64)
    assert np.abs(m - naive).max() <= 1 and np.count_nonzero(m != naive) <= 2
    back = ctx.decode(m.astype(np.float64), scale)
    assert np.abs(back - z).max() <= 0.5 * N / scale
    # constant in every slot encodes to a constant polynomial
    mc = ctx.encode(np.full(N // 2, 0.25), scale)
    assert mc[0] == round(0.25 * scale) and np.all(mc[1:] == 0)


@pytest.mark.parametrize("g", [5, 25, 3, 63])
def test_automorphism_is_substitution(g):
    prm = tiny(log_n=5)
    ctx = O.Context(prm)
    rng = np.random.default_rng(10)
    a = rand_poly(rng, prm.q, prm.N)
    out = ctx.automorph_coeff(a, list(range(len(prm.q))), g)
    for i, m in enumerate(prm.q):
        ref = [x % m for x in substitute(a[i].tolist(), g)]
        assert out[i].tolist() == ref


# --------------------------------------------------------------------------- base conversion

def test_modup_error_set():
    prm = tiny(log_n=4, nq=5, np_=2, dnum=2)  # alpha = 3: digits {q0,q1,q2}, {q3,q4}
    ctx = O.Context(prm)
    rng = np.random.default_rng(11)
    alpha = ctx.alpha
    assert alpha == 3
    for level in (4, 3, 1):
        c = rand_poly(rng, prm.q[: level + 1], prm.N)
        rows = prm.q[: level + 1] + prm.p
        for j in range(-(-(level + 1) // alpha)):
            D = list(range(j * alpha, min((j + 1) * alpha, level + 1)))
            Dprod = prod([prm.q[i] for i in D])
            ext = ctx.modup_coeff(c, level, j)
            for t in D:
                assert np.array_equal(ext[t], c[t])
            Mall = prod(rows)
            for x in range(prm.N):
                X = crt([int(c[i, x]) for i in D], [prm.q[i] for i in D])
                E = centred(crt([int(ext[t, x]) for t in range(len(rows))], rows), Mall)
                u, rem = divmod(E - centred(X, Dprod), Dprod)
                assert rem == 0 and abs(u) <= (alpha + 1) // 2


def test_moddown_error_set():
    prm = tiny(log_n=4, nq=4, np_=3, dnum=2)
    ctx = O.Context(prm)
    rng = np.random.default_rng(12)
    K = len(prm.p)
    P = prod(prm.p)
    for level in (3, 1):
        rows = prm.q[: level + 1] + prm.p
        u = rand_poly(rng, rows, prm.N)
        out = ctx.moddown_coeff(u, level)
        Q = prod(prm.q[: level + 1])
        seen = set()
        for x in range(prm.N):
            X = crt([int(u[t, x]) for t in range(len(rows))], rows)
            o = crt([int(out[i, x]) for i in range(level + 1)], prm.q[: level + 1])
            w = centred(round_div(X, P) - o, Q)
            assert abs(w) <= (K + 1) // 2
            seen.add(w)
        assert 0 in seen


def test_rescale_is_exact_rounding():
    prm = tiny(log_n=4, nq=4, np_=1, dnum=4)
    ctx = O.Context(prm)
    rng = np.random.default_rng(13)
    for level in (3, 2, 1):
        c = rand_poly(rng, prm.q[: level + 1], prm.N)[None].repeat(2, axis=0)
        c[1] = rand_poly(rng, prm.q[: level + 1], prm.N)
        out = ctx.to_coeff(ctx.rescale(ctx.to_eval(c), level))
        ql = prm.q[level]
        Qm = prod(prm.q[:level])
        for p in range(2):
            for x in range(prm.N):
                X = crt([int(c[p, i, x]) for i in range(level + 1)], prm.q[: level + 1])
                o = crt([int(out[p, i, x]) for i in range(level)], prm.q[:level])
                assert o == round_div(X, ql) % Qm


# --------------------------------------------------------------------------- keys and key switching

def _keys(ctx, prm, seed=0):
    N = prm.N
    s = S.secret_key(seed, 99, N)
    qp = prm.q + prm.p
    a, e = S.swk_rand(seed, 99, qp, prm.dnum, N, None)
    return s, ctx.swk_gen(s, 0, a, e)


def _phase_error(ctx, prm, s, ks_eval, level, target_coef):
    ks = ctx.to_coeff(ks_eval)
    mods = prm.q[: level + 1]
    Q = prod(mods)
    sl = [int(v) for v in s]
    phase = []
    for i, m in enumerate(mods):
        t = negacyclic_mul(ks[1, i].tolist(), [v % m for v in sl], m)
        phase.append([(int(ks[0, i, x]) + t[x]) % m for x in range(prm.N)])
    err = []
    for x in range(prm.N):
        ph = crt([phase[i][x] for i in range(len(mods))], mods)
        tg = crt([target_coef[i][x] % mods[i] for i in range(len(mods))], mods)
        err.append(centred(ph - tg, Q))
    return err


@pytest.mark.parametrize("level", [3, 2])
def test_keyswitch_phase_bound(level):
    prm = tiny(log_n=5, nq=4, np_=2, dnum=2, qbits=26, pbits=40)
    ctx = O.Context(prm)
    s, rlk = _keys(ctx, prm)
    rng = np.random.default_rng(14)
    c_coef = rand_poly(rng, prm.q[: level + 1], prm.N)
    out = ctx.keyswitch(ctx.to_eval(c_coef), level, rlk)
    s2 = negacyclic_mul_int(s.tolist(), s.tolist())
    target = [negacyclic_mul(c_coef[i].tolist(), [v % m for v in s2], m) for i, m in enumerate(prm.q[: level + 1])]
    err = _phase_error(ctx, prm, s, out, level, target)
    alpha, K, N, P = ctx.alpha, len(prm.p), prm.N, prod(prm.p)
    beta = -(-(level + 1) // alpha)
    Dmax = max(prod(prm.q[j * alpha: min((j + 1) * alpha, level + 1)]) for j in range(beta))
    bound = beta * N * alpha * Dmax * S.ERR_BOUND / (2 * P) + K * (1 + N) / 2
    assert max(abs(e) for e in err) <= bound
    # the bound is meaningful: a wrong key (s instead of s^2) breaks it by orders of magnitude
    wrong = [[v % m for v in s.tolist()] for m in prm.q[: level + 1]]
    target_bad = [negacyclic_mul(c_coef[i].tolist(), wrong[i], m) for i, m in enumerate(prm.q[: level + 1])]
    assert max(abs(e) for e in _phase_error(ctx, prm, s, out, level, target_bad)) > 1000 * bound


# --------------------------------------------------------------------------- encrypt / decrypt

@pytest.fixture(scope="module")
def toy():
    w = S.TOY
    prm = O.params_toy()
    ctx = O.Context(prm)
    N = prm.N
    s = S.secret_key(w.seed, w.config, N)
    a, e = S.pk_rand(w.seed, w.config, prm.q, N)
    pk = ctx.pk_gen(s, a, e)
    qp = prm.q + prm.p
    ar, er = S.swk_rand(w.seed, w.config, qp, prm.dnum, N, None)
    rlk = ctx.swk_gen(s, 0, ar, er)
    sched = O.default_schedule(prm.slots)
    rk = {}
    for r in O.rotations_of_schedule(sched) + [3]:
        ar, er = S.swk_rand(w.seed, w.config, qp, prm.dnum, N, r)
        rk[r] = ctx.swk_gen(s, ctx.galois(r), ar, er)
    return dict(w=w, prm=prm, ctx=ctx, s=s, pk=pk, rlk=rlk, rk=rk, sched=sched)


def _enc(T, z, client=0, chunk=0):
    prm, ctx = T["prm"], T["ctx"]
    m = ctx.encode(z, prm.scale)
    r, e0, e1 = S.enc_rand(T["w"].seed, T["w"].config, client, chunk, prm.N)
    return ctx.encrypt(T["pk"], m, r, e0, e1), m


def test_decrypt_of_fresh_ciphertext(toy):
    prm, ctx = toy["prm"], toy["ctx"]
    z = np.random.default_rng(15).normal(0, 1, prm.slots)
    ct, m = _enc(toy, z)
    res = ctx.decrypt_residues(toy["s"], ct, prm.L)
    v = np.array(ctx.crt_centered(res), dtype=object)
    noise = np.array([int(a) - int(b) for a, b in zip(v, m)])
    # |e0 + r e_pk + e1 s| <= 19 (1 + 2N)
    assert np.abs(noise).max() <= S.ERR_BOUND * (1 + 2 * prm.N)
    assert abs(noise.mean()) < 20
    assert np.abs(ctx.decrypt(toy["s"], ct, prm.L, prm.scale) - z).max() < 1e-4


def test_product_relin_rescale_decrypts_to_product(toy):
    prm, ctx = toy["prm"], toy["ctx"]
    rng = np.random.default_rng(16)
    a, b = rng.normal(0, 1, prm.slots), rng.normal(0, 1, prm.slots)
    ca, _ = _enc(toy, a, 0, 0)
    cb, _ = _enc(toy, b, 1, 0)
    t = ctx.tensor(ca, cb, prm.L)
    assert np.abs(ctx.decrypt(toy["s"], t, prm.L, prm.scale ** 2) - a * b).max() < 1e-3
    r = ctx.relin(t, prm.L, toy["rlk"])
    rs = ctx.rescale(r, prm.L)
    sc = prm.scale ** 2 / prm.q[prm.L]
    assert np.abs(ctx.decrypt(toy["s"], rs, prm.L - 1, sc) - a * b).max() < 1e-3


def test_rotations_decrypt_to_rolled_slots(toy):
    prm, ctx = toy["prm"], toy["ctx"]
    z = np.random.default_rng(17).normal(0, 1, prm.slots)
    ct, _ = _enc(toy, z)
    rots = [1, 2, 3, 1024]
    outs = ctx.rotate_hoisted(ct, prm.L, rots, [toy["rk"][r] for r in rots])
    for r, o in zip(rots, outs):
        err = ctx.decrypt(toy["s"], o, prm.L, prm.scale) - np.roll(z, -r)
        assert np.abs(err).max() < 2e-4 and abs(err.mean()) < 2e-6
    # one ModUp shared by all rotations: identical to separate single rotations
    for r, o in zip(rots, outs):
        single = ctx.rotate_hoisted(ct, prm.L, [r], [toy["rk"][r]])[0]
        assert np.array_equal(single, o)


def test_hoisted_group_and_counters(toy):
    prm, ctx = toy["prm"], toy["ctx"]
    z = np.random.default_rng(18).normal(0, 1, prm.slots)
    ct, _ = _enc(toy, z)
    ctx.reset_counters()
    y1 = ctx.rotate_sum(ct, prm.L, [1, 1], toy["rk"])
    assert ctx.counters() == (2, 2)
    ctx.reset_counters()
    y2 = ctx.rotate_sum(ct, prm.L, [2], toy["rk"])  # rotations 1,2,3 from one ModUp
    assert ctx.counters() == (3, 1)
    outs = ctx.rotate_hoisted(ct, prm.L, [1, 2, 3], [toy["rk"][r] for r in (1, 2, 3)])
    ref = ct
    for o in outs:
        ref = ctx.add(ref, o, prm.L)
    assert np.array_equal(y2, ref)
    ref_slots = z + np.roll(z, -1) + np.roll(z, -2) + np.roll(z, -3)
    for y in (y1, y2):
        assert np.abs(ctx.decrypt(toy["s"], y, prm.L, prm.scale) - ref_slots).max() < 5e-4


def test_qp_sum_hoisting_variant(toy):
    """One-ModDown hoisting (inner products of a group summed in Q U P): identical bits for
    groups of one rotation, correct decryption and one ModUp per group of three rotations."""
    prm, ctx = toy["prm"], toy["ctx"]
    z = np.random.default_rng(20).normal(0, 1, prm.slots)
    ct, _ = _enc(toy, z)
    a = ctx.rotate_sum(ct, prm.L, [1, 1], toy["rk"])
    b = ctx.rotate_sum(ct, prm.L, [1, 1], toy["rk"], qp_sum=True)
    assert np.array_equal(a, b)
    ctx.reset_counters()
    y = ctx.rotate_sum(ct, prm.L, [2], toy["rk"], qp_sum=True)
    assert ctx.counters() == (3, 1)
    ref_slots = z + np.roll(z, -1) + np.roll(z, -2) + np.roll(z, -3)
    assert np.abs(ctx.decrypt(toy["s"], y, prm.L, prm.scale) - ref_slots).max() < 5e-4
    per_rot = ctx.rotate_sum(ct, prm.L, [2], toy["rk"])
    assert not np.array_equal(y, per_rot)  # a different rounding, not the same algorithm


def toy_distance_tolerance(prm):
    """10x the predicted 1-sigma error of a toy distance (rotation key-switch noise dominates):
    per rotation the switched noise is about sqrt(N) * 3.2 * q0/sqrt(12) / P per coefficient,
    i.e. sqrt(N) times that per slot; rotate-and-sum adds about `slots` such terms."""
    per_coef = math.sqrt(prm.N) * S.SIGMA * prm.q[0] / math.sqrt(12) / prm.p[0]
    per_slot = per_coef * math.sqrt(prm.N) / (prm.scale ** 2 / prm.q[prm.L])
    return 10 * per_slot * math.sqrt(prm.slots)


def test_toy_workload_end_to_end(toy):
    """Distances within 10 sigma of FP64, lazy relinearisation count, Krum selection, masked sum."""
    from paper_2408_06197_b300 import kgc

    w, prm, ctx = toy["w"], toy["prm"], toy["ctx"]
    W = S.client_updates(w)
    X = S.split_chunks(W, prm.slots)
    cts = np.zeros((w.n_clients, w.chunks, 2, prm.L + 1, prm.N), dtype=np.uint64)
    for i in range(w.n_clients):
        for k in range(w.chunks):
            cts[i, k], _ = _enc(toy, X[i, k], i, k)
    ctx.reset_counters()
    D = ctx.distances(cts, toy["rlk"], toy["sched"], toy["rk"])
    ks, mu = ctx.counters()
    assert ks == w.n_pairs * (1 + len(toy["sched"])) and mu == ks
    sc = prm.scale ** 2 / prm.q[prm.L]
    tol = toy_distance_tolerance(prm)
    dist = np.zeros((w.n_clients, w.n_clients))
    k = 0
    for i in range(w.n_clients):
        for j in range(i + 1, w.n_clients):
            v = ctx.decrypt(toy["s"], D[k], prm.L - 1, sc)
            ref = float(np.sum((W[i] - W[j]) ** 2))
            assert abs(v[0] - ref) <= tol
            assert np.abs(v - ref).max() <= tol  # every slot holds the full sum
            dist[i, j] = dist[j, i] = v[0]
            k += 1
    sel = kgc.krum_select(dist, f=w.f, n_select=w.n_select)
    ref_d = np.array([[np.sum((W[i] - W[j]) ** 2) for j in range(w.n_clients)] for i in range(w.n_clients)])
    assert sel == kgc.krum_select(ref_d, f=w.f, n_select=w.n_select)
    assert 3 not in sel
    weights = kgc.mask_weights(w.n_clients, sel, average=False)
    masks = np.stack([_enc(toy, np.full(prm.slots, weights[i]), i, S.MASK_CHUNK)[0] for i in range(w.n_clients)])
    agg = ctx.masked_aggregate(cts, masks, toy["rlk"])
    got = ctx.decrypt(toy["s"], agg[0], prm.L - 1, sc)
    ref = sum(weights[i] * X[i, 0] for i in range(w.n_clients))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-3


def test_level_drop_before_rotations(toy):
    """Distances with the rescaled pairs dropped to a lower level before the rotate-and-sum: at
    the rescaled level itself the drop is the identity (bit-exact with the plain distances); one
    level lower (limb q_0 only) every slot still decrypts to the FP64 distance within the toy
    tolerance and Krum picks the same clients; a fresh ciphertext dropped to level 0 decrypts to
    the same residues mod q_0 as the full one (a level drop keeps the message)."""
    from paper_2408_06197_b300 import kgc

    w, prm, ctx = toy["w"], toy["prm"], toy["ctx"]
    W = S.client_updates(w)
    X = S.split_chunks(W, prm.slots)
    cts = np.zeros((w.n_clients, w.chunks, 2, prm.L + 1, prm.N), dtype=np.uint64)
    for i in range(w.n_clients):
        for k in range(w.chunks):
            cts[i, k], _ = _enc(toy, X[i, k], i, k)
    D = ctx.distances(cts, toy["rlk"], toy["sched"], toy["rk"])
    assert np.array_equal(ctx.distances(cts, toy["rlk"], toy["sched"], toy["rk"], rot_level=prm.L - 1), D)
    D0 = ctx.distances(cts, toy["rlk"], toy["sched"], toy["rk"], rot_level=0)
    assert D0.shape == (w.n_pairs, 2, 1, prm.N)
    sc = prm.scale ** 2 / prm.q[prm.L]
    tol = toy_distance_tolerance(prm)
    dist = np.zeros((w.n_clients, w.n_clients))
    k = 0
    for i in range(w.n_clients):
        for j in range(i + 1, w.n_clients):
            v = ctx.decrypt(toy["s"], D0[k], 0, sc)
            ref = float(np.sum((W[i] - W[j]) ** 2))
            assert np.abs(v - ref).max() <= tol
            dist[i, j] = dist[j, i] = v[0]
            k += 1
    ref_d = np.array([[np.sum((W[i] - W[j]) ** 2) for j in range(w.n_clients)] for i in range(w.n_clients)])
    assert kgc.krum_select(dist, f=w.f, n_select=w.n_select) == kgc.krum_select(ref_d, f=w.f, n_select=w.n_select)
    # a fresh ciphertext dropped to level 0: its decryption residues mod q_0 are those of the
    # full ciphertext
    ct = cts[0, 0]
    full = ctx.decrypt_residues(toy["s"], ct, prm.L)
    low = ctx.decrypt_residues(toy["s"], np.ascontiguousarray(ct[:, :1]), 0)
    assert np.array_equal(full[0], low[0])


@pytest.mark.slow
def test_production_parameters_square_relin_rescale_rotate():
    prm = O.params_production()
    ctx = O.Context(prm)
    N = prm.N
    s = S.secret_key(3, 98, N)
    a, e = S.pk_rand(3, 98, prm.q, N)
    pk = ctx.pk_gen(s, a, e)
    qp = prm.q + prm.p
    ar, er = S.swk_rand(3, 98, qp, prm.dnum, N, None)
    rlk = ctx.swk_gen(s, 0, ar, er)
    ar, er = S.swk_rand(3, 98, qp, prm.dnum, N, 5)
    rk5 = ctx.swk_gen(s, ctx.galois(5), ar, er)
    z = np.random.default_rng(19).normal(0, 0.05, prm.slots)
    r, e0, e1 = S.enc_rand(3, 98, 0, 0, N)
    ct = ctx.encrypt(pk, ctx.encode(z, prm.scale), r, e0, e1)
    sq = ctx.rescale(ctx.relin(ctx.tensor(ct, ct, prm.L), prm.L, rlk), prm.L)
    sc = prm.scale ** 2 / prm.q[prm.L]
    assert np.abs(ctx.decrypt(s, sq, prm.L - 1, sc) - z * z).max() < 1e-6
    rot = ctx.rotate_hoisted(sq, prm.L - 1, [5], [rk5])[0]
    assert np.abs(ctx.decrypt(s, rot, prm.L - 1, sc) - np.roll(z * z, -5)).max() < 1e-6


# ------------------------------------------------------------------------- device-randomness mode

def _numpy_philox_block(ctr, key):
    """numpy's Philox4x64-10 bit generator advances its counter before each block, so the block
    of counter c is the first output of a generator started at c - 1 (256-bit little-endian)."""
    c = list(ctr)
    for i in range(4):  # c - 1 with borrow
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = (1 << 64) - 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


def test_philox_matches_numpy_bit_generator():
    g = np.random.default_rng(31)
    cases = [([0, 0, 0, 0], [0, 0]), ([1, 0, 0, 0], [0, 0]), ([0, 0, 0, 1], [2 ** 64 - 1, 5])]
    for _ in range(20):
        cases.append(([int(v) for v in g.integers(0, 2 ** 63, 4)], [int(v) for v in g.integers(0, 2 ** 63, 2)]))
    for ctr, key in cases:
        assert O.philox4x64(ctr, key) == _numpy_philox_block(ctr, key)


def test_encryption_sampler_follows_its_rule_and_distribution():
    seed, first, count, n = 77, 1000, 3, 4096
    r, e0, e1 = O.sample_enc(seed, first, count, n)
    # the rule, recomputed from numpy's generator for a few coefficients
    m21 = (1 << 21) - 1
    for b, k in [(0, 0), (1, 17), (2, n - 1)]:
        w = _numpy_philox_block([k, first + b, 0, 0], [seed, 0])
        assert r[b, k] == (((w[0] >> 32) * 3) >> 32) - 1
        for p, e in ((1, e0), (2, e1)):
            w = _numpy_philox_block([k, first + b, p, 0], [seed, 0])
            assert e[b, k] == bin(w[0] & m21).count("1") - bin(w[1] & m21).count("1")
    # distributions: ternary uniform, centred binomial with variance 21/2
    vals, counts = np.unique(r, return_counts=True)
    assert list(vals) == [-1, 0, 1]
    expect = r.size / 3
    assert ((counts - expect) ** 2 / expect).sum() < 20  # chi-square, 2 dof
    e = np.concatenate([e0.ravel(), e1.ravel()])
    assert np.abs(e).max() <= 21
    assert abs(e.mean()) < 0.05 and abs(e.var() - 10.5) < 0.3
    # ciphertext index and seed change the draws
    r2, _, _ = O.sample_enc(seed, first + 1, 1, n)
    assert np.array_equal(r2[0], r[1]) and not np.array_equal(r2[0], r[0])
    r3, _, _ = O.sample_enc(seed + 1, first, 1, n)
    assert not np.array_equal(r3[0], r[0])
