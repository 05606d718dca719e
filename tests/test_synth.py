"""The seeded input recipe on the CPU: distributions, Byzantine rules, workload shapes and
determinism of the generators that both the oracle and the CUDA path consume."""
import math

import numpy as np

import synth as S


def test_draws_are_deterministic_and_tagged():
    a = S.rng(0, S.CFG_PLAIN, 0, 3, 5, S.P_ENC_R).integers(0, 1 << 62, 8)
    b = S.rng(0, S.CFG_PLAIN, 0, 3, 5, S.P_ENC_R).integers(0, 1 << 62, 8)
    assert np.array_equal(a, b)
    for other in (S.rng(1, S.CFG_PLAIN, 0, 3, 5, S.P_ENC_R), S.rng(0, S.CFG_PLAIN, 1, 3, 5, S.P_ENC_R),
                  S.rng(0, S.CFG_PLAIN, 0, 4, 5, S.P_ENC_R), S.rng(0, S.CFG_PLAIN, 0, 3, 6, S.P_ENC_R),
                  S.rng(0, S.CFG_PLAIN, 0, 3, 5, S.P_ENC_E0)):
        assert not np.array_equal(a, other.integers(0, 1 << 62, 8))


def test_ternary_and_error_distributions():
    g = S.rng(7, 0, 0, 0, 0, 0)
    t = S.ternary(g, 300_000)
    assert t.dtype == np.int8 and set(np.unique(t)) == {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs(np.mean(t == v) - 1 / 3) < 0.005
    e = S.gaussian_error(S.rng(7, 0, 0, 0, 0, 1), 300_000)
    assert e.dtype == np.int32 and np.abs(e).max() <= S.ERR_BOUND
    assert abs(e.mean()) < 0.03 and abs(e.std() - S.SIGMA) < 0.03
    # a bound of 3 forces redraws: nothing beyond it survives
    assert np.abs(S.gaussian_error(S.rng(7, 0, 0, 0, 0, 2), 10_000, bound=3)).max() <= 3


def test_uniform_residues_stay_below_their_moduli():
    qs = [(1 << 40) - 87, (1 << 60) - 93, 97]
    r = S.uniform_residues(S.rng(1, 0, 0, 0, 0, 3), qs, 50_000)
    assert r.shape == (3, 50_000) and r.dtype == np.uint64
    for i, q in enumerate(qs):
        assert int(r[i].max()) < q
    assert abs(float(r[2].mean()) - 48.0) < 1.0  # uniform over [0, 97)


def test_client_updates_follow_the_byzantine_rules():
    w = S.Workload("t", S.CFG_PLAIN, 12, 4, 40_000, 0, (3,), "flip5", 1, 1)
    X = S.client_updates(w)
    honest = S.client_updates(S.Workload("t", S.CFG_PLAIN, 12, 4, 40_000, 0, (), "flip5", 1, 1))
    assert np.array_equal(X[:3], honest[:3])
    assert np.allclose(X[3], -5.0 * honest[3])
    assert abs(honest.std() - 0.01) < 2e-4 and abs(honest.mean()) < 2e-4
    for rule, check in (("scale10", lambda x, h: np.allclose(x, 10 * h)),
                        ("scale5", lambda x, h: np.allclose(x, 5 * h)),
                        ("noise0.1", lambda x, h: abs((x - h).std() - 0.1) < 2e-3)):
        wr = S.Workload("t", S.CFG_PLAIN, 12, 4, 40_000, 0, (3,), rule, 1, 1)
        assert check(S.client_updates(wr, [3])[0], honest[3])


def test_workload_shapes_match_the_configurations():
    assert (S.TOY.n_clients, S.TOY.log_n, S.TOY.chunks, S.TOY.n_pairs) == (4, 12, 1, 6)
    assert (S.PLAIN.n_clients, S.PLAIN.chunks, S.PLAIN.n_pairs, S.PLAIN.byzantine) == (10, 64, 45, (8, 9))
    assert (S.BATCHED.n_clients, S.BATCHED.chunks, S.BATCHED.n_pairs) == (50, 256, 1225)
    assert S.BATCHED.byzantine == tuple(range(40, 50))
    x = S.split_chunks(np.arange(5.0), 4)
    assert x.shape == (2, 4) and list(x[1]) == [4.0, 0.0, 0.0, 0.0]


def test_uneven_jobs_and_serving_stream():
    jobs = S.uneven_jobs()
    assert len(jobs) == 8 and [j.job for j in jobs] == list(range(8))
    for j in jobs:
        assert j.n_clients in (5, 10, 20, 40) and j.d in (1 << 16, 1 << 18, 1 << 20, 1 << 22)
        nb = j.n_clients // 5
        assert j.byzantine == tuple(range(j.n_clients - nb, j.n_clients)) and j.byz_rule == "scale5"
    assert [(j.n_clients, j.d) for j in jobs] == [(j.n_clients, j.d) for j in S.uneven_jobs()]
    r1 = S.serving_rounds(n_rounds=4000, rate=1.0)
    r5 = S.serving_rounds(n_rounds=4000, rate=5.0)
    assert [(a.tenant, a.n_clients, a.d) for a in r1] == [(b.tenant, b.n_clients, b.d) for b in r5]
    gaps = np.diff([0.0] + [a.arrival for a in r5])
    assert abs(gaps.mean() - 0.2) < 0.01 and np.all(gaps > 0)
    assert abs(np.var(gaps) - 0.04) < 0.005           # exponential: variance = mean^2
    assert set(a.tenant for a in r1) == {0, 1, 2, 3}
    assert math.isclose(r5[-1].arrival * 5.0, r1[-1].arrival, rel_tol=1e-12)
