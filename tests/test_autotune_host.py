"""Host logic of the autotuner on the CPU: candidate schedules filtered by the loaded rotation
keys and the key budget, the fastest schedule kept, then each knob set by coordinate descent and
left on the context.  Device timing is replaced by a deterministic cost model (no GPU); the GPU
test (tests/test_tuning.py) checks that every option computes the same bits."""
import pytest

pytest.importorskip("torch")

from paper_2408_06197_b300 import autotune  # noqa: E402
from paper_2408_06197_b300 import lancelot as LC  # noqa: E402


class FakeCtx:
    log_n, N, nq, np_, dnum, L = 15, 1 << 15, 15, 4, 4, 14

    def __init__(self):
        self.knobs = {k: opts[0] for k, opts in LC.TUNING_OPTIONS.items()}
        self.calls = []

    def set_tuning(self, knob, value):
        assert value in LC.TUNING_OPTIONS[knob]
        self.knobs[knob] = value

    def get_tuning(self, knob):
        return self.knobs[knob]

    def tuning(self):
        return {LC.TUNING_NAMES[k]: v for k, v in self.knobs.items()}

    def empty(self, *shape):
        return None

    def distances(self, evk, cts, n, chunks, scale, mode=0, groups=None, out=None):
        self.calls.append((tuple(groups), mode, dict(self.knobs)))


class FakeEvk:
    def __init__(self, rotations):
        self.rotations = list(rotations)


# cost model: schedule base cost, plus one preferred option per knob (the second one listed)
BASE = {"log": 50.0, "g2qp": 40.0, "g3qp": 30.0}


def _cost(ctx, groups):
    name = {tuple(v): k for k, v in autotune.candidate_schedules(15).items()}[tuple(groups)]
    ms = BASE.get(name, 35.0 + len(groups))  # the other compositions: slower than g3qp
    for knob, opts in LC.TUNING_OPTIONS.items():
        ms += 0.0 if ctx.knobs[knob] == opts[1 % len(opts)] else 1.0
    return ms


@pytest.fixture
def model(monkeypatch):
    def time_ms(ctx, fn, reps):
        fn()
        return _cost(ctx, ctx.calls[-1][0])
    monkeypatch.setattr(autotune, "_time_ms", time_ms)


def _all_rots():
    rots = set()
    for s in autotune.candidate_schedules(15).values():
        rots |= set(LC.rotations_of_schedule(s))
    return sorted(rots)


def test_picks_fastest_schedule_then_each_knob(model):
    ctx = FakeCtx()
    res = autotune.tune(ctx, FakeEvk(_all_rots()), None, 10, 64, 1.0)
    assert res["schedule"] == "g3qp" and res["groups"] == [3, 3, 3, 3, 2]
    assert res["mode"] == LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM
    for knob, opts in LC.TUNING_OPTIONS.items():  # coordinate descent found every preferred option
        assert ctx.knobs[knob] == opts[1 % len(opts)]
        assert res["knobs"][LC.TUNING_NAMES[knob]] == opts[1 % len(opts)]
    assert res["ms"] == pytest.approx(30.0)
    n_opts = sum(len(o) for o in LC.TUNING_OPTIONS.values())
    n_sched = len(autotune.candidate_schedules(15))
    assert res["schedules"] == n_sched >= 10
    assert len(res["trials"]) == n_sched + n_opts
    assert res["key_bytes"] == autotune.key_bytes(ctx, 31 + 1)


def test_candidates_need_their_keys_and_fit_the_budget(model):
    ctx = FakeCtx()
    log_keys = LC.rotations_of_schedule(autotune.candidate_schedules(15)["log"])
    res = autotune.tune(ctx, FakeEvk(log_keys), None, 10, 64, 1.0)
    assert res["schedule"] == "log"  # only the log-step keys are loaded
    # a budget that holds the 14 + 1 log-step keys but not the 21 + 1 or more of the others
    budget = autotune.key_bytes(ctx, 15) * 1.01
    res = autotune.tune(FakeCtx(), FakeEvk(_all_rots()), None, 10, 64, 1.0, key_budget_bytes=budget)
    assert res["schedule"] == "log"
    with pytest.raises(LC.LancelotError):
        autotune.tune(FakeCtx(), FakeEvk([1, 2]), None, 10, 64, 1.0)


def test_cache_file_reuses_a_tuned_shape(model, tmp_path):
    path = str(tmp_path / "tune.json")
    ctx = FakeCtx()
    first = autotune.tune(ctx, FakeEvk(_all_rots()), None, 10, 64, 1.0, cache_path=path, device="B300")
    assert "cached" not in first
    n_calls = len(ctx.calls)
    ctx2 = FakeCtx()
    again = autotune.tune(ctx2, FakeEvk(_all_rots()), None, 10, 64, 1.0, cache_path=path, device="B300")
    assert again["cached"] and ctx2.calls == []          # nothing timed
    assert again["schedule"] == first["schedule"] and again["groups"] == first["groups"]
    assert ctx2.tuning() == first["knobs"]               # the context got the cached knobs
    other = autotune.tune(FakeCtx(), FakeEvk(_all_rots()), None, 10, 32, 1.0, cache_path=path, device="B300")
    assert "cached" not in other                         # another shape is tuned and added
    import json
    assert len(json.load(open(path))) == 2
    assert n_calls > 0


def test_candidate_schedules_are_every_composition_up_to_four_bits():
    """The search space: "log" plus every largest-first composition of log2(N/2) into groups of at
    most 4 bits with at most one single-bit group; each needs 2^g - 1 keys per group."""
    c = autotune.candidate_schedules(15)
    assert c["log"] == [1] * 14 and c["g2qp"] == [2] * 7 and c["g3qp"] == [3, 3, 3, 3, 2]
    assert c["g4442qp"] == [4, 4, 4, 2] and c["g4433qp"] == [4, 4, 3, 3]
    qp = [v for k, v in c.items() if k != "log"]
    assert len(qp) == 13 and len({tuple(v) for v in qp}) == 13
    for v in qp:
        assert sum(v) == 14 and v == sorted(v, reverse=True) and max(v) <= 4 and v.count(1) <= 1
    assert autotune.schedule_keys([4, 4, 4, 2]) == 48 and autotune.schedule_keys([1] * 14) == 14
    # the union of all their rotation keys (what a server loads to search them all)
    rots = set()
    for v in c.values():
        rots |= set(LC.rotations_of_schedule(v))
    assert len(rots) == 61
