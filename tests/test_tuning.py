"""Every tile-shape option computes the same bits, and the autotuner leaves the context on a
valid setting (GPU)."""
import numpy as np
import pytest

import oracle as O
import synth as S
from test_gpu_parity import Env

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2408_06197_b300 import autotune
    sched = autotune.candidate_schedules(12)
    rots = set()
    for s in sched.values():
        rots |= set(O.rotations_of_schedule(s))
    return Env("toy", 12, S.CFG_TOY, extra_rot=sorted(rots))


def _inputs(env, n=6, chunks=3):
    w = S.Workload("tune", S.CFG_TOY, 12, n, chunks * env.prm.slots - 3, 12, (n - 1,), "scale10", 1, 1)
    X = S.split_chunks(S.client_updates(w), env.prm.slots)
    return env.encrypt_both(X, range(n), range(chunks))  # (oracle cts, GPU cts) of the same inputs


def test_every_tuning_option_gives_identical_distances(env):
    LC = env.LC
    g = env.g
    _, gcs = _inputs(env)
    sched = [3, 3, 3, 2]
    mode = LC.LC_MODE_BATCHED | LC.LC_HOIST_QP_SUM
    ref, _ = g.distances(env.gevk, gcs, 6, 3, env.prm.scale, mode=mode, groups=sched)
    for knob, options in LC.TUNING_OPTIONS.items():
        for v in options:
            g.set_tuning(knob, v)
            assert g.get_tuning(knob) == v
            got, _ = g.distances(env.gevk, gcs, 6, 3, env.prm.scale, mode=mode, groups=sched)
            assert torch.equal(got, ref), (LC.TUNING_NAMES[knob], v)
        g.set_tuning(knob, options[0])
    with pytest.raises(LC.LancelotError):
        g.set_tuning(LC.LC_TUNE_TENSOR_WARPS, 7)
    assert g.get_tuning(LC.LC_TUNE_TENSOR_WARPS) == LC.TUNING_OPTIONS[LC.LC_TUNE_TENSOR_WARPS][0]


def test_autotune_picks_a_loaded_schedule_and_valid_knobs(env):
    from paper_2408_06197_b300 import autotune
    LC = env.LC
    g = env.g
    ocs, gcs = _inputs(env)
    res = autotune.tune(g, env.gevk, gcs, 6, 3, env.prm.scale, reps=2)
    assert res["schedule"] in autotune.candidate_schedules(12)
    for knob, name in LC.TUNING_NAMES.items():
        assert res["knobs"][name] in LC.TUNING_OPTIONS[knob]
        assert g.get_tuning(knob) == res["knobs"][name]
    n_opts = sum(len(o) for o in LC.TUNING_OPTIONS.values())
    assert len(res["trials"]) == len(autotune.candidate_schedules(12)) + n_opts
    # the tuned setting computes the oracle's bits
    ref = env.o.distances(ocs, env.orlk, res["groups"], env.ork, qp_sum=res["schedule"].endswith("qp"))
    got, _ = g.distances(env.gevk, gcs, 6, 3, env.prm.scale, mode=res["mode"], groups=res["groups"])
    assert np.array_equal(env.g_coeff(got, env.L - 1), env.o_coeff(ref))
    # a key budget below one key set leaves no candidate
    with pytest.raises(LC.LancelotError):
        autotune.tune(g, env.gevk, gcs, 6, 3, env.prm.scale, reps=1, key_budget_bytes=1)
    for knob, options in LC.TUNING_OPTIONS.items():
        g.set_tuning(knob, options[0])



def test_alu_probes_count_their_operations_and_reject_bad_arguments(env):
    """The integer-pipe probes report blocks x 256 threads x iters x 64 operations (32 butterflies
    per iteration for the butterfly probe), a positive device time, and rates below the issue
    ceiling of the GPU (148 SMs x 128 thread instructions per clock at most 2.1 GHz)."""
    LC, g = env.LC, env.g
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * 2.1e9
    for kind, per in ((LC.LC_PROBE_IMAD, 64), (LC.LC_PROBE_IMAD_WIDE, 64), (LC.LC_PROBE_NTT_BFLY, 32)):
        r = g.alu_probe(kind, iters=64, blocks_per_sm=2)
        assert r["ops"] == sms * 2 * 256 * 64 * per
        assert r["ms"] > 0 and r["ops_per_s"] < ceiling
    for bad in ((3, 64, 2), (0, 0, 2), (0, 64, 0), (0, 64, 33)):
        with pytest.raises(LC.LancelotError):
            g.alu_probe(*bad)
    g.sync()


def test_bounded_wait_runs_out_and_is_reported(env):
    """The bounded shared-memory-barrier wait of the bulk-copy kernels: a wait that completes
    returns LC_OK with the copied bytes intact; a wait on a barrier at which nothing arrives runs
    out after its poll limit and the next sync reports LC_ETIMEOUT (-6); the context stays usable
    and the error word is cleared."""
    LC, g = env.LC, env.g
    assert g.wait_selftest(never_arrive=False) == 0
    assert g.wait_selftest(never_arrive=True, max_polls=1 << 12) == -6
    assert g.wait_selftest(never_arrive=False) == 0
    a = np.stack([np.random.default_rng(3).integers(0, q, size=env.N, dtype=np.uint64) for q in env.prm.q])
    ev = g.to_eval(LC.u64_to_torch(a), env.L)
    assert np.array_equal(LC.torch_to_u64(g.to_coeff(ev, env.L)), a)
    g.sync()
