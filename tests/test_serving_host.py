"""Host logic of the serving loop on the CPU: admission by the HBM budget in arrival order, an
oversized round admitted alone, rounds that arrive together sharing batches, the KGC step between
the phases, and the footprint returned when a round finishes.  The library calls are replaced by
recording fakes (no GPU); the device arithmetic itself is covered by tests/test_serving.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2408_06197_b300 import lancelot as LC  # noqa: E402
from paper_2408_06197_b300 import serving as SV  # noqa: E402


class FakeCtx:
    """The context attributes the scheduler reads (production shape), with recorded calls."""
    log_n, N, nq, L = 15, 1 << 15, 15, 14
    scale = float(1 << 40)
    q = [(1 << 40) - 87] * 15

    def __init__(self):
        self.syncs = 0

    def sync(self):
        self.syncs += 1

    def decrypt_const(self, s, out_dist, level, scale):
        return np.asarray(out_dist, dtype=np.float64)

    def encrypt(self, pk, m, r, e0, e1):
        return ("masks", m.shape[0])


class FakeJob:
    def __init__(self, evk, cts, n, chunks, masks=None):
        self.evk, self.cts, self.n, self.chunks, self.masks = evk, cts, n, chunks, masks
        self.out_dist = None
        self.out_agg = None


@pytest.fixture
def fake_lib(monkeypatch):
    calls = {"dist": [], "agg": []}

    def batch_distances(ctx, jobs, flags=0, groups=None):
        calls["dist"].append([j.rid for j in jobs])
        for j in jobs:  # distances of client i to j: |i - j| + 1 (client 0 is the outlier-free centre)
            j.out_dist = np.array([abs(a - b) + 1.0 for a in range(j.n) for b in range(a + 1, j.n)])

    def batch_aggregate(ctx, jobs):
        calls["agg"].append([j.rid for j in jobs])
        for j in jobs:
            j.out_agg = ("agg", j.chunks)

    monkeypatch.setattr(LC, "Job", FakeJob)
    monkeypatch.setattr(LC, "batch_distances", batch_distances)
    monkeypatch.setattr(LC, "batch_aggregate", batch_aggregate)
    return calls


def _server(budget_rounds, tenants=2):
    ctx = FakeCtx()
    ten = [SV.Tenant(evk=f"evk{t}", pk=f"pk{t}", s=np.zeros(ctx.N, np.int8)) for t in range(tenants)]

    def ingest(r):
        return ("cts", r.rid)

    def mask_rand(r, i):
        z = np.zeros(ctx.N)
        return z.astype(np.int8), z.astype(np.int32), z.astype(np.int32)

    probe = SV.Server(ctx, ten, 1.0, ingest, mask_rand, groups=[3, 3, 3, 3, 2])
    one = probe.footprint(SV.Round(0, 0, 10, 64, 0.0))
    srv = SV.Server(ctx, ten, budget_rounds * one * 1.0001, ingest, mask_rand, groups=[3, 3, 3, 3, 2])
    return srv, one


def _tag_jobs(srv):
    """Make the fake jobs carry their round id (for the call records)."""
    orig = srv._admit

    def admit():
        before = set(id(r) for r in srv.active)
        orig()
        for r in srv.active:
            if id(r) not in before:
                r.job.rid = r.rid
    srv._admit = admit


def test_admission_by_budget_in_arrival_order(fake_lib):
    srv, one = _server(budget_rounds=2)
    _tag_jobs(srv)
    rounds = [SV.Round(i, i % 2, 10, 64, 0.0, f=1, n_select=3) for i in range(5)]
    for r in rounds:
        srv.submit(r)
    srv.tick()
    # two rounds fit: they share the first distances batch; the others wait in order
    assert fake_lib["dist"][0] == [0, 1]
    assert [r.rid for r in srv.waiting] == [2, 3, 4]
    assert srv.used == pytest.approx(2 * one)
    while srv.tick():
        assert srv.used <= srv.budget
    assert [r.rid for r in srv.done] == [0, 1, 2, 3, 4]
    assert srv.used == pytest.approx(0.0)
    assert all(r.state == SV.DONE and r.cts is None for r in srv.done)
    # every round went through distances, the KGC step and the aggregate, in that order
    for r in srv.done:
        assert r.t_admit <= r.t_dist <= r.t_kgc <= r.t_done
        assert r.selected is not None and len(r.selected) == 3
    assert sorted(x for b in fake_lib["agg"] for x in b) == [0, 1, 2, 3, 4]


def test_oversized_round_is_admitted_alone(fake_lib):
    srv, one = _server(budget_rounds=1)
    _tag_jobs(srv)
    big = SV.Round(0, 0, 40, 256, 0.0, f=8, n_select=21)
    small = SV.Round(1, 1, 5, 4, 0.0)
    srv.submit(big)
    srv.submit(small)
    assert srv.footprint(big) > srv.budget
    srv.tick()
    assert fake_lib["dist"][0] == [0]          # alone, although it exceeds the budget
    assert [r.rid for r in srv.waiting] == [1]  # nothing joins it
    while srv.tick():
        pass
    assert [r.rid for r in srv.done] == [0, 1]
    assert srv.stats["max_used"] == pytest.approx(srv.footprint(big))


def test_rounds_arriving_while_others_run_join_the_next_wave(fake_lib):
    srv, one = _server(budget_rounds=4)
    _tag_jobs(srv)
    srv.submit(SV.Round(0, 0, 10, 64, 0.0))
    srv.tick()                                   # round 0: distances, KGC
    srv.submit(SV.Round(1, 1, 5, 16, 0.0))
    srv.submit(SV.Round(2, 0, 20, 4, 0.0))
    srv.tick()                                   # round 0 aggregates while 1 and 2 start
    assert fake_lib["agg"][0] == [0]
    assert fake_lib["dist"][1] == [1, 2]
    while srv.tick():
        pass
    assert fake_lib["agg"][1] == [1, 2]
    assert srv.stats["rounds_batched"] == 3 and srv.stats["distance_batches"] == 2


def test_latency_summary():
    rs = []
    for i, lat in enumerate([0.1, 0.2, 0.3, 0.4]):
        r = SV.Round(i, 0, 5, 1, arrival=1.0)
        r.t_done = 1.0 + lat
        r.kgc_seconds = 0.001 * (i + 1)
        rs.append(r)
    s = SV.latency_summary(rs)
    assert s["rounds"] == 4 and s["pairs"] == 40
    assert s["p50_ms"] == pytest.approx(250.0)
    assert s["p99_ms"] == pytest.approx(397.0)


def test_cancelled_rounds_leave_and_release_their_budget(fake_lib):
    srv, one = _server(budget_rounds=1)
    _tag_jobs(srv)
    for i in range(4):
        srv.submit(SV.Round(i, 0, 10, 64, 0.0))
    assert srv.cancel(2)                       # waiting: leaves the queue at once
    assert [r.rid for r in srv.waiting] == [0, 1, 3]
    srv.tick()                                 # round 0: distances + KGC
    assert srv.cancel(0)                       # admitted: dropped at the next phase boundary
    srv.tick()
    assert fake_lib["agg"] == []               # round 0 never aggregated
    assert fake_lib["dist"][1] == [1]          # its budget went to the next round
    assert not srv.cancel(0) and not srv.cancel(99)
    while srv.tick():
        pass
    assert [r.rid for r in srv.done] == [1, 3]
    assert sorted(r.rid for r in srv.cancelled) == [0, 2]
    assert all(r.state == SV.CANCELLED for r in srv.cancelled)
    assert srv.used == pytest.approx(0.0)


# ------------------------------------------------------------------------------- lanes (device KGC)

class _Arr:
    """Stands for a small device tensor: .cpu() gives back something with .numpy() / .tolist()."""

    def __init__(self, v):
        self.v = np.asarray(v)

    def cpu(self):
        return self

    def numpy(self):
        return self.v

    def tolist(self):
        return self.v.tolist()


class FakeKgcKey:
    def __init__(self, ctx, s):
        self.ctx = ctx

    def readout(self, out_dist, level, scale):
        return _Arr(out_dist)

    def krum(self, vals, n, f, n_select, average):
        return _Arr(np.ones(n)), _Arr(np.arange(n_select))


class FakeLane(SV.Lane):
    """A lane whose batches finish after `polls` completion checks (time on the GPU)."""

    def __init__(self, ctx, max_pairs, name, polls, log):
        super().__init__(ctx, max_pairs, name)
        self.polls, self.log = polls, log

    def mark(self):
        lane, state = self, {"left": self.polls}

        class _M:
            def query(self):
                state["left"] -= 1
                if state["left"] <= 0:
                    lane.log.append(("done", lane.name))
                    return True
                return False
        return _M()


class FakeLaneCtx(FakeCtx):
    stream = None

    def encrypt_const_seeded(self, pk, w, scale, seed, first):
        return ("masks", first)


def _lane_server(monkeypatch, fake_lib, polls_fast, polls_bulk, fast_pairs=45):
    monkeypatch.setattr(LC, "KgcKey", FakeKgcKey)
    log = []
    fast, bulk = FakeLaneCtx(), FakeLaneCtx()
    lanes = [FakeLane(fast, fast_pairs, "fast", polls_fast, log), FakeLane(bulk, None, "bulk", polls_bulk, log)]
    ten = [SV.Tenant(evk=f"evk{t}", pk=f"pk{t}", s=np.zeros(fast.N, np.int8)) for t in range(2)]
    srv = SV.Server(fast, ten, 1e15, lambda r: ("cts", r.rid), lambda r, i: None, groups=[3, 3, 3, 3, 2],
                    device_kgc_seed=5, lanes=lanes)
    orig = srv._admit_lanes

    def admit():
        before = set(id(r) for r in srv.active)
        orig()
        for r in srv.active:
            if id(r) not in before:
                r.job.rid = r.rid
    srv._admit_lanes = admit
    return srv, lanes, log


def test_lanes_keep_small_rounds_clear_of_a_large_one(monkeypatch, fake_lib):
    """A large round (780 pairs) goes to the bulk lane; small rounds that arrive while it is on
    the GPU launch on the fast lane at once and finish before it."""
    srv, lanes, log = _lane_server(monkeypatch, fake_lib, polls_fast=2, polls_bulk=50)
    rounds = [SV.Round(0, 0, 40, 256, 0.0, f=8, n_select=21), SV.Round(1, 1, 5, 4, 0.0, n_select=2),
              SV.Round(2, 0, 10, 16, 0.0, n_select=5)]
    done = srv.run(rounds, realtime=False)
    assert [r.rid for r in done][-1] == 0          # the large round finishes last
    assert fake_lib["dist"][0] in ([0], [1, 2])    # separate batches per lane
    assert sorted(map(tuple, fake_lib["dist"])) == [(0,), (1, 2)]
    by = {r.rid: r for r in done}
    assert by[0].lane == 1 and by[1].lane == 0 and by[2].lane == 0
    # both small rounds were done while the large round's batch was still in flight
    assert log.index(("done", "fast")) < log.index(("done", "bulk"))
    for r in done:
        assert r.state == SV.DONE and r.selected == list(range(r.n_select))
        assert r.distances.shape == (r.n, r.n)
    assert srv.used == pytest.approx(0.0) and not srv.active
    assert lanes[0].batches == 1 and lanes[1].batches == 1


def test_lanes_one_batch_per_lane_in_flight(monkeypatch, fake_lib):
    """Rounds that reach a busy lane wait and share its next batch; every round's distances, KGC
    step and aggregate go out in one batch (no host round trip between them)."""
    srv, lanes, log = _lane_server(monkeypatch, fake_lib, polls_fast=3, polls_bulk=3, fast_pairs=1000)
    srv.submit(SV.Round(0, 0, 10, 64, 0.0))
    srv._admit_lanes()
    assert srv._launch(0)
    for i in (1, 2, 3):
        srv.submit(SV.Round(i, i % 2, 5, 8, 0.0))
    srv._admit_lanes()
    assert lanes[0].inflight is not None
    assert all(r.state == SV.DIST for r in srv.active if r.rid > 0)
    while not srv._poll():
        pass
    assert srv._launch(0)
    assert fake_lib["dist"] == [[0], [1, 2, 3]] and fake_lib["agg"] == [[0], [1, 2, 3]]
    while not srv._poll():
        pass
    assert [r.rid for r in srv.done] == [0, 1, 2, 3]


def test_lanes_cancel_before_launch_and_in_flight(monkeypatch, fake_lib):
    srv, lanes, log = _lane_server(monkeypatch, fake_lib, polls_fast=2, polls_bulk=2)
    for i in range(3):
        srv.submit(SV.Round(i, 0, 5, 8, 0.0))
    srv._admit_lanes()
    assert srv.cancel(1)                      # admitted, not launched: dropped at the launch
    srv._launch(0)
    assert fake_lib["dist"] == [[0, 2]]
    assert srv.cancel(2)                      # in flight: finishes on the GPU, then leaves
    while not srv._poll():
        pass
    assert [r.rid for r in srv.done] == [0]
    assert sorted(r.rid for r in srv.cancelled) == [1, 2]
    assert srv.used == pytest.approx(0.0)


def test_last_lane_must_take_every_size():
    ctx = FakeLaneCtx()
    with pytest.raises(ValueError):
        SV.Server(ctx, [], 1.0, None, None, lanes=[SV.Lane(ctx, 10)])
