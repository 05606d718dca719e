"""Serving loop for encrypted aggregation rounds (continuous batching on one GPU).

A round is one federated-learning aggregation of one tenant (Algorithm 1): its clients'
ciphertexts arrive on the device, the server computes the encrypted pair distances, the key
generation center decrypts them, selects the clients (Algorithm 2) and returns an encrypted
mask, and the server computes the masked aggregate.  The loop

* admits waiting rounds in arrival order while their device footprint fits the HBM budget;
* at every tick runs ONE batched distances call over all admitted rounds in the distance phase
  and ONE batched aggregate call over all rounds in the aggregate phase
  (lc_batch_distances / lc_batch_aggregate: rounds of different sizes and tenants share the
  same launches, so rounds that arrive while others run join the next wave);
* runs the KGC step between the phases (read-out of the distances on the GPU, Krum /
  Multi-Krum on the host, encryption of the masks on the GPU) and times it separately;
* keeps the tenants' evaluation keys resident for the whole run.

With the KGC step on the device a round needs no host round trip, and the loop runs
asynchronously on lanes instead of ticks: a lane is a CUDA stream with its own library context;
one batch per lane is in flight at a time, and it carries its rounds all the way (distances,
read-out, selection, mask encryption, aggregate) before a CUDA event marks them done.  With two
lanes -- small rounds on a high-priority stream, rounds above a pair cap on a low-priority one --
a large round no longer holds back the small rounds that arrive while it runs: their batches
launch at once and the GPU's block scheduler gives their blocks precedence.

Results of a round do not depend on which other rounds share its batches or its lane (exact
integer arithmetic; every context has the same tables); tests/test_serving.py checks this.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np
import torch

from . import kgc
from . import lancelot as LC

WAITING, DIST, AGG, DONE, CANCELLED = "waiting", "distances", "aggregate", "done", "cancelled"
RUNNING = "running"  # lanes: the round's whole batch (distances .. aggregate) is on the GPU


class Lane:
    """A CUDA stream with its own library context (own scratch arena).  Batches on one lane run
    one after another; batches on different lanes overlap on the device.  Rounds with at most
    `max_pairs` pairs go to the first lane that takes them (None: any size)."""

    def __init__(self, ctx: "LC.Context", max_pairs: Optional[int] = None, name: str = ""):
        self.ctx, self.max_pairs, self.name = ctx, max_pairs, name
        self.inflight = None  # (completion marker, rounds)
        self.batches = 0

    def stream(self):
        return getattr(self.ctx, "stream", None)

    def mark(self):
        """A completion marker for the work enqueued on this lane so far (query() -> bool)."""
        ev = torch.cuda.Event()
        ev.record(self.ctx.stream)
        return ev

    def takes(self, r: "Round") -> bool:
        return self.max_pairs is None or r.pairs <= self.max_pairs


@dataclasses.dataclass
class Tenant:
    """A tenant's resident keys.  `s` stands for the KGC's secret (the KGC step runs in-process)."""
    evk: "LC.EvalKeys"
    pk: torch.Tensor
    s: np.ndarray


@dataclasses.dataclass
class Round:
    rid: int
    tenant: int
    n: int
    chunks: int
    arrival: float                      # seconds since the start of the run
    f: int = 1                          # assumed Byzantine count for Krum
    n_select: int = 1                   # clients kept (Multi-Krum averages them)
    average: bool = False
    cts: Optional[torch.Tensor] = None  # device [n][chunks][2][nq][N], filled at admission
    state: str = WAITING
    job: Optional["LC.Job"] = None
    selected: Optional[List[int]] = None
    distances: Optional[np.ndarray] = None
    t_admit: float = 0.0
    t_dist: float = 0.0
    t_kgc: float = 0.0
    t_done: float = 0.0
    kgc_seconds: float = 0.0
    device_kgc: Optional[tuple] = None  # (read-out values, kept indices) on the device, until read back
    cancel_requested: bool = False
    lane: int = 0                       # lanes: index of the lane that runs the round

    @property
    def pairs(self) -> int:
        return self.n * (self.n - 1) // 2

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class Server:
    def __init__(self, ctx: "LC.Context", tenants: Sequence[Tenant], budget_bytes: float,
                 ingest: Callable[[Round], torch.Tensor],
                 mask_rand: Callable[[Round, int], tuple],
                 groups: Optional[Sequence[int]] = None, flags: int = LC.LC_HOIST_QP_SUM,
                 keep_outputs: bool = False, device_kgc_seed: Optional[int] = None,
                 lanes: Optional[Sequence[Lane]] = None):
        """keep_outputs: keep each finished round's device buffers (distances, masks, aggregate) on
        its Job; otherwise they are released as soon as the round no longer needs them.
        device_kgc_seed: run the KGC step on the device (resident KGC keys, device read-out and
        Krum, masks encrypted with device randomness of this seed, ciphertext indices
        rid * 2^20 + client) instead of on the host with `mask_rand`; run() then uses the
        asynchronous lane pipeline.  lanes: the lanes of that pipeline (default: one lane on
        `ctx`); the last lane must take rounds of any size."""
        self.ctx, self.tenants, self.budget = ctx, list(tenants), float(budget_bytes)
        self.keep = keep_outputs
        self.device_kgc_seed = device_kgc_seed
        self.lanes = list(lanes) if lanes else [Lane(ctx, None, "main")]
        if self.lanes[-1].max_pairs is not None:
            raise ValueError("the last lane must take rounds of any size")
        self._kgc_keys: Dict[tuple, "LC.KgcKey"] = {}
        self.ingest, self.mask_rand = ingest, mask_rand
        self.groups = list(groups) if groups else [2] * ((ctx.log_n - 1) // 2) + [1] * ((ctx.log_n - 1) % 2)
        self.flags = flags
        self.waiting: List[Round] = []
        self.active: List[Round] = []
        self.done: List[Round] = []
        self.cancelled: List[Round] = []
        self.used = 0.0
        self.stats = {"distance_batches": 0, "rounds_batched": 0, "aggregate_batches": 0, "max_used": 0.0}
        self.t0 = time.perf_counter()

    # ------------------------------------------------------------------ accounting
    def footprint(self, r: Round) -> float:
        c = self.ctx
        words = (r.n * r.chunks * 2 * c.nq + r.pairs * 2 * c.L + r.n * 2 * c.nq + r.chunks * 2 * c.L) * c.N
        return 8.0 * words

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, r: Round):
        self.waiting.append(r)

    def cancel(self, rid: int) -> bool:
        """Cancels round `rid`: a waiting round leaves the queue at once; an admitted round is
        dropped at its next phase boundary (a batch already on the GPU is not interrupted) and
        its device buffers and budget are released.  False if the round is unknown or done."""
        for r in self.waiting:
            if r.rid == rid:
                self.waiting.remove(r)
                r.state = CANCELLED
                self.cancelled.append(r)
                return True
        for r in self.active:
            if r.rid == rid:
                r.cancel_requested = True
                return True
        return False

    def _drop_cancelled(self):
        for r in [r for r in self.active if r.cancel_requested]:
            self.active.remove(r)
            self.used -= self.footprint(r)
            r.state = CANCELLED
            r.cts = None
            r.device_kgc = None
            if r.job is not None:
                r.job.cts = r.job.masks = r.job.out_dist = r.job.out_agg = None
            self.cancelled.append(r)

    # ------------------------------------------------------------------ scheduling
    def _admit(self):
        while self.waiting:
            r = self.waiting[0]
            fp = self.footprint(r)
            if self.used + fp > self.budget and self.active:
                break
            self.waiting.pop(0)
            self.used += fp
            self.stats["max_used"] = max(self.stats["max_used"], self.used)
            r.cts = self.ingest(r)
            r.job = LC.Job(self.tenants[r.tenant].evk, r.cts, r.n, r.chunks)
            r.state, r.t_admit = DIST, self.now()
            self.active.append(r)

    def _kgc_device(self, r: Round, c: Optional["LC.Context"] = None):
        """The KGC step without a host round trip: read-out and selection on the device, masks
        encrypted with device randomness; the selection is read back after the aggregate."""
        t = time.perf_counter()
        c = c or self.ctx
        ten = self.tenants[r.tenant]
        kk = (id(c), r.tenant)
        if kk not in self._kgc_keys:
            self._kgc_keys[kk] = LC.KgcKey(c, ten.s)
        key = self._kgc_keys[kk]
        sc = c.scale * c.scale / c.q[c.L]
        vals = key.readout(r.job.out_dist, c.L - 1, sc)
        w, sel = key.krum(vals, r.n, r.f, r.n_select, r.average)
        r.job.masks = c.encrypt_const_seeded(ten.pk, w, c.scale, self.device_kgc_seed, r.rid << 20)
        r.device_kgc = (vals, sel)
        if not self.keep:
            r.job.out_dist = None
        r.kgc_seconds = time.perf_counter() - t
        r.state, r.t_kgc = AGG, self.now()

    def _kgc(self, r: Round):
        """Decrypt the pair distances, select the clients, encrypt the mask (one ciphertext per
        client holding its weight in every slot)."""
        if self.device_kgc_seed is not None:
            return self._kgc_device(r)
        t = time.perf_counter()
        c, ten = self.ctx, self.tenants[r.tenant]
        sc = c.scale * c.scale / c.q[c.L]
        vals = c.decrypt_const(ten.s, r.job.out_dist, c.L - 1, sc)
        d = np.zeros((r.n, r.n))
        k = 0
        for i in range(r.n):
            for j in range(i + 1, r.n):
                d[i, j] = d[j, i] = vals[k]
                k += 1
        r.distances = d
        if not self.keep:
            r.job.out_dist = None  # the KGC has read the distances out
        r.selected = kgc.krum_select(d, r.f, r.n_select)
        w = kgc.mask_weights(r.n, r.selected, average=r.average)
        m = np.zeros((r.n, c.N), dtype=np.int64)
        m[:, 0] = np.rint(w * c.scale).astype(np.int64)  # a constant in every slot encodes to (w scale, 0, ...)
        rs, e0s, e1s = zip(*[self.mask_rand(r, i) for i in range(r.n)])
        r.job.masks = c.encrypt(ten.pk, m, np.stack(rs), np.stack(e0s), np.stack(e1s))
        r.kgc_seconds = time.perf_counter() - t
        r.state, r.t_kgc = AGG, self.now()

    def tick(self) -> bool:
        """One scheduler step; returns False when there was nothing to run."""
        self._drop_cancelled()
        self._admit()
        dist = [r for r in self.active if r.state == DIST]
        agg = [r for r in self.active if r.state == AGG]
        if not dist and not agg:
            return False
        if agg:
            LC.batch_aggregate(self.ctx, [r.job for r in agg])
            self.stats["aggregate_batches"] += 1
            self.ctx.sync()
            now = self.now()
            for r in agg:
                r.state, r.t_done = DONE, now
                if r.device_kgc is not None:  # selection record from the device
                    vals, sel = r.device_kgc
                    r.selected = [int(x) for x in sel.cpu().tolist()]
                    v = vals.cpu().numpy()
                    d = np.zeros((r.n, r.n))
                    iu = np.triu_indices(r.n, 1)
                    d[iu] = v
                    r.distances = d + d.T
                    r.device_kgc = None
                self.active.remove(r)
                self.done.append(r)
                self.used -= self.footprint(r)
                r.cts = None  # the round's ciphertexts leave the device
                r.job.cts = None
                if not self.keep:
                    r.job.masks = r.job.out_agg = None
        if dist:
            LC.batch_distances(self.ctx, [r.job for r in dist], LC.LC_MODE_BATCHED | self.flags, self.groups)
            self.stats["distance_batches"] += 1
            self.stats["rounds_batched"] += len(dist)
            self.ctx.sync()
            now = self.now()
            for r in dist:
                r.t_dist = now
                self._kgc(r)
        return True

    # ------------------------------------------------------------------ lanes (device KGC)
    def _lane_of(self, r: Round) -> int:
        for k, lane in enumerate(self.lanes):
            if lane.takes(r):
                return k
        return len(self.lanes) - 1

    def _admit_lanes(self):
        """Admission as in _admit; the round's ciphertexts are assembled on its lane's stream."""
        while self.waiting:
            r = self.waiting[0]
            fp = self.footprint(r)
            if self.used + fp > self.budget and self.active:
                break
            self.waiting.pop(0)
            self.used += fp
            self.stats["max_used"] = max(self.stats["max_used"], self.used)
            r.lane = self._lane_of(r)
            lane = self.lanes[r.lane]
            with torch.cuda.stream(lane.stream()):
                r.cts = self.ingest(r)
            r.job = LC.Job(self.tenants[r.tenant].evk, r.cts, r.n, r.chunks)
            r.state, r.t_admit = DIST, self.now()
            self.active.append(r)

    def _launch(self, k: int) -> bool:
        """Enqueues one batch on lane k: the distances of every admitted round of the lane, the
        KGC step of each, and their aggregates; nothing waits on the host."""
        lane = self.lanes[k]
        for r in [r for r in self.active if r.lane == k and r.state == DIST and r.cancel_requested]:
            self._release(r, CANCELLED)
        rs = [r for r in self.active if r.lane == k and r.state == DIST]
        if not rs:
            return False
        c = lane.ctx
        with torch.cuda.stream(lane.stream()):
            LC.batch_distances(c, [r.job for r in rs], LC.LC_MODE_BATCHED | self.flags, self.groups)
            now = self.now()
            for r in rs:
                r.t_dist = now
                self._kgc_device(r, c)
            LC.batch_aggregate(c, [r.job for r in rs])
            lane.inflight = (lane.mark(), rs)
        for r in rs:
            r.state = RUNNING
        lane.batches += 1
        self.stats["distance_batches"] += 1
        self.stats["aggregate_batches"] += 1
        self.stats["rounds_batched"] += len(rs)
        return True

    def _release(self, r: Round, state: str):
        self.active.remove(r)
        self.used -= self.footprint(r)
        r.state = state
        r.cts = None
        r.device_kgc = None
        if r.job is not None:
            r.job.cts = None
            if state == CANCELLED or not self.keep:
                r.job.masks = r.job.out_agg = None
            if state == CANCELLED:
                r.job.out_dist = None
        (self.cancelled if state == CANCELLED else self.done).append(r)

    def _poll(self) -> bool:
        """Completes the lanes whose batch has finished on the GPU."""
        progressed = False
        for lane in self.lanes:
            if lane.inflight is None or not lane.inflight[0].query():
                continue
            _, rs = lane.inflight
            lane.inflight = None
            now = self.now()
            with torch.cuda.stream(lane.stream()):  # read-backs on the (idle) lane stream
                for r in rs:
                    r.t_done = now
                    if r.cancel_requested:
                        self._release(r, CANCELLED)
                        continue
                    vals, sel = r.device_kgc
                    r.selected = [int(x) for x in sel.cpu().tolist()]
                    v = vals.cpu().numpy()
                    d = np.zeros((r.n, r.n))
                    d[np.triu_indices(r.n, 1)] = v
                    r.distances = d + d.T
                    self._release(r, DONE)
            progressed = True
        return progressed

    def _run_lanes(self, rounds: Sequence[Round], realtime: bool) -> List[Round]:
        pending = sorted(rounds, key=lambda r: r.arrival)
        self.t0 = time.perf_counter()
        while pending or self.waiting or self.active:
            now = self.now()
            while pending and (not realtime or pending[0].arrival <= now):
                self.submit(pending.pop(0))
            progressed = self._poll()
            self._admit_lanes()
            for k, lane in enumerate(self.lanes):
                if lane.inflight is None:
                    progressed |= self._launch(k)
            if not progressed:
                nxt = pending[0].arrival - self.now() if (pending and realtime) else 0.0
                time.sleep(max(0.0, min(0.0005, nxt)) if nxt > 0 or self.active else 0.0)
        return self.done

    def run(self, rounds: Sequence[Round], realtime: bool = True) -> List[Round]:
        """Feeds rounds at their arrival times (or all at once) and runs until all are done."""
        if self.device_kgc_seed is not None:
            return self._run_lanes(rounds, realtime)
        pending = sorted(rounds, key=lambda r: r.arrival)
        self.t0 = time.perf_counter()
        while pending or self.waiting or self.active:
            now = self.now()
            while pending and (not realtime or pending[0].arrival <= now):
                self.submit(pending.pop(0))
            if not self.tick() and pending:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - self.now())))
        return self.done


def latency_summary(done: Sequence[Round]) -> Dict[str, float]:
    lat = np.array([r.latency for r in done]) * 1e3
    kg = np.array([r.kgc_seconds for r in done]) * 1e3
    return {"rounds": len(done), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "kgc_p50_ms": float(np.percentile(kg, 50)), "pairs": int(sum(r.pairs for r in done))}


def round_on_device(ctx: "LC.Context", evk: "LC.EvalKeys", pk: torch.Tensor, kgc_key: "LC.KgcKey",
                    cts: torch.Tensor, n: int, chunks: int, f: int, n_select: int, seed: int, first: int,
                    groups: Optional[Sequence[int]] = None, flags: int = LC.LC_HOIST_QP_SUM,
                    average: bool = True, out: Optional[dict] = None) -> dict:
    """One aggregation round with the KGC step on the device (Algorithm 1 with Algorithm 2 in
    between): encrypted distances, read-out of the distances with the resident KGC key, Krum /
    Multi-Krum selection, mask ciphertexts encrypted with device randomness (ciphertext indices
    first .. first+n-1 of `seed`), masked aggregate.  Nothing synchronises the host, so the whole
    round can be captured in one CUDA graph (pass preallocated buffers in `out`)."""
    out = dict(out or {})
    L = ctx.L
    if "dist" not in out:
        out["dist"] = ctx.empty(n * (n - 1) // 2, 2, L, ctx.N)
    if "agg" not in out:
        out["agg"] = ctx.empty(chunks, 2, L, ctx.N)
    if "masks" not in out:
        out["masks"] = ctx.empty(n, 2, ctx.nq, ctx.N)
    if "values" not in out:
        out["values"] = torch.empty(n * (n - 1) // 2, dtype=torch.float64, device=cts.device)
    if "weights" not in out:
        out["weights"] = torch.empty(n, dtype=torch.float64, device=cts.device)
    if "selected" not in out:
        out["selected"] = torch.empty(n_select, dtype=torch.int32, device=cts.device)
    _, sc = ctx.distances(evk, cts, n, chunks, ctx.scale, mode=LC.LC_MODE_BATCHED | flags, groups=groups,
                          out=out["dist"])
    kgc_key.readout(out["dist"], L - 1, sc, out=out["values"])
    kgc_key.krum(out["values"], n, f, n_select, average, w=out["weights"], sel=out["selected"])
    ctx.encrypt_const_seeded(pk, out["weights"], ctx.scale, seed, first, out=out["masks"])
    ctx.masked_aggregate(evk, cts, n, chunks, ctx.scale, out["masks"], ctx.scale, out=out["agg"])
    return out
