"""Autotuner for the batched distance step: hoisting schedule and tile shapes.

The library exposes tile-shape knobs (`lc_set_tuning`) whose options all compute identical
results, and the rotate-and-sum schedule is a call argument (Section "Dynamic Hoisting": group
sizes g trade key memory for fewer ModUp/ModDown rounds).  `tune` times one workload shape on the
context's stream with CUDA events and keeps, by coordinate descent, the fastest schedule and then
the fastest option of each knob in turn, leaving the context set to the winner.  Candidate
schedules are those whose rotation keys are loaded in `evk` and whose key set fits
`key_budget_bytes`.  Results can be kept in a JSON cache file keyed by GPU model and workload
shape, so that a server tunes once per shape.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Dict, List, Optional, Sequence

import torch

from . import lancelot as LC


MAX_GROUP = 4  # the fused one-ModDown group kernel takes groups of up to 4 rotation bits (15 rotations)


def _partitions(b: int, m: int):
    """Non-increasing lists of positive integers <= m summing to b."""
    if b == 0:
        yield []
        return
    for p in range(min(b, m), 0, -1):
        for rest in _partitions(b - p, p):
            yield [p] + rest


def candidate_schedules(log_n: int, max_group: int = MAX_GROUP) -> Dict[str, List[int]]:
    """The unfoldings of the rotate-and-sum the search considers (Section "Dynamic Hoisting": how
    many rotation bits each hoisted group takes): "log", one rotation per group with a ModDown per
    rotation (log2(N/2) groups), and every composition of log2(N/2) into one-ModDown groups of at
    most `max_group` bits, largest first, with at most one single-bit group (two single-bit groups
    cost more than one group of two).  A group of g bits needs 2^g - 1 rotation keys.  The uniform
    ones keep short names: g2qp = groups of 2, g3qp = groups of 3 (the remainder last); the others
    are named by their group sizes, e.g. g4442qp."""
    b = log_n - 1
    out = {"log": [1] * b}
    for g in (2, 3):
        out[f"g{g}qp"] = [g] * (b // g) + ([b % g] if b % g else [])
    for parts in _partitions(b, max_group):
        if parts.count(1) > 1 or parts in out.values():
            continue
        out["g" + "".join(map(str, parts)) + "qp"] = parts
    return out


def schedule_keys(sched: Sequence[int]) -> int:
    """Rotation keys a schedule needs: 2^g - 1 per group."""
    return sum((1 << g) - 1 for g in sched)


def schedule_mode(name: str) -> int:
    return LC.LC_MODE_BATCHED | (LC.LC_HOIST_QP_SUM if name.endswith("qp") else 0)


def key_bytes(ctx: "LC.Context", n_keys: int) -> int:
    """Device bytes of n switching keys at the top level: dnum x 2 x (L+1+K) limbs of N words."""
    return n_keys * ctx.dnum * 2 * (ctx.nq + ctx.np_) * ctx.N * 8


def _time_ms(ctx: "LC.Context", fn, reps: int) -> float:
    fn()  # warm: scratch sized, kernels loaded
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record(ctx.stream)
    for k in range(reps):
        fn()
        ev[k + 1].record(ctx.stream)
    torch.cuda.synchronize()
    return statistics.median(ev[k].elapsed_time(ev[k + 1]) for k in range(reps))


def cache_key(ctx: "LC.Context", n: int, chunks: int, candidates: Sequence[str], device: Optional[str] = None) -> str:
    """Key of one tuned workload shape: the GPU model, the ring degree, clients, chunks and the
    candidate schedules considered."""
    if device is None:
        device = torch.cuda.get_device_name(getattr(ctx, "device", 0)) if torch.cuda.is_available() else "cpu"
    return f"{device}|log_n={ctx.log_n}|n={n}|chunks={chunks}|schedules={','.join(sorted(candidates))}"


def tune(ctx: "LC.Context", evk: "LC.EvalKeys", cts: torch.Tensor, n: int, chunks: int, scale: float,
         reps: int = 3, schedules: Optional[Dict[str, Sequence[int]]] = None,
         key_budget_bytes: Optional[float] = None, out: Optional[torch.Tensor] = None,
         cache_path: Optional[str] = None, device: Optional[str] = None) -> dict:
    """Returns {"schedule", "groups", "mode", "knobs", "ms", "trials", "schedules" (candidates
    timed), "key_bytes" (device bytes of the winner's relinearisation + rotation keys)}; the
    context keeps the chosen knob settings (the schedule is an argument of each distances call).

    cache_path: a JSON file of earlier results keyed by `cache_key`; a hit sets the cached knobs
    and returns the cached result (with "cached": True) without timing anything, a miss tunes and
    adds the result to the file."""
    have = set(evk.rotations)
    cands = {}
    for name, sched in (schedules or candidate_schedules(ctx.log_n)).items():
        rots = set(LC.rotations_of_schedule(sched))
        if not rots <= have:
            continue
        if key_budget_bytes is not None and key_bytes(ctx, len(rots) + 1) > key_budget_bytes:
            continue
        cands[name] = list(sched)
    if not cands:
        raise LC.LancelotError("autotune: no candidate schedule has all its rotation keys loaded")
    key = cache_key(ctx, n, chunks, list(cands), device) if cache_path else None
    if key:
        cache = _load_cache(cache_path)
        hit = cache.get(key)
        if hit and hit.get("schedule") in cands:
            names = {v: k for k, v in LC.TUNING_NAMES.items()}
            for name, v in hit["knobs"].items():
                if name in names and v in LC.TUNING_OPTIONS[names[name]]:
                    ctx.set_tuning(names[name], v)
            return dict(hit, groups=cands[hit["schedule"]], mode=schedule_mode(hit["schedule"]),
                        knobs=ctx.tuning(), cached=True)
    if out is None:
        out = ctx.empty(n * (n - 1) // 2, 2, ctx.L, ctx.N)
    trials = []

    def run(name):
        return lambda: ctx.distances(evk, cts, n, chunks, scale, mode=schedule_mode(name), groups=cands[name],
                                     out=out)

    best, best_ms = None, float("inf")
    for name in cands:
        ms = _time_ms(ctx, run(name), reps)
        trials.append({"schedule": name, "ms": ms})
        if ms < best_ms:
            best, best_ms = name, ms
    for knob, options in LC.TUNING_OPTIONS.items():
        times = {}
        for v in options:
            ctx.set_tuning(knob, v)
            times[v] = _time_ms(ctx, run(best), reps)
            trials.append({LC.TUNING_NAMES[knob]: v, "ms": times[v]})
        pick = min(times, key=times.get)
        ctx.set_tuning(knob, pick)
        best_ms = min(best_ms, times[pick])
    res = {"schedule": best, "groups": cands[best], "mode": schedule_mode(best), "knobs": ctx.tuning(),
           "ms": best_ms, "trials": trials, "schedules": len(cands),
           "key_bytes": key_bytes(ctx, len(set(LC.rotations_of_schedule(cands[best]))) + 1)}
    if key:
        cache = _load_cache(cache_path)
        cache[key] = {"schedule": best, "knobs": res["knobs"], "ms": best_ms, "trials": trials}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return res


def _load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}
