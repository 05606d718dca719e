#!/usr/bin/env python3
"""Benchmark of the Lancelot server evaluation on B300.

Metric: encrypted client-pair distances/s at N = 2^15, d = 2^20 (n = 10 clients, 64 ciphertexts
per client, 45 pairs).  One step = one pass of the whole hot path over one batch of synthetic
input: all 45 encrypted pair distances (sub, square, lazy relinearisation, rescale,
rotate-and-sum with 14 rotations) plus the masked aggregate over all 64 chunks.  Inputs are
generated on the device once (client ciphertexts: 4.8 GB, larger than L2) and stay resident.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode batched|perop] [--impl reference]

Under torchrun each rank runs an independent replica on its own GPU (weak scaling); rank 0 prints
one JSON line.  The reference arm (--impl reference) times the CPU oracle on the host cores on a
bounded sample per step (1 pair + 1 aggregate chunk), extrapolated to the same workload.

Other modes, one JSON line each (per rate / ring degree where stated):
  --workload batched   n = 50 clients, d = 2^22 (94 GB resident), 1,225 pairs + aggregate
  --workload uneven    8 jobs with their own key sets (147 GB resident) in shared launches
  --serving            Poisson round arrivals per rate, p50/p99 round latency
  --sweep              the same round at N = 2^13 .. 2^16
  --probes             register-resident integer-pipe probes (the ALU roofline's peak)
  --micro              small isolated kernel case for profiler captures (NVTX ranges)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth as S  # noqa: E402

METRIC = "encrypted client-pair distances/s (N=2^15, d=2^20); p50/p99 round latency"
UNIT = "pairs/s"
WORKLOAD = "plain_N32768_L14_K4_dnum4_n10_d2^20_64chunks_45pairs+masked_aggregate"


def plain_config(world: int) -> dict:
    """The workload as both arms name it (the run-specific details go to "run_detail")."""
    w = S.PLAIN
    return {"workload": WORKLOAD, "n_clients": w.n_clients, "d": w.d, "chunks": w.chunks, "pairs": w.n_pairs,
            "log_n": 15, "limbs_q": 15, "limbs_p": 4, "dnum": 4, "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (4.8 GB client ciphertexts resident)"}


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int) -> float:
    """The largest of the ranks' values (all_reduce MAX); the timing rule takes the slowest rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = f"cuda:{torch.cuda.current_device()}" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas: every rank processes units_per_rank per step, the
    job lasts as long as its slowest rank."""
    return world * units_per_rank * steps / seconds


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def run_batched(args):
    """The batched workload at full size: 50 clients x 256 chunks (94 GB of ciphertexts resident),
    1,225 pair distances + the masked aggregate of 256 chunks per step, autotuned schedule and
    tiles, eager launches (the library runs the pairs in waves).  Inputs are encrypted on the GPU
    with device randomness (the clients' batched step), which is outside the timed region."""
    import torch
    from paper_2408_06197_b300 import autotune, kgc
    from paper_2408_06197_b300 import lancelot as LC

    w = S.BATCHED
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    with torch.cuda.stream(stream):
        g = LC.Context.production(device=0, stream=stream)
        N = g.N
        s = S.secret_key(w.seed, w.config, N)
        pk = g.pk_gen(s, *S.pk_rand(w.seed, w.config, g.q, N))
        evk = g.evk()
        qp = g.q + g.p
        evk.add(s, None, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, None))
        rots = set()
        for nm in SCHEDULES:
            rots |= set(LC.rotations_of_schedule(SCHEDULES[nm]))
        for r in sorted(rots):
            evk.add(s, r, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, r))
        cts = g.empty(w.n_clients, w.chunks, 2, g.nq, N)
        flat = cts.view(w.n_clients * w.chunks, 2, g.nq, N)
        sq = np.zeros((w.n_clients, w.n_clients))
        Ws = []
        for i in range(w.n_clients):
            Wi = S.client_updates(w, [i])[0]
            Ws.append(Wi)
            z = torch.tensor(S.split_chunks(Wi, g.slots), device="cuda:0")
            g.encode_encrypt_seeded(pk, z, g.scale, w.seed, i * w.chunks, out=flat[i * w.chunks:(i + 1) * w.chunks])
        for i in range(w.n_clients):
            for j in range(i + 1, w.n_clients):
                sq[i, j] = sq[j, i] = float(np.sum((Ws[i] - Ws[j]) ** 2))
        del Ws
        sel = kgc.krum_select(sq, w.f, w.n_select)
        wts = torch.tensor(kgc.mask_weights(w.n_clients, sel, average=True), dtype=torch.float64, device="cuda:0")
        masks = g.encrypt_const_seeded(pk, wts, g.scale, w.seed, 1 << 40)
        out_d = g.empty(w.n_pairs, 2, g.L, N)
        out_a = g.empty(w.chunks, 2, g.L, N)
        t0 = time.perf_counter()
        # tune on a 10-client slice of the same ciphertexts (the tiles and schedule do not depend
        # on the client count; a full-size trial would take seconds each)
        sub = cts[:10].contiguous()
        tun = autotune.tune(g, evk, sub, 10, w.chunks, g.scale, schedules=dict(SCHEDULES))
        del sub
        tune_s = time.perf_counter() - t0
        mode = autotune.schedule_mode(tun["schedule"])

        def step():
            g.distances(evk, cts, w.n_clients, w.chunks, g.scale, mode=mode, groups=tun["groups"], out=out_d)
            g.masked_aggregate(evk, cts, w.n_clients, w.chunks, g.scale, masks, g.scale, out=out_a)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        run = step
        eager_ms = None
        if not args.no_graph:
            # every wave of both calls captured into one CUDA graph, replayed in the timed region;
            # the eager time of the same step is kept beside it
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            eager_ms = e0.elapsed_time(e1)
            graph = g.capture(step)
            graph.launch()
            g.sync()
            run = graph.launch
        clocks = Clocks(0)
        clocks.start()
        l0 = LC.launches()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        for k in range(args.steps):
            run()
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        launches = LC.launches() - l0
        ck = clocks.stop()
        step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
        ms = sum(step_ms) / args.steps
        # accuracy of the last step's read-outs against the FP64 distances (untimed)
        _, sc = g.distances(evk, cts, w.n_clients, w.chunks, g.scale, mode=mode, groups=tun["groups"], out=out_d)
        got = g.decrypt_const(s, out_d, g.L - 1, sc)
        ref = np.array([sq[i, j] for i in range(w.n_clients) for j in range(i + 1, w.n_clients)])
        rel = float(np.max(np.abs(got - ref) / ref))
        g.sync()
    line = {"metric": "encrypted client-pair distances/s (N=2^15, d=2^22, n=50)", "value": w.n_pairs / (ms / 1e3),
            "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (GPU encode + encryption with device randomness)",
            "config": {"workload": "batched_N32768_n50_d2^22_256chunks_1225pairs+masked_aggregate",
                       "n_clients": w.n_clients, "d": w.d, "chunks": w.chunks, "pairs": w.n_pairs,
                       "rotation_schedule": tun["schedule"], "tuning": tun["knobs"], "tune_seconds": tune_s,
                       "schedules_tried": tun.get("schedules"),
                       "launch": ("eager (pairs in waves inside the library)" if args.no_graph else
                                  "cuda_graph_replay (every wave of the step in one captured graph)"),
                       "l2": "inputs larger than L2 (94 GB client ciphertexts resident)"},
            "gpu_launches": launches, "eager_ms_per_step": eager_ms,
            "aggregate_chunks_per_s": w.chunks / (ms / 1e3), "clocks": ck, "max_rel_err_vs_fp64": rel,
            "round_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))}}
    print(json.dumps(line), flush=True)


def run_uneven(args):
    """The uneven batch at full size: 8 jobs (seed 2), each with its own key set (relinearisation +
    the rotation keys of the schedule: [4,4,3,3], 44 keys, unless --schedule names another), n in
    {5,10,20,40}, d in {2^16..2^22}
    (147 GB of ciphertexts resident), distances + masked aggregates of all jobs per step in
    shared launches (lc_batch_distances / lc_batch_aggregate: ragged pair and chunk lists packed
    into waves).  Beside it, the same jobs one after another through lc_distances /
    lc_masked_aggregate.  Inputs are encrypted on the GPU with device randomness (untimed)."""
    import torch
    from paper_2408_06197_b300 import kgc
    from paper_2408_06197_b300 import lancelot as LC

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    sname = REFERENCE_SCHEDULE if args.schedule == "auto" else args.schedule
    sched = SCHEDULES[sname]
    jobs_w = S.uneven_jobs()
    with torch.cuda.stream(stream):
        g = LC.Context.production(device=0, stream=stream)
        N, qp = g.N, g.q + g.p
        jobs, evks, keys_s = [], [], []
        for j, w in enumerate(jobs_w):
            s = S.secret_key(w.seed, w.config, N, job=j)
            pk = g.pk_gen(s, *S.pk_rand(w.seed, w.config, g.q, N, job=j))
            evk = g.evk()
            evk.add(s, None, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, None, job=j))
            for r in LC.rotations_of_schedule(sched):
                evk.add(s, r, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, r, job=j))
            cts = g.empty(w.n_clients, w.chunks, 2, g.nq, N)
            flat = cts.view(w.n_clients * w.chunks, 2, g.nq, N)
            W = np.stack([S.client_updates(w, [i])[0] for i in range(w.n_clients)])
            for i in range(w.n_clients):
                z = torch.tensor(S.split_chunks(W[i], g.slots), device="cuda:0")
                g.encode_encrypt_seeded(pk, z, g.scale, w.seed * 1000 + j, i * w.chunks,
                                        out=flat[i * w.chunks:(i + 1) * w.chunks])
            gram = W @ W.T
            sq = np.diag(gram)[:, None] + np.diag(gram)[None, :] - 2 * gram
            del W
            wts = kgc.mask_weights(w.n_clients, kgc.krum_select(sq, w.f, w.n_select), average=True)
            masks = g.encrypt_const_seeded(pk, torch.tensor(wts, dtype=torch.float64, device="cuda:0"), g.scale,
                                           w.seed * 1000 + j, 1 << 40)
            jobs.append(LC.Job(evk, cts, w.n_clients, w.chunks, masks))
            evks.append(evk)
            keys_s.append(s)
        torch.cuda.synchronize()
        qpf = LC.LC_HOIST_QP_SUM
        n_pairs = sum(w.n_pairs for w in jobs_w)
        pair_chunks = sum(w.n_pairs * w.chunks for w in jobs_w)

        def batched():
            LC.batch_distances(g, jobs, qpf, sched)
            LC.batch_aggregate(g, jobs)

        def alone():
            for jb in jobs:
                g.distances(jb.evk, jb.cts, jb.n, jb.chunks, g.scale, mode=LC.LC_MODE_BATCHED | qpf, groups=sched,
                            out=jb.out_dist)
                g.masked_aggregate(jb.evk, jb.cts, jb.n, jb.chunks, g.scale, jb.masks, g.scale, out=jb.out_agg)

        def timed(fn, steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
            ev[0].record(stream)
            for k in range(steps):
                fn()
                ev[k + 1].record(stream)
            torch.cuda.synchronize()
            return [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]

        # the same jobs split over two contexts on two streams, balanced by work, launched from two
        # host threads: the jobs of one stream fill the SMs the other leaves idle (tensor phases,
        # wave tails), so ragged jobs share the GPU instead of running one after another
        stream2 = torch.cuda.Stream(0)
        g2 = LC.Context.production(device=0, stream=stream2)
        for k in LC.TUNING_OPTIONS:
            g2.set_tuning(k, g.get_tuning(k))
        order = sorted(range(len(jobs)), key=lambda k: -(jobs_w[k].n_pairs * (jobs_w[k].chunks + 40)))
        groups2, load = [[], []], [0.0, 0.0]
        for k in order:
            t = 0 if load[0] <= load[1] else 1
            groups2[t].append(jobs[k])
            load[t] += jobs_w[k].n_pairs * (jobs_w[k].chunks + 40)

        def half(ctx, js, st):
            with torch.cuda.stream(st):
                if js:
                    LC.batch_distances(ctx, js, qpf, sched)
                    LC.batch_aggregate(ctx, js)

        def two_streams():
            import threading
            mark = torch.cuda.Event()
            mark.record(stream)
            stream2.wait_event(mark)
            th = threading.Thread(target=half, args=(g2, groups2[1], stream2))
            th.start()
            half(g, groups2[0], stream)
            th.join()
            done2 = torch.cuda.Event()
            done2.record(stream2)
            stream.wait_event(done2)

        for _ in range(args.warmup):
            batched()
        torch.cuda.synchronize()
        clocks = Clocks(0)
        clocks.start()
        step_ms = timed(batched, args.steps)
        ck = clocks.stop()
        two_streams()
        two_ms = timed(two_streams, max(1, args.steps))
        alone()
        alone_ms = timed(alone, max(1, args.steps))
        # accuracy of the batched read-outs against the FP64 distances of one small job (untimed)
        batched()
        j0 = min(range(len(jobs_w)), key=lambda k: jobs_w[k].n_clients * jobs_w[k].chunks)
        w0 = jobs_w[j0]
        W0 = np.stack([S.client_updates(w0, [i])[0] for i in range(w0.n_clients)])
        ref = np.array([np.sum((W0[a] - W0[b]) ** 2) for a in range(w0.n_clients) for b in range(a + 1, w0.n_clients)])
        got = g.decrypt_const(keys_s[j0], jobs[j0].out_dist, g.L - 1, g.scale * g.scale / g.q[g.L])
        rel = float(np.max(np.abs(got - ref) / ref))
        g.sync()
    ms = sum(step_ms) / len(step_ms)
    ams = sum(alone_ms) / len(alone_ms)
    tms = sum(two_ms) / len(two_ms)
    line = {"metric": "encrypted client-pair distances/s (uneven batch of 8 jobs, N=2^15)",
            "value": n_pairs / (ms / 1e3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic (GPU encode + encryption with device randomness)",
            "config": {"workload": "uneven_8jobs_seed2_n{5,10,20,40}_d{2^16..2^22}",
                       "jobs": [{"n": w.n_clients, "d": w.d, "chunks": w.chunks, "pairs": w.n_pairs} for w in jobs_w],
                       "pairs": n_pairs, "pair_chunks": pair_chunks, "rotation_schedule": sname,
                       "launch": "lc_batch_distances + lc_batch_aggregate (shared waves)",
                       "l2": "inputs larger than L2 (147 GB client ciphertexts resident)"},
            "pair_chunks_per_s": pair_chunks / (ms / 1e3), "clocks": ck,
            "jobs_one_after_another": {"ms_per_step": ams, "pairs_per_s": n_pairs / (ams / 1e3),
                                       "batched_over_alone": ams / ms},
            "two_streams": {"ms_per_step": tms, "pairs_per_s": n_pairs / (tms / 1e3), "over_alone": ams / tms,
                            "form": "jobs split by work over two contexts / streams, each running "
                                    "lc_batch_distances + lc_batch_aggregate on its share, overlapping"},
            "max_rel_err_vs_fp64": rel, "accuracy_job": j0,
            "round_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))}}
    print(json.dumps(line), flush=True)


def run_probes(args):
    """One JSON line: each probe at 4, 8 and 16 resident blocks of 256 threads per SM."""
    import torch
    from paper_2408_06197_b300 import lancelot as LC
    g = LC.Context.toy(device=0)
    out = {}
    for kind, name in ((LC.LC_PROBE_IMAD, "imad"), (LC.LC_PROBE_IMAD_WIDE, "imad_wide"),
                       (LC.LC_PROBE_NTT_BFLY, "ntt_butterfly")):
        iters = args.probe_iters if kind != LC.LC_PROBE_NTT_BFLY else max(1, args.probe_iters // 2)
        for bps in (4, 8, 16):
            r = g.alu_probe(kind, iters, bps)
            out[f"{name}_x{bps}"] = {"ms": r["ms"], "T_ops_per_s": r["ops_per_s"] / 1e12}
    g.sync()
    torch.cuda.synchronize()
    print(json.dumps({"probes": out, "unit": "T operations/s (butterflies for ntt_butterfly)"}), flush=True)


# Integer-pipe roofline.  The transforms are bound by 64-bit modular arithmetic emulated on the
# 32-bit integer pipes, not by DRAM.  Their ceiling is measured the way the copy bandwidth and the
# GEMM rate are: the library's register-resident probe runs the very butterfly of the transforms
# (lazy Shoup Cooley-Tukey, twiddles in registers, no memory traffic) on every SM, live in the same
# run at the same clock.  The IMAD probe checks the unit count behind it: 148 SMs x 64 32-bit
# multiply-adds per clock x 2.03 GHz = 19.2 T/s nominal, 19.2 T/s measured on a B300.
BFLY_INSTR = 17.78  # thread instructions per lazy butterfly of the register-resident probe (ncu)
# The fewest thread instructions a lazy Shoup Cooley-Tukey butterfly on 64-bit words can take on
# 32-bit integer pipes, counted from its partial products, in the form the transforms use for the
# primes below 2^46 (a quotient that may fall up to two short, products in [0, 4q)):
#   quotient t ~ y * w' / 2^64   1 wide + 2 high-half products + 2 carry additions          5
#   low 64 bits of y * w         1 wide + 2 32-bit multiply-adds into the high word         3
#   low 64 bits of t * q         the same                                                     3
#   r = y w - t q                64-bit subtraction (low with borrow, high)                  2
#   x + r, x + 4q - r            two 64-bit additions (three-input adds with carry)          4
# = 17 (19 with the exact quotient's four partial products, which the 60-bit primes keep).  The
# issue bound of the SM (148 SMs x 4 schedulers x 32 lanes, one instruction per clock) divided by
# it is the nominal integer roofline of the transforms.
BFLY_MIN_INSTR = 17


def alu_roofline(g, ntt_bytes: float, ntt_ms: float, sm_mhz):
    """NTT butterflies/s against the nominal integer-issue bound of the minimal butterfly, with the
    live register-resident probe of the library's own butterfly beside it."""
    probes = {}
    for kind, name, iters in ((0, "imad", 4096), (1, "imad_wide", 4096), (2, "ntt_butterfly", 2048)):
        r = g.alu_probe(kind, iters, 8)
        probes[name] = {"T_ops_per_s": r["ops_per_s"] / 1e12, "ms": r["ms"]}
    limbs = ntt_bytes / (16.0 * g.N)
    bfly = limbs * (g.N // 2) * g.log_n
    achieved = bfly / (ntt_ms / 1e3) / 1e12 if ntt_ms > 0 else 0.0
    peak = probes["ntt_butterfly"]["T_ops_per_s"]
    mhz = sm_mhz or 2032.0
    # the nominal view beside it: 148 SMs x 4 schedulers x 32 lanes issue one instruction per clock;
    # the lazy butterfly is BFLY_INSTR thread instructions (ncu count of the probe), so issue
    # alone would allow this many butterflies per second (the probe sustains ~0.58 of it: the mix
    # saturates the integer pipes first)
    issue_bfly = 148 * 4 * 32 * mhz * 1e6 / BFLY_INSTR / 1e12
    issue_min = 148 * 4 * 32 * mhz * 1e6 / BFLY_MIN_INSTR / 1e12
    return {"achieved": achieved, "peak": issue_min, "unit": "T butterflies/s", "frac": achieved / issue_min,
            "peak_source": f"nominal integer issue bound: 148 SMs x 4 x 32 lanes x {mhz:.0f} MHz / "
                           f"{BFLY_MIN_INSTR} instructions per butterfly (the minimal count from its partial "
                           f"products)",
            "butterflies": bfly, "imad_nominal_T_per_s": 148 * 64 * mhz * 1e6 / 1e12, "sm_mhz": mhz,
            "probe_T_butterflies_per_s": peak, "frac_of_probe": achieved / peak,
            "probe_instructions_per_butterfly": BFLY_INSTR,
            "issue_bound_at_probe_count_T_per_s": issue_bfly, "frac_of_issue_bound_at_probe_count": achieved / issue_bfly,
            "probes": probes}


# ----------------------------------------------------------------------------- clocks sampler
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- workload (GPU)
def _schedules():
    from paper_2408_06197_b300.autotune import candidate_schedules
    return candidate_schedules(15)


# the hoisting schedules at N = 2^15: "log" (14 single rotations), g2qp ([2]*7), g3qp
# ([3,3,3,3,2]) and every other composition of 14 into one-ModDown groups of at most 4 bits
SCHEDULES = _schedules()
# the schedule the autotuner picks for the benchmark workload on a B300 (every run so far); the
# reference arm, which cannot time GPU candidates, runs the oracle with it
REFERENCE_SCHEDULE = "g4433qp"

# DRAM bytes per limb of one transform (column + row pass, N = 2^15), from the ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the 960-limb case of `bench.py --micro`:
# forward 457.0 + 454.4 MB, inverse 453.0 + 444.9 MB per 960 limbs (column cap 8, row cap 5).
# Valid for the current transform kernels only.
NTT_DRAM_BYTES_PER_LIMB = (457.0e6 + 454.4e6 + 453.0e6 + 444.9e6) / (2 * 960)
# SM throughput (% of peak) of the key-switch kernel classes in their ncu captures (k_inner_gather
# 68-79 %, k_modup 81 %, k_moddown_bconv 82 %).  Static: ncu does not run inside the benchmark.
KS_SM_PCT = {"inner": "68-79", "modup": "81", "moddown": "82"}


def build_workload(LC, g, w: S.Workload, sched_name: str = "auto"):
    N = g.N
    # keys of the schedule (every candidate schedule for "auto") plus the 14 log-step keys of the
    # plain form
    names = sorted(SCHEDULES) if sched_name == "auto" else [sched_name]
    rots = set(LC.rotations_of_schedule([1] * (g.log_n - 1)))
    for nm in names:
        rots |= set(LC.rotations_of_schedule(SCHEDULES[nm]))
    rots = sorted(rots)
    sched = SCHEDULES["g3qp" if sched_name == "auto" else sched_name]
    s = S.secret_key(w.seed, w.config, N)
    pa, pe = S.pk_rand(w.seed, w.config, g.q, N)
    pk = g.pk_gen(s, pa, pe)
    evk = g.evk()
    qp = g.q + g.p
    evk.add(s, None, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, None))
    for r in rots:
        evk.add(s, r, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, r))
    W = S.client_updates(w)
    X = S.split_chunks(W, g.slots)
    cts = g.empty(w.n_clients, w.chunks, 2, g.nq, N)
    flat = cts.view(w.n_clients * w.chunks, 2, g.nq, N)
    for i in range(w.n_clients):
        m = np.stack([g.encode(X[i, k], g.scale) for k in range(w.chunks)])
        r, e0, e1 = S.enc_rand_batch(w.seed, w.config, [i], range(w.chunks), N)
        g.encrypt(pk, m, r, e0, e1, out=flat[i * w.chunks:(i + 1) * w.chunks])
    # KGC side (plaintext, untimed): Multi-Krum on the FP64 distances of the synthetic updates
    from paper_2408_06197_b300 import kgc
    d = np.array([[np.sum((W[i] - W[j]) ** 2) for j in range(w.n_clients)] for i in range(w.n_clients)])
    sel = kgc.krum_select(d, w.f, w.n_select)
    wts = kgc.mask_weights(w.n_clients, sel, average=True)
    mm = np.stack([g.encode(np.full(g.slots, wts[i]), g.scale) for i in range(w.n_clients)])
    r, e0, e1 = S.enc_rand_batch(w.seed, w.config, range(w.n_clients), [S.MASK_CHUNK], N)
    masks = g.encrypt(pk, mm, r, e0, e1)
    return evk, cts, masks, sched, s, pk


# ----------------------------------------------------------------------------- CPU oracle sample
def oracle_sample(w: S.Workload, reps: int = 1, sched_name: str = "g3qp"):
    """Times the oracle (as it stands) on 1 pair of distances + 1 aggregate chunk, `reps` times,
    with the rotation schedule the GPU line runs (one-ModDown groups for the "qp" schedules).
    Returns (pairs/s extrapolated to the workload, per-rep seconds, threads, step seconds)."""
    import oracle as O
    prm = O.params_production()
    o = O.Context(prm)
    threads = O.set_threads(0)
    N = prm.N
    sched = SCHEDULES[sched_name]
    qp_sum = sched_name.endswith("qp")
    s = S.secret_key(w.seed, w.config, N)
    pk = o.pk_gen(s, *S.pk_rand(w.seed, w.config, prm.q, N))
    qp = prm.q + prm.p
    rlk = o.swk_gen(s, 0, *S.swk_rand(w.seed, w.config, qp, prm.dnum, N, None))
    rk = {r: o.swk_gen(s, o.galois(r), *S.swk_rand(w.seed, w.config, qp, prm.dnum, N, r))
          for r in O.rotations_of_schedule(sched)}
    W = S.client_updates(w)
    X = S.split_chunks(W, prm.slots)
    # pair sample: clients 0 and 1, all chunks; aggregate sample: chunk 0 of every client
    cts = np.zeros((2, w.chunks, 2, prm.L + 1, N), dtype=np.uint64)
    agg_in = np.zeros((w.n_clients, 1, 2, prm.L + 1, N), dtype=np.uint64)
    for i in range(w.n_clients):
        ks = range(w.chunks) if i < 2 else [0]
        r, e0, e1 = S.enc_rand_batch(w.seed, w.config, [i], ks, N)
        for t, k in enumerate(ks):
            ct = o.encrypt(pk, o.encode(X[i, k], prm.scale), r[t], e0[t], e1[t])
            if i < 2:
                cts[i, k] = ct
            if k == 0:
                agg_in[i, 0] = ct
    masks = np.ascontiguousarray(agg_in[:, 0])
    per = []
    t_pair = t_chunk = 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        o.distances(cts, rlk, sched, rk, qp_sum=qp_sum)
        t1 = time.perf_counter()
        o.masked_aggregate(agg_in, masks, rlk)
        t2 = time.perf_counter()
        t_pair, t_chunk = t1 - t0, t2 - t1
        per.append((t_pair, t_chunk))
    t_pair = min(p[0] for p in per)
    t_chunk = min(p[1] for p in per)
    step = w.n_pairs * t_pair + w.chunks * t_chunk
    return w.n_pairs / step, per, threads, step


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores.  Each step is a bounded
    sample of the workload -- the encrypted distance of one pair (64 chunks, the one-ModDown
    schedule the benchmark's autotuner picks on a B300, [4,4,3,3], unless --schedule names
    another) and the masked aggregate of one chunk -- and ms_per_step is that sample's measured
    time; the throughput is the workload's (45 pairs + 64 chunks per step) at the sample's
    per-pair and per-chunk times."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    w = S.PLAIN
    total = args.warmup + args.steps
    sname = REFERENCE_SCHEDULE if args.schedule == "auto" else args.schedule
    groups = SCHEDULES[sname]
    _, per, threads, _ = oracle_sample(w, reps=total, sched_name=sname)
    timed = per[args.warmup:]
    t_pair = statistics.median(p[0] for p in timed)
    t_chunk = statistics.median(p[1] for p in timed)
    full_step = w.n_pairs * t_pair + w.chunks * t_chunk
    value = w.n_pairs / full_step
    sample_ms = statistics.mean(p[0] + p[1] for p in timed) * 1e3
    sample = (f"per step: oracle distances of 1 pair (64 chunks, rotation schedule {sname} = one-ModDown groups "
              f"{groups}, {sum((1 << gb) - 1 for gb in groups)} rotation keys) and masked aggregate of 1 chunk "
              f"({sample_ms:.0f} ms measured); "
              f"throughput at the workload's 45 pairs + 64 chunks per step (median pair {t_pair:.2f} s, chunk "
              f"{t_chunk:.2f} s -> {full_step:.1f} s per full step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sample_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": plain_config(world),
            "run_detail": {"rotation_schedule": sname, "sample_units_per_step": "1 pair + 1 aggregate chunk",
                           "full_step_s": full_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- kernel micro case
def run_micro(args):
    """Small isolated case for profiler captures (about 4 GB on the device, inputs larger than
    L2): batched distances of 10 clients x C chunks (C = --micro-chunks, default 8; 45 pairs,
    rotation schedule --schedule) and their masked aggregate (C chunks), 960 limbs transformed forward and
    back, 16 degree-2 triples relinearised and rescaled at level 14, and 16 ciphertexts rotated
    at level 13.  Prints per-class timings."""
    import torch
    from paper_2408_06197_b300 import lancelot as LC
    w = S.PLAIN
    g = LC.Context.production()
    N = g.N
    s = S.secret_key(w.seed, w.config, N)
    evk = g.evk()
    qp = g.q + g.p
    evk.add(s, None, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, None))
    evk.add(s, 1, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, 1))
    B = 16
    gen = torch.Generator(device="cuda").manual_seed(7)
    ct3 = torch.randint(0, 1 << 40, (B, 3, g.nq, N), device="cuda", generator=gen)
    cts = torch.randint(0, 1 << 40, (B, 2, g.L, N), device="cuda", generator=gen)
    xl = torch.randint(0, 1 << 40, (64, g.nq, N), device="cuda", generator=gen)
    # batched distances over 10 clients x C chunks of random residues (45 pairs, 75 MB per chunk),
    # rotate-and-sum in one-ModDown groups of the chosen schedule
    sname = "g3qp" if args.schedule == "auto" else args.schedule
    sched = SCHEDULES[sname]
    qpf = LC.LC_HOIST_QP_SUM if sname.endswith("qp") else 0
    for r in LC.rotations_of_schedule(sched):
        if r != 1:
            evk.add(s, r, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, r))
    rng = np.random.default_rng(5)
    C = args.micro_chunks
    dc = np.empty((10, C, 2, g.nq, N), dtype=np.uint64)
    for i, q in enumerate(g.q):
        dc[:, :, :, i] = rng.integers(0, q, size=(10, C, 2, N), dtype=np.uint64)
    dcts = LC.u64_to_torch(dc)
    dm = np.empty((10, 2, g.nq, N), dtype=np.uint64)
    for i, q in enumerate(g.q):
        dm[:, :, i] = rng.integers(0, q, size=(10, 2, N), dtype=np.uint64)
    dmasks = LC.u64_to_torch(dm)
    del dc, dm
    dout = g.empty(45, 2, g.L, N)
    aout = g.empty(C, 2, g.L, N)
    nvtx = torch.cuda.nvtx
    for it in range(args.warmup + args.steps):
        if it == args.warmup:
            g.profile_start()
        # NVTX ranges name the phases for profiler filters (ncu --nvtx --nvtx-include "ntt/")
        nvtx.range_push("distances")
        g.distances(evk, dcts, 10, C, g.scale, mode=LC.LC_MODE_BATCHED | qpf, groups=sched, out=dout)
        nvtx.range_pop()
        nvtx.range_push("aggregate")
        g.masked_aggregate(evk, dcts, 10, C, g.scale, dmasks, g.scale, out=aout)
        nvtx.range_pop()
        nvtx.range_push("ntt")  # 960 limbs forward then inverse, in place
        g.to_eval(xl, g.L, inplace=True)
        g.to_coeff(xl, g.L, inplace=True)
        nvtx.range_pop()
        nvtx.range_push("relin_rescale")
        r2 = g.relin(evk, ct3, g.L)
        g.rescale(r2, g.L)
        nvtx.range_pop()
        nvtx.range_push("rotate")
        for b in range(B):
            g.rotate(evk, cts[b], g.L - 1, [1])
        nvtx.range_pop()
    prof = g.profile_stop()
    print(json.dumps({"micro": {k: {"ms_per_iter": v["ms"] / args.steps, "GBps": v["bytes"] / v["ms"] / 1e6
                                    if v["ms"] else 0.0, "launches_per_iter": v["launches"] / args.steps}
                                for k, v in prof.items()}}), flush=True)


# ----------------------------------------------------------------------------- packing-size sweep
def run_sweep(args):
    """Packing-size sweep (the paper's cryptographic-hyperparameter analysis): the same round
    (n = 10 clients, d = 2^20, 45 distances + masked aggregate) at N = 2^13 .. 2^16 with the
    production modulus chain at each N; chunks = d / (N/2) shrink as N grows.  One JSON line per N
    (device time per round, CUDA events, autotuned schedule and tiles)."""
    import torch
    from paper_2408_06197_b300 import autotune
    from paper_2408_06197_b300 import lancelot as LC
    rank, world, local = dist_info()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(local)
    for log_n in [int(x) for x in args.sweep_log_n.split(",")]:
        with torch.cuda.stream(stream):
            g = LC.Context.production(log_n, device=local, stream=stream)
            w = S.Workload(f"sweep_N2^{log_n}_n10_d2^20", S.CFG_PLAIN, log_n, 10, 1 << 20, 0, (8, 9), "flip5", 6, 2)
            N = g.N
            cands = autotune.candidate_schedules(log_n)
            rots = set()
            for sc in cands.values():
                rots |= set(LC.rotations_of_schedule(sc))
            s = S.secret_key(w.seed, w.config, N)
            pk = g.pk_gen(s, *S.pk_rand(w.seed, w.config, g.q, N))
            evk = g.evk()
            qp = g.q + g.p
            evk.add(s, None, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, None))
            for r in sorted(rots):
                evk.add(s, r, *S.swk_rand(w.seed, w.config, qp, g.dnum, N, r))
            X = S.split_chunks(S.client_updates(w), g.slots)
            cts = g.empty(w.n_clients, w.chunks, 2, g.nq, N)
            flat = cts.view(-1, 2, g.nq, N)
            for i in range(w.n_clients):
                m = np.stack([g.encode(X[i, k], g.scale) for k in range(w.chunks)])
                r, e0, e1 = S.enc_rand_batch(w.seed, w.config, [i], range(w.chunks), N)
                g.encrypt(pk, m, r, e0, e1, out=flat[i * w.chunks:(i + 1) * w.chunks])
            mm = np.zeros((w.n_clients, N), dtype=np.int64)
            mm[:, 0] = int(round(g.scale / w.n_select))
            r, e0, e1 = S.enc_rand_batch(w.seed, w.config, range(w.n_clients), [S.MASK_CHUNK], N)
            masks = g.encrypt(pk, mm, r, e0, e1)
            out_d = g.empty(w.n_pairs, 2, g.L, N)
            out_a = g.empty(w.chunks, 2, g.L, N)
            tun = autotune.tune(g, evk, cts, w.n_clients, w.chunks, g.scale, schedules=cands, out=out_d)

            def step():
                g.distances(evk, cts, w.n_clients, w.chunks, g.scale, mode=tun["mode"], groups=tun["groups"],
                            out=out_d)
                g.masked_aggregate(evk, cts, w.n_clients, w.chunks, g.scale, masks, g.scale, out=out_a)

            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for _ in range(args.steps):
                step()
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1]) / args.steps
            print(json.dumps({"metric": "round time vs packing size (45 distances + masked aggregate)",
                              "impl": "ours", "log_n": log_n, "slots": g.slots, "chunks": w.chunks,
                              "ms_per_round": ms, "pairs_per_s": w.n_pairs / (ms / 1e3),
                              "rotation_schedule": tun["schedule"], "tuning": tun["knobs"], "dtype": "u64",
                              "data": "synthetic", "config": {"workload": w.name, "limbs_q": 15, "limbs_p": 4,
                                                              "dnum": 4}}), flush=True)
            del g, evk, cts, masks, out_d, out_a
            torch.cuda.empty_cache()


# ----------------------------------------------------------------------------- serving
def build_serving(LC, g, tenants: int, sched, seed: int = 3, honest: int = 48, byz: int = 16):
    """Tenants with resident keys (relin + the rotation keys of the schedule) and, per
    tenant, a device pool of encrypted update chunks (`honest` draws of N(0, 0.01^2) per slot and
    `byz` draws scaled by 5) from which arriving rounds are assembled."""
    import torch
    from paper_2408_06197_b300 import serving as SV
    N, slots = g.N, g.slots
    qp = g.q + g.p
    out = []
    for t in range(tenants):
        s = S.secret_key(seed, S.CFG_SERVING, N, job=t)
        pa, pe = S.pk_rand(seed, S.CFG_SERVING, g.q, N, job=t)
        pk = g.pk_gen(s, pa, pe)
        evk = g.evk()
        evk.add(s, None, *S.swk_rand(seed, S.CFG_SERVING, qp, g.dnum, N, None, job=t))
        for r in LC.rotations_of_schedule(sched):
            evk.add(s, r, *S.swk_rand(seed, S.CFG_SERVING, qp, g.dnum, N, r, job=t))
        vals = [S.rng(seed, S.CFG_SERVING, t, i, 0, S.P_UPDATE).normal(0.0, 0.01, slots) for i in range(honest + byz)]
        vals = [v * (5.0 if i >= honest else 1.0) for i, v in enumerate(vals)]
        m = np.stack([g.encode(v, g.scale) for v in vals])
        r, e0, e1 = S.enc_rand_batch(seed, S.CFG_SERVING, range(honest + byz), [0], N, job=t)
        pool = g.encrypt(pk, m, r, e0, e1)
        out.append((SV.Tenant(evk, pk, s), pool))
    return out


class ServingSetup:
    """Tenants, device pools and lanes of the serving runs (see build_serving)."""

    def __init__(self, args, g, local, sched, flags, honest=48, byz=16):
        import torch
        from paper_2408_06197_b300 import lancelot as LC
        from paper_2408_06197_b300 import serving as SV
        self.g, self.sched, self.flags = g, sched, flags
        self.honest, self.byz = honest, byz
        self.args = args
        ten = build_serving(LC, g, args.tenants, sched, honest=honest, byz=byz)
        self.tenants = [t for t, _ in ten]
        self.pools = [p for _, p in ten]
        self.device_kgc = not args.host_kgc
        if self.device_kgc and args.lanes == 2:
            # small rounds on a high-priority stream, large ones on a low-priority stream; each lane
            # has its own context (scratch); the tenants' keys are shared
            hi = torch.cuda.Stream(local, priority=-1)
            lo = torch.cuda.Stream(local, priority=0)
            self.lanes = [SV.Lane(LC.Context.production(device=local, stream=hi), args.fast_pairs, "fast"),
                          SV.Lane(LC.Context.production(device=local, stream=lo), None, "bulk")]
            for lane in self.lanes:  # the same tile shapes as the tuned main context
                for k in LC.TUNING_OPTIONS:
                    lane.ctx.set_tuning(k, g.get_tuning(k))
        else:
            self.lanes = None

    def ingest(self, r):
        """Round r's client chunks, assembled on the device from its tenant's pool (honest
        clients from the honest draws, the last n/5 clients from the x5 draws)."""
        import torch
        g = self.g
        pick = S.rng(3, S.CFG_SERVING, r.rid, 0, 0, S.P_JOB)
        idx = pick.integers(0, self.honest, size=(r.n, r.chunks))
        nb = r.n // 5
        if nb:
            idx[r.n - nb:] = self.honest + pick.integers(0, self.byz, size=(nb, r.chunks))
        pool = self.pools[r.tenant]
        it = torch.from_numpy(idx.reshape(-1)).to(pool.device, non_blocking=True)
        return pool.index_select(0, it).view(r.n, r.chunks, 2, g.nq, g.N)

    def mask_rand(self, r, i):
        return S.enc_rand(3, S.CFG_SERVING, i, S.MASK_CHUNK, self.g.N, job=r.rid)

    def rounds_of(self, stream_rounds):
        from paper_2408_06197_b300 import serving as SV
        out = []
        for x in stream_rounds:
            nb = x.n_clients // 5
            out.append(SV.Round(x.rid, x.tenant, x.n_clients, max(1, -(-x.d // self.g.slots)), x.arrival, f=nb,
                                n_select=max(1, x.n_clients - 2 * nb - 3), average=True))
        return out

    def server(self):
        from paper_2408_06197_b300 import serving as SV
        a = self.args
        return SV.Server(self.g, self.tenants, a.budget_gb * 1e9, self.ingest, self.mask_rand, groups=self.sched,
                         flags=self.flags, device_kgc_seed=3 if self.device_kgc else None, lanes=self.lanes)

    def warm(self, n_rounds):
        import torch
        warm = self.rounds_of(S.serving_rounds(seed=4, n_rounds=n_rounds, rate=1e9, tenants=self.args.tenants))
        self.server().run(warm, realtime=False)
        torch.cuda.synchronize()

    def run_rate(self, rate, n_rounds, local):
        """One Poisson stream of n_rounds rounds at `rate` rounds/s; its summary (one JSON object)."""
        import torch
        from paper_2408_06197_b300 import lancelot as LC
        from paper_2408_06197_b300 import serving as SV
        rounds = self.rounds_of(S.serving_rounds(seed=3, n_rounds=n_rounds, rate=rate, tenants=self.args.tenants))
        srv = self.server()
        clocks = Clocks(local)
        clocks.start()
        l0 = LC.launches()
        t0 = time.perf_counter()
        done = srv.run(rounds, realtime=True)
        span = time.perf_counter() - t0
        torch.cuda.synchronize()
        ck = clocks.stop()
        summ = SV.latency_summary(done)
        lat = sorted(r.latency * 1e3 for r in done)
        return {"rate_per_s": rate, "rounds": summ["rounds"], "p50_ms": summ["p50_ms"], "p99_ms": summ["p99_ms"],
                "p99_over_p50": summ["p99_ms"] / summ["p50_ms"] if summ["p50_ms"] else None,
                "max_ms": lat[-1] if lat else None, "kgc_p50_ms": summ["kgc_p50_ms"],
                "pairs_per_s": summ["pairs"] / span, "rounds_per_s": len(done) / span,
                "mean_rounds_per_batch": srv.stats["rounds_batched"] / max(1, srv.stats["distance_batches"]),
                "max_resident_gb": srv.stats["max_used"] / 1e9, "gpu_launches": LC.launches() - l0,
                "lanes": ([{"name": ln.name, "max_pairs": ln.max_pairs, "batches": ln.batches} for ln in srv.lanes]
                          if self.device_kgc else "ticks (host KGC)"),
                "clocks": ck}


def serving_leg(args, g, stream, local, sched, flags):
    """The default run's serving leg: a bounded Poisson stream (args.serving_rounds rounds at
    args.serving_rate rounds/s, seed 3, sizes of the uneven workload, 4 tenants with resident keys,
    KGC step on the device) through the serving loop; p50/p99 of arrival -> aggregate ready."""
    import torch
    with torch.cuda.stream(stream):
        st = ServingSetup(args, g, local, sched, flags)
        st.warm(6)
        out = st.run_rate(args.serving_rate, args.serving_rounds, local)
    out.update({"definition": "round latency = arrival -> masked aggregate ready (distances, KGC read-out + "
                              "Multi-Krum + mask encryption on the device, aggregate); rounds of the uneven "
                              "workload's sizes (n in {5,10,20,40}, d in {2^16..2^22}), Poisson arrivals",
                "tenants": args.tenants, "budget_gb": args.budget_gb, "seed": 3})
    del st
    torch.cuda.synchronize()
    return out


def run_serving(args):
    """Poisson round stream over 4 tenants (sizes of the uneven-batch workload: n in {5,10,20,40},
    d in {2^16..2^22}), HBM admission budget, continuous batching, KGC step on the device (or on
    the host with --host-kgc).  One JSON line per arrival rate."""
    import torch
    from paper_2408_06197_b300 import lancelot as LC
    rank, world, local = dist_info()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(local)
    with torch.cuda.stream(stream):
        g = LC.Context.production(device=local, stream=stream)
        sname = REFERENCE_SCHEDULE if args.schedule == "auto" else args.schedule
        sched = SCHEDULES[sname]
        flags = LC.LC_HOIST_QP_SUM if sname.endswith("qp") else 0
        st = ServingSetup(args, g, local, sched, flags)
        st.warm(args.warmup)
        for rate in [float(x) for x in args.rates.split(",")]:
            r = st.run_rate(rate, args.rounds, local)
            line = {"metric": "served aggregation rounds: round latency (arrival -> aggregate ready)",
                    "impl": "ours", **r, "dtype": "u64", "data": "synthetic",
                    "config": {"workload": "serving_N32768_4tenants_n{5,10,20,40}_d{2^16..2^22}_poisson",
                               "tenants": args.tenants, "budget_gb": args.budget_gb,
                               "rotation_schedule": sname, "seed": 3,
                               "kgc": "host" if args.host_kgc else "device",
                               "lanes": args.lanes if not args.host_kgc else 1}}
            print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- main arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--mode", choices=["batched", "perop"], default="batched")
    ap.add_argument("--schedule", choices=sorted(SCHEDULES) + ["auto"], default="auto",
                    help="rotate-and-sum hoisting: log = 14 single rotations; g2qp = 7 groups of 3 rotations "
                         "with one ModDown per group (21 rotation keys); g3qp = 4 groups of 7 + 1 of 3 (31 keys); "
                         "auto = the autotuner picks among them (and the kernel tile shapes)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile shapes")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the per-operation reference measurement")
    ap.add_argument("--no-client", action="store_true", help="skip the client-side encode+encrypt measurement")
    ap.add_argument("--no-graph", action="store_true", help="launch kernels eagerly instead of replaying a CUDA graph")
    ap.add_argument("--micro", action="store_true", help="small isolated kernel case for profiler captures")
    ap.add_argument("--micro-chunks", type=int, default=8, help="chunks per client in the --micro distances")
    ap.add_argument("--serving", action="store_true", help="Poisson-arrival serving loop; one line per rate")
    ap.add_argument("--rates", default="1,2,5", help="serving arrival rates (rounds/s), comma separated")
    ap.add_argument("--rounds", type=int, default=100, help="serving rounds per rate")
    ap.add_argument("--tenants", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serving HBM admission budget")
    ap.add_argument("--host-kgc", action="store_true",
                    help="serving: KGC step on the host (default: on the device, no host round trip)")
    ap.add_argument("--workload", choices=["plain", "batched", "uneven"], default="plain",
                    help="batched = n=50 clients, d=2^22 (256 ciphertexts each, 94 GB resident), 1,225 pairs; "
                         "uneven = 8 jobs with their own keys, n in {5..40}, d in {2^16..2^22} (147 GB "
                         "resident), in shared launches; one JSON line beside the headline workload")
    ap.add_argument("--probes", action="store_true",
                    help="integer-pipe probes only (register-resident IMAD, wide IMAD, NTT butterfly)")
    ap.add_argument("--probe-iters", type=int, default=4096)
    ap.add_argument("--no-serving", action="store_true", help="skip the served-rounds leg of the default run")
    ap.add_argument("--serving-rounds", type=int, default=100, help="rounds of the default run's serving leg")
    ap.add_argument("--serving-rate", type=float, default=2.0, help="arrival rate of the default run's serving leg")
    ap.add_argument("--lanes", type=int, default=2, choices=[1, 2],
                    help="serving: 2 = small rounds on a high-priority stream, large ones on a low-priority "
                         "stream (device KGC only); 1 = one stream")
    ap.add_argument("--fast-pairs", type=int, default=190,
                    help="serving with 2 lanes: rounds of at most this many pairs take the high-priority lane")
    ap.add_argument("--sweep", action="store_true", help="packing-size sweep; one line per N")
    ap.add_argument("--sweep-log-n", default="13,14,15,16")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.micro:
        run_micro(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.probes:
        run_probes(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "uneven":
        os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")
        run_uneven(args)
        return
    if args.serving:
        # rounds of 0.1-75 GiB come and go: let the caching allocator grow segments instead of
        # fragmenting the device into blocks too small for the next large round
        os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")
        run_serving(args)
        return

    import torch
    from paper_2408_06197_b300 import lancelot as LC

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(local)
    w = S.PLAIN
    with torch.cuda.stream(stream):
        g = LC.Context.production(device=local, stream=stream)
        evk, cts, masks, sched, s, evk_pk = build_workload(LC, g, w, args.schedule)
        mode = LC.LC_MODE_BATCHED if args.mode == "batched" else LC.LC_MODE_PER_OP
        out_d = g.empty(w.n_pairs, 2, g.L, g.N)
        out_a = g.empty(w.chunks, 2, g.L, g.N)
        sched_name = "g3qp" if args.schedule == "auto" else args.schedule
        tuning = None
        if args.mode == "batched" and not args.no_autotune:
            from paper_2408_06197_b300 import autotune
            t0 = time.perf_counter()
            cand = dict(SCHEDULES) if args.schedule == "auto" else {args.schedule: SCHEDULES[args.schedule]}
            tuning = autotune.tune(g, evk, cts, w.n_clients, w.chunks, g.scale, schedules=cand, out=out_d)
            tuning["seconds"] = time.perf_counter() - t0
            sched_name, sched = tuning["schedule"], tuning["groups"]
        dmode = mode | (LC.LC_HOIST_QP_SUM if sched_name.endswith("qp") else 0)

        def step():
            g.distances(evk, cts, w.n_clients, w.chunks, g.scale, mode=dmode, groups=sched, out=out_d)
            g.masked_aggregate(evk, cts, w.n_clients, w.chunks, g.scale, masks, g.scale, mode=mode, out=out_a)

        def plain_step():  # the plain per-operation form: one pair / chunk per launch sequence, 14 keys
            g.distances(evk, cts, w.n_clients, w.chunks, g.scale, mode=LC.LC_MODE_PER_OP, out=out_d)
            g.masked_aggregate(evk, cts, w.n_clients, w.chunks, g.scale, masks, g.scale, mode=LC.LC_MODE_PER_OP,
                               out=out_a)

        def barrier():
            if world > 1:
                torch.distributed.barrier()

        for _ in range(args.warmup):
            step()
        g.sync()
        use_graph = args.mode == "batched" and not args.no_graph
        run = step
        if use_graph:  # one step captured into a CUDA graph, replayed in the timed region
            graph = g.capture(step)
            for _ in range(2):
                graph.launch()
            g.sync()
            run = graph.launch
        clocks = Clocks(local)
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        time.sleep(0.3)
        l0 = LC.launches()
        if not use_graph:
            g.profile_start()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev0, ev1 = evs[0], evs[-1]
        ev0.record(stream)
        for k in range(args.steps):
            run()
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
        step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
        launches = LC.launches() - l0
        if use_graph:
            # per-kernel-class timing needs eager launches: a second timed region of the same steps
            g.profile_start()
            for _ in range(args.steps):
                step()
            torch.cuda.synchronize()
        prof = g.profile_stop()
        barrier()
        ck = clocks.stop()
        ms = max_over_ranks(ev0.elapsed_time(ev1), world)
        ms_per_step = ms / args.steps
        value = whole_job_rate(w.n_pairs, world, args.steps, ms / 1e3)

        # end-to-end through the C ABI: every step copies its inputs in from pinned host memory and
        # its results out, in the wire form (lc_pack / lc_unpack: residues of 40-bit primes in 5
        # bytes, 78 instead of 120 bytes per coefficient at level 14), unpacked and packed on the
        # device inside the step.  Serial form: copy in, compute, copy out.  Pipelined form
        # (reported as e2e): double-buffered device buffers, the next step's inputs copied in and
        # the previous step's results copied out on the context's copy streams while this step
        # computes (lc_copy_async / lc_copy_wait).
        e2e = e2e_serial = None
        if not args.no_e2e:
            L = g.L
            nct, nmk = w.n_clients * w.chunks, w.n_clients
            wb_in, wb_out = g.wire_bytes(2, L), g.wire_bytes(2, L - 1)
            h_cts = LC.pinned_empty((nct, wb_in), np.uint8)
            h_masks = LC.pinned_empty((nmk, wb_in), np.uint8)
            h_out_d = LC.pinned_empty((w.n_pairs, wb_out), np.uint8)
            h_out_a = LC.pinned_empty((w.chunks, wb_out), np.uint8)
            wc, wm = g.pack(cts.view(nct, 2, g.nq, g.N), 2, L), g.pack(masks, 2, L)
            g.sync()
            h_cts[...] = wc.cpu().numpy()
            h_masks[...] = wm.cpu().numpy()
            del wc, wm
            torch.cuda.synchronize()

            def wire_set():
                u8 = dict(dtype=torch.uint8, device=cts.device)
                return (torch.empty((nct, wb_in), **u8), torch.empty((nmk, wb_in), **u8),
                        torch.empty((w.n_pairs, wb_out), **u8), torch.empty((w.chunks, wb_out), **u8))
            bufs = [wire_set() for _ in range(2)]
            d_cts, d_masks = torch.empty_like(cts), torch.empty_like(masks)
            h2d_bytes = int(h_cts.nbytes + h_masks.nbytes)
            d2h_bytes = int(h_out_d.nbytes + h_out_a.nbytes)

            def compute(b):
                w_cts, w_masks, w_d, w_a = b
                g.unpack(w_cts, nct, 2, L, out=d_cts)
                g.unpack(w_masks, nmk, 2, L, out=d_masks)
                g.distances(evk, d_cts, w.n_clients, w.chunks, g.scale, mode=dmode, groups=sched, out=out_d)
                g.masked_aggregate(evk, d_cts, w.n_clients, w.chunks, g.scale, d_masks, g.scale, mode=mode, out=out_a)
                g.pack(out_d, 2, L - 1, out=w_d)
                g.pack(out_a, 2, L - 1, out=w_a)

            def serial_step():
                w_cts, w_masks, w_d, w_a = bufs[0]
                g.h2d(w_cts, h_cts)
                g.h2d(w_masks, h_masks)
                compute(bufs[0])
                g.d2h(h_out_d, w_d)
                g.d2h(h_out_a, w_a)
                g.sync()

            def pipelined(steps):
                tin = [None, None]
                tout = [None, None]
                tin[0] = [g.copy_async(bufs[0][0], h_cts), g.copy_async(bufs[0][1], h_masks)]
                for k in range(steps):
                    a, b = k % 2, (k + 1) % 2
                    if k + 1 < steps:  # ordered after step k-1, the last user of buffer set b
                        tin[b] = [g.copy_async(bufs[b][0], h_cts), g.copy_async(bufs[b][1], h_masks)]
                    for t in tin[a]:
                        g.copy_wait(t)
                    for t in (tout[a] or []):  # results of step k-2 leave buffer set a first
                        g.copy_wait(t)
                    compute(bufs[a])
                    tout[a] = [g.copy_async(h_out_d, bufs[a][2]), g.copy_async(h_out_a, bufs[a][3])]
                g.sync()
                torch.cuda.synchronize()

            def timed(fn):
                barrier()
                t0 = time.perf_counter()
                fn()
                return max_over_ranks(time.perf_counter() - t0, world)

            serial_step()
            el = timed(lambda: [serial_step() for _ in range(args.steps)])
            e2e_serial = {"value": whole_job_rate(w.n_pairs, world, args.steps, el), "unit": UNIT,
                          "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes}
            pipelined(2)
            el = timed(lambda: pipelined(args.steps))
            e2e = {"value": whole_job_rate(w.n_pairs, world, args.steps, el), "unit": UNIT,
                   "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
                   "link_GBps": (h2d_bytes + d2h_bytes) * args.steps / el / 1e9,
                   "bound": "host link: the step's wire-form copies take longer than its compute "
                            "(link_GBps is the copies' bytes over the pipelined wall time)",
                   "form": "wire form (lc_pack/lc_unpack on the device); double-buffered: next step's H2D and "
                           "previous step's D2H overlap this step's compute",
                   "serial": e2e_serial}
            del bufs, d_cts, d_masks

    # the two halves of a step timed alone (device time, CUDA events): distances and the masked
    # aggregate (chunks/s beside the pair metric)
    parts = None
    if args.mode == "batched":
        with torch.cuda.stream(stream):
            def tm(fn, reps=3):
                fn()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    fn()
                e1.record(stream)
                torch.cuda.synchronize()
                return e0.elapsed_time(e1) / reps
            dms = tm(lambda: g.distances(evk, cts, w.n_clients, w.chunks, g.scale, mode=dmode, groups=sched,
                                         out=out_d))
            ams = tm(lambda: g.masked_aggregate(evk, cts, w.n_clients, w.chunks, g.scale, masks, g.scale, mode=mode,
                                                out=out_a))
        parts = {"distances_ms": dms, "pairs_per_s": w.n_pairs / (dms / 1e3), "aggregate_ms": ams,
                 "aggregate_chunks_per_s": w.chunks / (ams / 1e3), "launch": "eager"}

    # the clients' step on the device: GPU encode + encryption with device randomness of all
    # n x chunks update chunks (beside the server metric; not part of a step)
    client = None
    if not args.no_client:
        with torch.cuda.stream(stream):
            X = S.split_chunks(S.client_updates(w), g.slots)
            zt = torch.tensor(X.reshape(-1, g.slots), device=f"cuda:{local}")
            dst = torch.empty_like(cts)
            g.encode_encrypt_seeded(evk_pk, zt, g.scale, 1, 0, out=dst)  # warm
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                g.encode_encrypt_seeded(evk_pk, zt, g.scale, 1, 0, out=dst)
            e1.record(stream)
            torch.cuda.synchronize()
            cms = e0.elapsed_time(e1) / 3
            client = {"ciphertexts": int(zt.shape[0]), "ms": cms, "ciphertexts_per_s": zt.shape[0] / (cms / 1e3),
                      "form": "GPU FP64 encode + encryption with device randomness (Philox4x64-10)"}
            del zt, dst

    # the plain per-operation form on the same inputs (reference point of the batched form)
    plain = None
    if args.mode == "batched" and not args.no_plain:
        with torch.cuda.stream(stream):
            plain_step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                plain_step()
            e1.record(stream)
            torch.cuda.synchronize()
            pms = e0.elapsed_time(e1) / 2
        plain = {"value": w.n_pairs / (pms / 1e3), "unit": UNIT, "ms_per_step": pms,
                 "form": "per-operation launches (one pair / chunk at a time), log-step rotations, 14 keys",
                 "batched_over_plain": (w.n_pairs / (ms_per_step / 1e3)) / (w.n_pairs / (pms / 1e3))}

    # the same step with the rescaled pairs dropped to level 1 (q_0 q_1) before the rotate-and-sum
    # (LC_ROTATE_AT_LEVEL(1)): the rotations' key switches on 2 limbs instead of 14 (beside the
    # headline, which keeps the rotations at level 13)
    level_drop = None
    if args.mode == "batched" and not args.no_plain:
        with torch.cuda.stream(stream):
            out_d1 = g.empty(w.n_pairs, 2, 2, g.N)

            def drop_step():
                g.distances(evk, cts, w.n_clients, w.chunks, g.scale, mode=dmode, groups=sched, out=out_d1,
                            rot_level=1)
                g.masked_aggregate(evk, cts, w.n_clients, w.chunks, g.scale, masks, g.scale, mode=mode, out=out_a)
            drop_step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                drop_step()
            e1.record(stream)
            torch.cuda.synchronize()
            lms = e0.elapsed_time(e1) / 3
            _, sc1 = g.distances(evk, cts, w.n_clients, w.chunks, g.scale, mode=dmode, groups=sched, out=out_d1,
                                 rot_level=1)
            got = g.decrypt_const(s, out_d1, 1, sc1)
            W0 = S.client_updates(w)
            ref = np.array([np.sum((W0[i] - W0[j]) ** 2) for i in range(w.n_clients) for j in range(i + 1, w.n_clients)])
            del out_d1, W0
        level_drop = {"rot_level": 1, "value": w.n_pairs / (lms / 1e3), "unit": UNIT, "ms_per_step": lms,
                      "max_rel_err_vs_fp64": float(np.max(np.abs(got - ref) / ref)),
                      "form": "same step with LC_ROTATE_AT_LEVEL(1): rescaled pairs reduced to q_0 q_1 before the "
                              "rotate-and-sum (eager launches)"}

    # roofline of the dominant kernel class
    hbm, peak_kind = peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] > 0 else 0.0
    traffic = None
    if dom == "ntt" and d["launches"]:
        # one "launch" = one batched transform call (column + row pass); algorithmic bytes are
        # 2 N 8 per limb, so limbs per call = bytes / (16 N) / calls
        limbs_per_call = d["bytes"] / (16.0 * g.N) / d["launches"]
        traffic = NTT_DRAM_BYTES_PER_LIMB * limbs_per_call
    hbm_view = {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    alu = None
    if dom == "ntt":
        with torch.cuda.stream(stream):
            alu = alu_roofline(g, d["bytes"], d["ms"], ck.get("sm_mhz"))
    if alu is not None:  # the transforms are bound by integer issue, not by DRAM
        roof = {"bound": "alu", "kernel": dom, "achieved": alu["achieved"], "peak": alu["peak"],
                "unit": alu["unit"], "frac": alu["frac"], "peak_source": alu["peak_source"],
                "frac_of_probe": alu["frac_of_probe"], "hbm": hbm_view, "alu": alu}
    else:
        roof = {"bound": "hbm", "kernel": dom, **hbm_view}
    # the key-switch kernels beside it: algorithmic HBM bytes over their device time, against the
    # measured copy bandwidth; their SM throughput comes from the committed ncu captures
    ks = {}
    for cls, sm in (("inner", KS_SM_PCT.get("inner")), ("modup", KS_SM_PCT.get("modup")),
                    ("moddown", KS_SM_PCT.get("moddown"))):
        v = prof.get(cls)
        if v and v["ms"] > 0:
            gbs = v["bytes"] / (v["ms"] / 1e3) / 1e9
            ks[cls] = {"GBps": gbs, "frac_hbm": gbs / hbm, "ms_per_step": v["ms"] / args.steps,
                       "sm_throughput_pct_ncu": sm}
    roof["keyswitch"] = ks
    ntt_hbm = hbm_view["frac"] if dom == "ntt" else None
    ks_hbm = max((x["frac_hbm"] for x in ks.values()), default=None)
    roof["hbm_gate"] = {"target_frac": 0.6, "ntt_frac": ntt_hbm, "keyswitch_best_frac": ks_hbm,
                        "met": bool(ntt_hbm is not None and ntt_hbm >= 0.6 and ks_hbm is not None and ks_hbm >= 0.6),
                        "why_not": "the transforms and key-switch kernels are bound by 64-bit modular arithmetic "
                                   "on the 32-bit integer pipes (SM throughput 70-82 % in ncu) well before DRAM; "
                                   "see frac (integer issue bound) and frac_of_probe"}
    roof.update({
        "traffic": traffic,
        "traffic_source": ("ncu dram__bytes of the 960-limb transform case, per limb x limbs per call"
                           if traffic else None),
        "launches": d["launches"], "avg_launch_us": d["ms"] * 1e3 / max(1, d["launches"]),
        "share_of_step": d["ms"] / (ms if not use_graph else sum(v["ms"] for v in prof.values()) or 1.0),
        "measured_in": "timed region with per-launch CUDA events" + (" (eager replay of the graph's steps)"
                                                                     if use_graph else ""),
        "classes": {k: {"ms_per_step": v["ms"] / args.steps, "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9)
                        if v["ms"] > 0 else 0.0, "launches_per_step": v["launches"] / args.steps}
                    for k, v in prof.items()}})
    # served rounds: a bounded Poisson stream through the serving loop (untimed by the step clock)
    serving = None
    if rank == 0 and world == 1 and args.mode == "batched" and not args.no_serving and args.serving_rounds > 0:
        serving = serving_leg(args, g, stream, local, sched, dmode & LC.LC_HOIST_QP_SUM)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": plain_config(world),
            "run_detail": {"mode": args.mode, "rotation_schedule": sched_name,
                           "rotation_keys_loaded": len(evk.rotations),
                           "tuning": ({"knobs": tuning["knobs"], "ms": tuning["ms"], "seconds": tuning["seconds"],
                                       "trials": len(tuning["trials"]), "schedules_tried": tuning.get("schedules")}
                                      if tuning else g.tuning()),
                           "launch": "cuda_graph_replay" if use_graph else "eager"},
            "gpu_launches": launches, "clocks": ck, "roofline": roof, "e2e": e2e, "plain_form": plain,
            "client_step": client, "step_parts": parts, "serving": serving, "level_drop": level_drop,
            "round_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                                 "definition": "per-step device time of the fixed n=10 step (45 pair distances + "
                                               "masked aggregate of 64 chunks); served latencies are in 'serving'"}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        osched = sched_name if sched_name in SCHEDULES else "g3qp"
        v, per, threads, step_s = oracle_sample(w, reps=1, sched_name=osched)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"1 pair (64 chunks, rotation schedule {osched}"
                                          f"{' = one-ModDown groups ' + str(SCHEDULES[osched]) if osched.endswith('qp') else ''}"
                                          f") + 1 aggregate chunk, at the workload's 45 pairs + 64 chunks; measured "
                                          f"pair {per[0][0]:.2f} s, chunk {per[0][1]:.2f} s ({step_s:.0f} s per full step)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
