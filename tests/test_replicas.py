"""The multi-GPU form is replicas only (no collective on the data path): each rank runs the whole
workload, timing is the slowest rank's, and the job's throughput counts every rank's units.
Checked with two gloo ranks on the CPU (bench.py's own helpers)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [2.0, 2.5][rank]  # rank 1 is the slow one
        slowest = bench.max_over_ranks(secs, world)
        rate = bench.whole_job_rate(45, world, 5, slowest)
        q.put((rank, slowest, rate, bench.dist_info()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_units():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, info in res:
        assert slowest == 2.5
        assert rate == pytest.approx(2 * 45 * 5 / 2.5)
        assert info == (rank, 2, 0)


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.whole_job_rate(45, 1, 5, 0.2) == pytest.approx(1125.0)


def test_both_arms_name_the_same_workload():
    """The benchmark's own line and the reference arm's line carry one `config` (the workload and
    its shape); run-specific details go elsewhere.  The schedules the bench can run are the
    autotuner's search space."""
    sys.path.insert(0, ROOT)
    import bench
    cfg = bench.plain_config(1)
    assert cfg == bench.plain_config(1) and cfg["workload"] == bench.WORKLOAD
    assert (cfg["n_clients"], cfg["chunks"], cfg["pairs"], cfg["log_n"], cfg["limbs_q"]) == (10, 64, 45, 15, 15)
    assert "l2" in cfg and "rotation_schedule" not in cfg
    assert bench.plain_config(4)["parallelism"] == "replicas4"
    assert bench.SCHEDULES["g3qp"] == [3, 3, 3, 3, 2] and bench.SCHEDULES["g4433qp"] == [4, 4, 3, 3]
    assert bench.BFLY_MIN_INSTR == 17  # the 40-bit primes' butterfly with the three-product quotient
