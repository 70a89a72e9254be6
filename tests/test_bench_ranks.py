"""Host logic of bench.py's multi-GPU mode on the CPU: two `gloo` ranks (world size 2).

With N > 1 every rank runs an independent replica of the workload; the job's time is the
slowest rank's (a MAX all-reduce) and its throughput counts every rank's units.  Only
rank 0 prints, and the CPU reference arm runs on rank 0 alone."""
import json
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        seconds = bench.max_over_ranks(dist, 1.0 + rank, "cpu")  # rank r took 1 + r seconds
        queue.put((rank, seconds, bench.job_throughput(world, 3e6, seconds)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
        assert p.exitcode == 0
    got = sorted(queue.get(timeout=10) for _ in range(2))
    for rank, seconds, value in got:
        assert seconds == 2.0                 # both ranks see the slower rank's time
        assert value == 2 * 3e6 / 2.0 / 1e6   # both replicas' units over that time


def test_single_process_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(None, 1.5, "cpu") == 1.5
    assert bench.job_throughput(1, 2e6, 0.5) == 4.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    args = bench.parse(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"])
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
