"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank runs
its own replica of the workload (independent problems, no collective on the
data path); the job time is the slowest rank's, the job rate counts every
rank's units; the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world, torch.device("cpu"))
        v = bench.job_throughput(1000.0, 5, world, t)
        dist.barrier()
        out.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_rate_counts_all_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [120.0, 150.0]  # ms of timed steps on rank 0, rank 1
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 150.0
        assert v == pytest.approx(1000.0 * 5 * world / 0.150)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, 1) == 7.0
    assert bench.job_throughput(10.0, 2, 1, 1000.0) == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun every rank starts bench.py --impl reference; the ranks
    other than 0 exit at once, doing no work and printing nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
