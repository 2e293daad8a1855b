"""Host logic of bench.py's multi-rank runs, on the CPU with two gloo ranks: each rank works on its
own gauge configuration (no data-path collective), the timed region of the job is the slowest
rank's (one MAX all-reduce of the times), and the job's rate counts the units of every rank.  The
reference arm under a launcher with several ranks runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, root, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, root)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.reduce_max_over_ranks(1.0 + 0.25 * rank, world, "cpu")
    q.put((rank, t, bench.dist_env(), bench.link_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_time_and_configurations():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, ROOT, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time
    assert [g[1] for g in got] == [1.25, 1.25]
    assert [g[2] for g in got] == [(0, 2, 0), (1, 2, 1)]
    # one gauge configuration per rank
    assert got[0][3] != got[1][3]
    sys.path.insert(0, ROOT)
    import bench
    # 10 noises per rank in 2.5 s of the slowest rank: the job ran 20 noises in 2.5 s
    assert bench.job_rate(10, 2, 2.5) == pytest.approx(8.0)
    assert bench.reduce_max_over_ranks(3.0, 1, "cpu") == 3.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
