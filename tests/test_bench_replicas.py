"""Host logic of bench.py's multi-GPU mode (independent replicas, no data-path
collective), run as two gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, B, steps, times, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.instance_seeds(rank, B)
        t_max = bench.max_over_ranks(times[rank], dist, "cpu")
        value = bench.whole_job_value(world, B, steps, t_max)
        q.put((rank, seeds, t_max, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    import torch.multiprocessing as mp

    world, B, steps = 2, 3, 4
    times = [1234.5, 987.25]  # ms of each rank's timed region
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, B, steps, times, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    seeds = [s for _, ss, _, _ in res for s in ss]
    assert len(set(seeds)) == world * B                      # disjoint instances
    for _, _, t_max, value in res:
        assert t_max == max(times)                           # the slowest rank's time
        assert value == pytest.approx(world * B * steps / (max(times) / 1e3))


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_single_process_reduction_is_identity():
    import bench

    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.instance_seeds(0, 2) == [0, 1]
    assert json.dumps(bench.whole_job_value(1, 32, 5, 2000.0)) == "80.0"
