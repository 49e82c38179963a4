"""The multi-GPU path of bench.py on CPU: two gloo ranks, each with its own
jobs (no data exchange), timing reduced to the slowest rank, and the
reference arm printing from rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    from paper_1910_13908_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank draws its own job: distinct seeds, distinct data
        spec = synth.config("c1", seed=bench.job_seed(rank))
        uvw = synth.station_uvw(spec)
        noise = synth.noise(spec, 0, 1)
        slowest = bench.max_over_ranks(10.0 + rank, world)
        out.put((rank, spec.seed, float(uvw.sum()), complex(noise.sum()), slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_jobs_and_take_the_slowest_time():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, u0, n0, t0), (r1, s1, u1, n1, t1) = res
    assert s0 != s1 and n0 != n1          # different jobs per rank
    assert u0 != u1
    assert t0 == t1 == 11.0               # max over ranks, identical everywhere


def test_reference_arm_prints_from_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
