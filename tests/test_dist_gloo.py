"""The multi-rank logic of bench.py on CPU with two gloo ranks: replicas only
(one independent cell per rank), max-over-ranks step time, whole-job value =
time per processed cell, reference arm printed by rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r pretends its replica took (1 + r) s/iter and 1000 (1 + r) ms per step
        value, s_iter, ms = bench.aggregate_over_ranks(1.0 + rank, 1000.0 * (1 + rank), world, "cpu")
        q.put((rank, value, s_iter, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_divide_by_world():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, s_iter, ms in got:
        assert s_iter == 2.0 and ms == 2000.0
        assert value == 1.0  # two cells per 2.0 s max step


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
