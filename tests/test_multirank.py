"""The bench's N > 1 path on CPU: two gloo ranks (replicas only, no data exchange).

Every rank times its own replica; the job reports the slowest rank's step
time and the source bytes of all ranks.  The reference arm runs on rank 0
only: other ranks exit at once without output.
"""
import importlib.util
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        mine = 1.0 + rank * 0.5  # rank r timed 1.0 + r/2 ms per step
        dist.barrier()
        worst = bench.max_over_ranks(mine, torch.device("cpu"))
        q.put((rank, worst, bench.whole_job_gbs(1_000_000, world, worst)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    world, port = 2, 29613
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, worst, gbs in got:
        assert worst == pytest.approx(1.5)  # max over ranks
        assert gbs == pytest.approx(2 * 1_000_000 / 1.5e-3 / 1e9)  # all ranks' bytes


def test_single_process_needs_no_group():
    bench = _bench()
    assert bench.max_over_ranks(3.25, torch.device("cpu")) == 3.25
    assert bench.whole_job_gbs(4096 * 2048 * 2, 1, 0.2) == pytest.approx(83.886, rel=1e-4)


def test_reference_arm_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
