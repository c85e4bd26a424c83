"""Multi-rank paths of bench.py on CPU: two gloo ranks aggregate their step
times with a MAX all-reduce (the slowest replica sets the whole-job time),
and the reference arm runs on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    total_ms = [40.0, 55.0][rank]
    res = bench.aggregate_over_ranks(total_ms, 10, 1e9, world, dist, "cpu")
    q.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        total, per_step, value = out[r]
        assert total == 55.0 and per_step == 5.5
        # both replicas' work over the slowest replica's time
        assert value == pytest.approx(1e9 * 10 * 2 / 0.055 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    total, per_step, value = bench.aggregate_over_ranks(20.0, 4, 2e9, 1)
    assert (total, per_step) == (20.0, 5.0)
    assert value == pytest.approx(2e9 * 4 / 0.02 / 1e9)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
