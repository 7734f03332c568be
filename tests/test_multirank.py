"""The multi-GPU path of bench.py is replicas only (the retrieval has no
exchange step): these CPU tests run its rank logic with the gloo backend,
world size 2, and check the whole-job aggregation (max time over ranks,
bytes of all ranks) and that the reference arm runs on rank 0 only."""
import os
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(dist, times[rank], "cpu")
    dist.barrier()
    out[rank] = (ms, bench.job_gbs(world, 2_040_000_000, ms))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    world, port = 2, 29517
    times = [0.9, 1.3]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, gbs = res[r]
        assert ms == pytest.approx(1.3)
        assert gbs == pytest.approx(2 * 2_040_000_000 / 1.3e-3 / 1e9)


def test_reference_arm_rank_nonzero_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""


def test_single_process_aggregation():
    import bench
    assert bench.max_over_ranks(None, 2.5, "cpu") == 2.5
    assert bench.job_gbs(1, 1_000_000_000, 1.0) == pytest.approx(1000.0)


def _failing_worker(rank, world, port, out):
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    import bench
    try:
        if rank == 1:
            raise RuntimeError("rank 1 fails before its step is aggregated")
        bench.max_over_ranks(dist, 1.0, "cpu")   # waits for rank 1, which never joins
        out[rank] = "completed"
    except RuntimeError as e:
        out[rank] = f"error: {type(e).__name__}"
    finally:
        if rank == 0:
            dist.destroy_process_group()


def test_a_failing_rank_ends_the_others_with_an_error_gloo():
    """A rank that raises before the cross-rank aggregation: the surviving
    rank's collective ends with an error once the process-group timeout
    passes, instead of waiting for ever."""
    world, port = 2, 29533
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_failing_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[1].startswith("error")
    assert res[0].startswith("error")
