"""The multi-GPU path is replicas only: each rank runs its own copy of the
workload with no collective on the data path, and the benchmark combines
ranks by the slowest rank's time.  This host logic runs here as two gloo
ranks on CPU (127.0.0.1)."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [40.0, 55.0][rank]                      # rank 1 is the slow one
    ms_max, value = bench.combine_ranks(ms, world, 1, 10, torch.device("cpu"))
    out[rank] = (ms_max, value)
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms_max, value = res[r]
        assert ms_max == 55.0
        assert value == pytest.approx(2 * 10 / 0.055)   # both ranks' products over the max time


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun the reference arm prints from rank 0 alone; other ranks
    exit 0 without work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
