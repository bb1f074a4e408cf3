"""The N > 1 path of bench.py on the CPU: gloo ranks (world size 2) for the whole-job
aggregation of independent replicas, and the reference arm's rank handling under torchrun.
No GPU is used."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank r timed 10 + 5 r ms for 1000 (r + 1) units
    ms, rate = bench.job_rate(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world, dist, device="cpu")
    out[rank] = (ms, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_all_units():
    world, port = 2, 29533
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == 15.0
        assert rate == pytest.approx(3000.0 / 15e-3)


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(20.0, 4000.0, 1) == (20.0, 4000.0 / 20e-3)


def test_reference_arm_non_zero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
