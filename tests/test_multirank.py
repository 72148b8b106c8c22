"""The multi-process path of bench.py on CPU (gloo, world size 2): every rank
takes its own maps, the job time is the slowest rank's, the throughput counts
the pixels of all ranks, and the reference arm runs on rank 0 only."""

import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = 0.010 + 0.005 * rank                       # rank 1 is slower
    tmax = bench.max_over_ranks(t, world, "cpu")
    out[rank] = (bench.first_map(rank, 32), tmax, bench.job_gpix(world, 32 * 12 * 1024 ** 2, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as man:
        out = man.dict()
        procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        r0, r1 = out[0], out[1]
    assert (r0[0], r1[0]) == (0, 32)                  # disjoint batches of maps
    assert r0[1] == r1[1] == pytest.approx(0.015)     # the slowest rank's time on every rank
    assert r0[2] == pytest.approx(2 * 32 * 12 * 1024 ** 2 / 0.015 / 1e9)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
