"""The multi-process side of `bench.py` on the CPU: N > 1 runs independent
replicas, one per rank, and reports the whole job's rate over the slowest
rank's time (no data-path collective; the only exchange is the MAX of the
timings).  Two gloo ranks on 127.0.0.1 stand in for two GPUs."""
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


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from bench import whole_job_rate
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # rank r timed 3 solves in 1 + r seconds
        rate, tot = whole_job_rate(1.0 + rank, 3, dist, "cpu")
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{rate!r} {tot!r}\n")
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    pytest.importorskip("torch.distributed")
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        rate, tot = map(float, (tmp_path / f"r{r}.txt").read_text().split())
        # every rank sees the slowest rank's time and all ranks' solves
        assert tot == 2.0
        assert rate == world * 3 / 2.0


def test_whole_job_rate_single_process():
    sys.path.insert(0, ROOT)
    from bench import whole_job_rate
    assert whole_job_rate(0.5, 4) == (8.0, 0.5)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "2", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
