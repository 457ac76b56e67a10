"""The multi-GPU path of bench.py on the CPU: with N ranks every rank runs an
independent replica of the workload (the step has no exchange between
GPUs), the job time is the max over ranks and the job rate is N times the
cells over that time.  Two gloo ranks check the helpers bench.py uses for
this, and the reference arm's rule that only rank 0 prints."""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.ranks_barrier()
        t = bench.max_over_ranks(0.1 * (rank + 1), "cpu")
        rate = bench.whole_job_rate(1000, world, t)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t!r} {rate!r}\n")
        bench.ranks_barrier()
    finally:
        tdist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        t, rate = (float(v) for v in open(tmp_path / f"r{r}.txt").read().split())
        assert t == 0.2                     # the slowest rank's time, on every rank
        assert rate == world * 1000 / 0.2


def test_helpers_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.ranks_barrier()
    assert bench.max_over_ranks(0.25, "cpu") == 0.25
    assert bench.whole_job_rate(100, 1, 0.5) == 200.0


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
