"""Host logic of the benchmark's multi-rank path, on CPU.  With N GPUs the benchmark
runs N independent replicas of the apply (the path does not shard on one GPU per
process); each times its own applies and the job's time is the slowest rank's, taken
with an all-reduce (gloo here, world size 2).  Under torchrun the reference arm runs on
rank 0 alone and the other ranks exit without work."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, values, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sys.path.insert(0, ROOT)
        import bench
        got = bench.max_over_ranks(values[rank], world, "cpu")
        with open(os.path.join(outdir, f"rank{rank}.txt"), "w") as f:
            f.write(repr(got))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_replica(tmp_path):
    import torch.multiprocessing as mp
    values = [0.25, 0.3125]
    mp.spawn(_replica, args=(2, _free_port(), values, str(tmp_path)), nprocs=2, join=True)
    got = [float((tmp_path / f"rank{r}.txt").read_text()) for r in range(2)]
    assert got == [max(values)] * 2


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, 1, "cpu") == 0.5


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_traffic_record_key_ignores_comments_only():
    """The DRAM-traffic record of a kernel is keyed to its code: comment or blank-line
    edits keep the key, any code edit changes it."""
    sys.path.insert(0, ROOT)
    import bench
    base = "int f(int x) {\n  // twice\n  return 2 * x;  /* doubled */\n}\n"
    assert bench._code_only(base) == bench._code_only(base.replace("// twice", "// two times") + "\n\n")
    assert bench._code_only(base) == bench._code_only(base.replace("/* doubled */", "/* x2\n spanning */"))
    assert bench._code_only(base) != bench._code_only(base.replace("2 * x", "3 * x"))
    assert "twice" not in bench._code_only(base) and "return 2 * x;" in bench._code_only(base)
