"""The multi-GPU path of bench.py is replicas only: every rank runs its own
convolutions and rank 0 reports all ranks' work over the slowest rank's time.
This checks that aggregation with two gloo ranks on the CPU (no GPU)."""
import os
import socket
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


WORKER = textwrap.dedent("""
    import os, sys
    sys.path.insert(0, {root!r})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="env://")
    world, rank, local = bench.dist_env()
    assert world == 2 and rank in (0, 1)
    bench.barrier(world)
    # rank r took (10 + 5 r) ms for (100 + r) units of work
    ms, units = bench.aggregate(10.0 + 5.0 * rank, 100.0 + rank, world, None)
    assert ms == 15.0, ms          # the slowest rank's time
    assert units == 201.0, units   # all ranks' work
    dist.destroy_process_group()
    print("ok", rank)
""")


@pytest.mark.timeout(120)
def test_two_rank_aggregation_max_time_sum_work(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=110)[0] for p in procs]
    for rank, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        assert f"ok {rank}" in out


def test_reference_arm_rank_one_does_no_work(tmp_path):
    """Under torchrun only rank 0 runs the reference arm; other ranks exit 0 without output."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""
