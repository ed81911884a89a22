"""The benchmark's multi-GPU path on the CPU: replicas on world_size 2 with the
gloo backend.  Every rank gets the slowest rank's time, and the whole-job
throughput counts the units of all ranks; under torchrun the reference arm
(the oracle) prints one line, from rank 0, and the other rank exits 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sync = bench.RankSync(dist, "cpu")
    sync.barrier()
    elapsed = 1.0 + rank                     # rank 1 is the slower replica
    slowest = sync.max(elapsed)
    value = bench.job_mlups(world, 1000, 50, slowest)
    sync.barrier()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as fh:
        json.dump({"slowest": slowest, "value": value}, fh)
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_every_rank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        with open(tmp_path / ("rank%d.json" % r)) as fh:
            got = json.load(fh)
        assert got["slowest"] == 2.0
        assert got["value"] == pytest.approx(2 * 1000 * 50 / 2.0 / 1e6)


def test_single_process_sync_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    s = bench.RankSync(None, "cpu")
    s.barrier()
    assert s.max(3.5) == 3.5
    assert bench.job_mlups(1, 2_097_152, 100, 0.075) == pytest.approx(2796.2, rel=1e-4)


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
