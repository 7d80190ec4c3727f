"""The N>1 bench path on CPU: replicas as gloo ranks (world size 2).

The solver for one geometry runs on one GPU; with N GPUs the bench runs N independent
replicas (rank r solves the star of seed r) and reports the units all ranks processed
over the slowest rank's time.  These tests run the host side of that contract as
processes with the gloo backend: the max-over-ranks reduction, distinct replica inputs,
the whole-job value, and the reference arm launched by torchrun with two ranks."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2210_08580_gb300 import inputs as I
    local_seconds = 0.5 + rank            # rank 1 is the slow one
    t = bench.reduce_max(local_seconds, dist, "cpu")
    verts, _, _ = I.equal_chord_mesh(I.random_star(bench.replica_seed(rank)), 64)
    np.save(os.path.join(out_dir, f"verts{rank}.npy"), verts)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"max": t, "value": bench.job_value(1024, world, t)}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_reduce_to_the_slowest_rank(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    r = [json.load(open(tmp_path / f"r{i}.json")) for i in range(world)]
    assert r[0]["max"] == r[1]["max"] == pytest.approx(1.5)
    assert r[0]["value"] == pytest.approx(1024 * 2 / 1.5)
    v0, v1 = (np.load(tmp_path / f"verts{i}.npy") for i in range(world))
    assert v0.shape == v1.shape and not np.allclose(v0, v1)   # independent problems


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
