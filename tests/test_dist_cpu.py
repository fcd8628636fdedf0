"""CPU tests of the multi-process path of bench.py (replicas, one process per GPU
on the GPU machine): the gloo process group, the max-over-ranks reduction of the
timed region and the barrier, with world size 2; and the reference arm launched
under torch.distributed.run with two ranks, where rank 0 alone prints the line
and every rank exits 0."""
import json
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


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench._dist()
    bench._init_pg(w, "gloo")
    bench._barrier(w)
    # each rank "times" a different duration; every rank must see the maximum
    m = bench._max_over_ranks(10.0 + 5.0 * r, w, "cpu")
    bench._barrier(w)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fh:
        json.dump({"rank": r, "world": w, "max": m}, fh)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_gloo_world2_max_over_ranks_and_barrier(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [g["rank"] for g in got] == [0, 1]
    assert all(g["world"] == 2 and g["max"] == 15.0 for g in got)


def test_single_process_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.25, 1, "cpu") == 3.25
    bench._barrier(1)  # no process group needed


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
