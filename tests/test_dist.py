"""Multi-process paths of bench.py on the CPU (gloo, world size 2).

One projection does not shard: `bench.py --gpus N` runs N replicas, joins
them with a barrier around the timed region and takes the maximum time over
the ranks; under torchrun the reference arm runs on rank 0 alone.  These
tests run those host-side paths with two gloo ranks on 127.0.0.1.
"""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_setup(0)  # no GPUs: the gloo backend
    import torch.distributed as dist
    bench.barrier(w)
    # each rank's time; every rank must see the largest
    m = bench.allreduce_max(10.0 + 5.0 * r, w, "cpu")
    # the whole-job value: all ranks' solves over the slowest rank's time
    steps = 4
    value = w * steps / (m / 1e3)
    out.put((r, w, local, m, value))
    dist.destroy_process_group()


def test_barrier_and_max_over_ranks_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 15.0 for r in res)  # the maximum over the two ranks
    assert all(abs(r[4] - 2 * 4 / 0.015) < 1e-9 for r in res)


def test_reference_arm_under_torchrun_prints_once():
    """torchrun with two ranks: rank 0 prints one JSON line of the CPU oracle
    arm, rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-budget", "0.1",
           "--edge", "16"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
