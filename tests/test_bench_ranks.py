"""The replica (N > 1) path of bench.py on the CPU: two gloo ranks.

* the rank logic: every rank sees the same whole-job throughput, all ranks'
  units over the slowest rank's time, after the barrier;
* the reference arm under torchrun: rank 0 alone prints one JSON line and
  every rank exits 0.
"""
import json
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


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws_, rank_, local = bench.dist_setup(None)
    assert (ws_, rank_, local) == (ws, rank, rank)
    bench.barrier(ws_)
    # rank r processed 1000 (r + 1) units in 0.01 (r + 1) s
    out = bench.replica_value(ws_, 1000.0, 0.01 * (rank + 1))
    mx = bench.max_over_ranks(ws_, float(rank))
    bench.barrier(ws_)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, out, mx))


def test_replica_value_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (value, sec), mx in res:
        assert sec == pytest.approx(0.02)             # the slowest rank's time
        assert value == pytest.approx(2 * 1000.0 / 0.02)
        assert mx == 1.0


def test_replica_value_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_value(1, 500.0, 0.5) == (1000.0, 0.5)


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["value"] > 0 and out["e2e"]["h2d_bytes_per_step"] == 0
    assert out["cpu_baseline"]["kind"] == "oracle"
