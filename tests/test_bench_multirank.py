"""The multi-rank paths of bench.py, on CPU with the gloo backend and world size 2:
whole-job aggregation (replicas, slowest rank's time) and the reference arm, which runs
on rank 0 only while the other ranks exit without work."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), AFMM_BENCH_GLOO="1")
    sys.path.insert(0, ROOT)
    import bench
    ws_, rank_, _ = bench.dist_setup()
    # aggregation: rank 0 took 100 ms, rank 1 took 250 ms for 1e6 units each
    val, t = bench.aggregate(ws_, 1e6, 100.0 if rank_ == 0 else 250.0, "cpu")
    bench.barrier(ws_)
    dist.destroy_process_group()
    # reference arm: rank 0 times the oracle on a tiny sample, others return at once
    args = type("A", (), dict(gpus=ws, steps=1, warmup=0, ns=300, nf=64))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(args)
    dist.destroy_process_group()
    q.put((rank_, val, t, rc, buf.getvalue()))


def test_world_size_two_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, val, t, rc, out in res:
        assert t == 250.0
        assert abs(val - 2e6 / 0.25) < 1e-6
        assert rc == 0
    assert res[1][4] == ""  # rank 1 prints nothing
    line = json.loads(res[0][4].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "modal ring interactions/s"
    assert line["cpu_baseline"]["kind"] == "oracle"
