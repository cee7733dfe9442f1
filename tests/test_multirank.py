"""The bench's multi-process path on CPU (gloo, world size 2, 127.0.0.1):
the timed region's max over ranks and the whole-job rate, and the reference
arm printing one JSON line from rank 0 only.  One process per GPU runs an
independent replica of the SpMV (the method has no data exchange between
replicas), so these reductions are the whole collective part of the path."""
import contextlib
import io
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)  # rank 1 is the slower one
        rate = bench.job_rate(ws, 1e9, ms)
        out = io.StringIO()

        class A:
            n, steps, warmup = 3000, 2, 1
        with contextlib.redirect_stdout(out):
            bench.run_reference(A, ws, rank)
        dist.barrier()
        q.put((rank, ms, rate, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_and_report():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, ms, rate, text in res:
        assert ms == 15.0                          # the slowest rank bounds the job
        assert abs(rate - 2 * 1e9 / 15e-3 / 1e9) < 1e-9
    assert res[1][3] == ""                         # rank 1 prints nothing
    line = json.loads(res[0][3].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
