"""The bench's N > 1 path, on CPU with two gloo ranks: every rank times its own time slice
(different data), the whole-job time is the slowest rank's (max over ranks), the throughput
counts every rank's units, only rank 0 prints the JSON line, and the reference arm runs on
rank 0 alone (the other ranks return 0 without work)."""
import argparse
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.world_env()
        t_slow = bench.max_over_ranks(0.5 + r, dist, "cpu")        # rank 1 is the slow one
        rate = bench.job_rate(w, 100.0, t_slow)
        out, old = io.StringIO(), sys.stdout
        sys.stdout = out
        try:
            bench.emit({"rank": r, "rate": rate}, r)
            rc = bench.run_reference(argparse.Namespace(steps=1, warmup=0), w, r) if r != 0 else None
        finally:
            sys.stdout = old
        q.put((r, w, lr, t_slow, rate, bench.slice_seed(r), out.getvalue(), rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    (r0, w0, l0, t0, v0, s0, out0, _), (r1, w1, l1, t1, v1, s1, out1, rc1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert t0 == t1 == 1.5                                     # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 100.0 / 1.5)          # both ranks' units over that time
    assert s0 != s1                                            # different time slices
    assert json.loads(out0) == {"rank": 0, "rate": v0} and out1 == ""
    assert rc1 == 0                                            # reference arm: no work off rank 0
