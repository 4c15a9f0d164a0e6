"""The multi-GPU path runs independent replicas (one per rank); the only
collective is the max over ranks of the timed region.  Checked here with two
CPU processes over gloo (127.0.0.1): the max, the whole-job throughput, and that
a rank raising before the collective makes the others fail with an error
(short process-group timeout) instead of hanging."""
import datetime
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, mode, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    try:
        if mode == "fail" and rank == 1:
            raise RuntimeError("rank 1 fails before the timed region")
        if mode == "fail":
            dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=5))
            d = dist
        else:
            _, _, _, d = bench.dist_setup(None, backend="gloo")
        ms = 10.0 + 5.0 * rank                           # rank 1 is the slowest
        total = bench.max_over_ranks(ms, d, device="cpu")
        value = bench.whole_job_value(1000, world, total)
        q.put((rank, "ok", total, value))
        d.destroy_process_group()
    except Exception as e:                               # reported to the parent
        q.put((rank, "error", type(e).__name__, str(e)[:80]))


def run(world, mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, mode, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(60)
        assert p.exitcode is not None, "rank hung"
    return sorted(q.get(timeout=5) for _ in range(world))


def test_max_over_ranks_gloo():
    res = run(2, "ok")
    assert [r[1] for r in res] == ["ok", "ok"]
    assert all(r[2] == 15.0 for r in res)                # max over ranks
    assert all(abs(r[3] - 2 * 1000 / 15e-3) < 1e-9 for r in res)


def test_failed_rank_does_not_hang():
    res = run(2, "fail")
    assert res[1][1] == "error" and "rank 1 fails" in res[1][3]
    assert res[0][1] == "error"                          # rendezvous / collective timed out
