"""The N > 1 host logic of bench.py on CPU: two gloo ranks on 127.0.0.1 agree on the slowest
rank's step time, aggregate the replicas' throughput, and only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init("gloo")
    try:
        my_ms = 10.0 + 5.0 * r                         # rank 1 is the slower replica
        bench.barrier(w)
        ms_max = bench.max_over_ranks(my_ms, w)
        value = bench.aggregate(ms_max, w)

        class A:
            gpus, steps, warmup = w, 1, 0

        printed = None
        if r != 0:
            # the reference arm returns at once on every rank but 0 (no oracle work, no output)
            printed = bench.run_reference(A(), w, r)
        q.put((r, w, local, ms_max, value, printed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_agree_on_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == pytest.approx(15.0) for o in out)          # max over ranks
    assert all(o[4] == pytest.approx(2 * 1000.0 / 15.0) for o in out)
    assert out[1][5] is None
