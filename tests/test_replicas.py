"""The multi-rank (independent replicas) path of the benchmark on CPU: two gloo ranks on
127.0.0.1 join through the same helpers bench.py uses; the whole-job throughput is the work of
all ranks over the slowest rank's time, and every rank sees the same result."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_2603_25233_gb300 import replicas
    w, r, _ = replicas.init()
    replicas.barrier(w)
    units = 1000.0 * (r + 1)            # rank r did (r + 1) thousand units
    seconds = 2.0 + r                   # in 2 + r seconds
    rate, t_max, total = replicas.aggregate(units, seconds, w)
    out.put((r, w, rate, t_max, total, replicas.reduce_max(float(r), w)))
    replicas.finalize(w)


def test_two_gloo_replicas_aggregate_throughput():
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
    for r, w, rate, t_max, total, mx in res:
        assert w == 2
        assert t_max == 3.0 and total == 3000.0 and mx == 1.0
        assert abs(rate - 1000.0) < 1e-12


def test_single_rank_needs_no_process_group():
    from paper_2603_25233_gb300 import replicas
    assert replicas.aggregate(10.0, 4.0, 1) == (2.5, 4.0, 10.0)
    replicas.barrier(1)
    replicas.finalize(1)
