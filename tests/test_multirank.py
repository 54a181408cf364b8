"""The multi-process path of bench.py on CPU (gloo, world size 2): replicas
only -- each rank runs its own copy of the workload with distinct Philox
replica indices, the timed region's duration is the maximum over the ranks,
the value counts every rank's atom-steps, and the reference arm runs on rank
0 alone.  No GPU and no data exchange beyond the timing reduction."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        ids = bench.rank_replica_ids(20, rank)
        all_ids = [None] * world
        dist.all_gather_object(all_ids, ids)
        ms = bench.max_over_ranks(10.0 + 2.5 * rank, dist, torch.device("cpu"))
        dist.barrier()
        rate = bench.whole_job_rate(1000 * 40480, world, ms)
        out = io.StringIO()
        if rank != 0:  # the reference arm: every rank but 0 exits at once, printing nothing
            args = type("A", (), {"steps": 3, "warmup": 3, "workload": "fl2"})()
            with redirect_stdout(out):
                bench.run_reference(args)
        q.put((rank, all_ids, ms, rate, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_bench_replicas_only_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, all_ids, ms, rate, printed in res:
        flat = [i for ids in all_ids for i in ids]
        assert sorted(flat) == list(range(40))            # distinct noise streams on the two ranks
        assert all_ids[rank] == list(range(20 * rank, 20 * rank + 20))
        assert ms == 12.5                                  # the slower rank's time, on both ranks
        assert rate == pytest.approx(2 * 1000 * 40480 / 12.5e-3)
    assert res[1][4] == ""                                 # rank 1 of the reference arm prints nothing
