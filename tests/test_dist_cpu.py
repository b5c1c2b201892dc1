"""The multi-rank path of bench.py on CPU with the gloo backend, world size 2:
each rank's timing reduces to the maximum over ranks, ranks draw disjoint
seeded instances (independent replicas, no data-path collective), and the
whole-job rate counts every rank's work against that maximum time."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t_local = 1.0 + 0.5 * rank
    t = bench.max_over_ranks(t_local, ws, "cpu")
    inst = bench.free_instances(rank, 1)[0]
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, float(np.abs(inst.u0).sum()), bench.whole_job_rate(100.0, ws, t)))


def test_two_rank_reduction_and_replica_seeds():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [1.5, 1.5]            # max over ranks on every rank
    assert res[0][2] != res[1][2]                       # different seeded instances per rank
    assert res[0][3] == pytest.approx(2 * 100.0 / 1.5)  # whole-job rate: all ranks' units / max time


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
