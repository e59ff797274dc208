"""Multi-process host logic of the benchmark on CPU (gloo, world size 2):
every rank works on its own independent batches (weak scaling, no collective
on the data path); the job time is the max over ranks and the throughput
counts every rank's units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_ms = 10.0 * (rank + 1)          # rank 1 is the slowest
    mx = bench.barrier_max(ws, local_ms)
    value = bench.weak_scaling_value(ws, 4096, 64, mx)
    # each rank draws its own inputs: seeds differ per rank
    from paper_2608_25666_b300 import workloads
    b = workloads.make_batch(workloads.WORKLOADS["single"], step=rank * 64)
    q.put((rank, mx, value, float(b["xi"][0, 0, 0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_host_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res[0][1] == res[1][1] == 20.0
    assert res[0][2] == pytest.approx(2 * 4096 * 64 / 0.020)
    assert res[0][3] != res[1][3]          # independent per-rank batches
