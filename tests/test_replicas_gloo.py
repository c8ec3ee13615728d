"""The multi-GPU form of this path is replicas over samples (no data-path
collective).  This checks the host-side logic with two gloo ranks on CPU:
each rank takes its own slice of the seeded sample stream (bench.rank_samples),
simulates it (here with the CPU oracle), and the max-over-ranks time reduction
and the gathered per-sample results equal a single-process run over all
samples."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, per_rank, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    import ranc_workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    net = W.tiny_5core()
    first, n = bench.rank_samples(rank, per_rank)
    x = W.rate_coded_inputs(net.meta["seed"], n, 8, 784, 0.15, first_sample=first)
    r = oracle.run(net, x, 9)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    outs = [torch.zeros((n, 10), dtype=torch.int64) for _ in range(ws)]
    dist.all_gather(outs, torch.from_numpy(r["out"].astype(np.int64)))
    if rank == 0:
        q.put((float(t.item()), torch.cat(outs).numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_samples(oracle_mod):
    import ranc_workloads as W
    ws, per_rank = 2, 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, per_rank, q)) for r in range(ws)]
    for p in procs:
        p.start()
    tmax, gathered = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == float(ws)
    net = W.tiny_5core()
    x = W.rate_coded_inputs(net.meta["seed"], ws * per_rank, 8, 784, 0.15)
    ref = oracle_mod.run(net, x, 9)
    np.testing.assert_array_equal(gathered, ref["out"].astype(np.int64))
