"""Multi-GPU runs are replicas: every rank tracks its own streams and only
timings and counts are reduced.  Checked here with two gloo ranks on CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth

    specs = synth.make_stream_mix(8, seed=bench.rank_seed(4, rank))
    local_feats = sum(sp.n_kp for sp in specs)
    local_ms = 10.0 + rank  # rank 1 is the slower one
    tot = bench.reduce_over_ranks(local_feats, "sum", dist)
    slow = bench.reduce_over_ranks(local_ms, "max", dist)
    out[rank] = (local_feats, tot, slow, tuple((sp.w, sp.h, sp.n_kp) for sp in specs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_reduce_only_timings():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        a, b = out[0], out[1]
    assert a[1] == b[1] == a[0] + b[0]  # whole-job features = sum over ranks
    assert a[2] == b[2] == 11.0  # job time = the slowest rank
    assert a[3] != b[3]  # replicas track different streams


def test_single_process_reduction_is_identity():
    import bench

    assert bench.reduce_over_ranks(5.0, "max") == 5.0
    assert bench.reduce_over_ranks(7.0, "sum") == 7.0
    assert bench.rank_seed(4, 0) != bench.rank_seed(4, 1)
