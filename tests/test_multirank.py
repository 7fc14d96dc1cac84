"""The N>1 bench path on CPU: two gloo ranks.

The transform shards by instance: every rank evaluates its own seeded
instance (N*M terms) with no collective on the data path, and the job's step
time is the maximum over ranks.  Checked here with world_size 2 on gloo:
* the ranks' inputs differ and are reproducible from the rank alone;
* max_over_ranks returns the slowest rank's time on every rank;
* job_value counts the units of all ranks;
* the oracle's result for a rank's shard depends only on that shard;
* the reference arm runs on rank 0 only (the other ranks return at once).
"""
import argparse
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N = 64
    c, w = bench.rank_workload(N, rank)
    c2, w2 = bench.rank_workload(N, rank)
    assert np.array_equal(c, c2) and np.array_equal(w, w2)
    shards = [None] * world
    dist.all_gather_object(shards, (c, w))
    for r in range(world):
        if r != rank:
            assert not np.array_equal(shards[r][0], c)
            assert not np.array_equal(shards[r][1], w)
    # each rank's step time differs; every rank sees the maximum
    ms = 1.0 + 0.5 * rank
    job_ms = bench.max_over_ranks(ms, dist, "cpu")
    assert job_ms == 1.0 + 0.5 * (world - 1)
    assert bench.job_value(world, N, N, job_ms) == pytest.approx(world * N * N / (job_ms * 1e-3))
    # the shard's result is a function of the shard alone
    f = oracle.flt_direct(c.astype(np.complex128), w[:8], threads=1)
    all_f = [None] * world
    dist.all_gather_object(all_f, f)
    for r in range(world):
        fr = oracle.flt_direct(shards[r][0].astype(np.complex128), shards[r][1][:8], threads=1)
        assert np.array_equal(fr, all_f[r])
    # reference arm: only rank 0 works; here every rank > 0 must return 0 at once
    if rank > 0:
        args = argparse.Namespace(N=N, steps=1, warmup=0)
        assert bench.run_reference(args) == 0
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"ok{rank}"), "w") as fh:
        fh.write("ok")


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        assert (tmp_path / f"ok{r}").read_text() == "ok"
