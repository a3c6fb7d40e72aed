"""The multi-GPU path of bench.py is replicas only: one independent job per rank, a barrier,
and two scalar reductions (max of the ranks' times, sum of their units). Checked here with
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    w, r, local, pg = bench.dist_setup(backend="gloo")
    try:
        bench.barrier(pg)
        # rank r processed (r + 1) * 1000 units in (r + 1) * 0.5 s
        value, total, t_max = bench.aggregate(pg, (r + 1) * 1000.0, (r + 1) * 0.5)
        make, _ = bench.workloads()["disks128"]
        wl = make(r)
        out[r] = (w, r, value, total, t_max, float(wl.image.sum()))
    finally:
        pg.destroy_process_group()


def test_two_gloo_replicas_aggregate_and_differ():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        w, rr, value, total, t_max, _ = res[r]
        assert (w, rr) == (2, r)
        assert total == 3000.0 and t_max == 1.0 and value == 3000.0   # sum of units / slowest rank
    # each rank runs its own independently seeded job
    assert res[0][5] != res[1][5]


def test_single_process_needs_no_group():
    assert bench.dist_setup() == (1, 0, 0, None)
    assert bench.aggregate(None, 10.0, 2.0) == (5.0, 10.0, 2.0)
