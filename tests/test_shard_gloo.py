"""Multi-rank sharding on CPU (gloo, world size 2): each rank integrates its
own block of cells with no exchange during integration; gathered, the blocks
equal the single-rank result cell by cell."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1309_2710_gb300 import shard, synth  # noqa: E402


def test_shard_cells_cover_and_balance():
    for total, world in ((10, 3), (262144, 8), (5, 8), (0, 2)):
        blocks = [shard.shard_cells(total, world, r) for r in range(world)]
        assert blocks[0][0] == 0 and blocks[-1][1] == total
        assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
        sizes = [b - a for a, b in blocks]
        assert max(sizes) - min(sizes) <= 1
    w = np.r_[np.full(100, 10.0), np.ones(900)]
    blocks = [shard.shard_cells(1000, 2, r, w) for r in range(2)]
    loads = [w[a:b].sum() for a, b in blocks]
    assert abs(loads[0] - loads[1]) <= 10.0 + 1e-9
    assert blocks[0][1] == blocks[1][0]


def test_shard_instances_longest_first():
    parts = shard.shard_instances([100, 60, 50, 40, 10], 2)
    assert sorted(sum(parts, [])) == [0, 1, 2, 3, 4]
    loads = [sum([100, 60, 50, 40, 10][i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= 20


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    name = "h2co_13sp_rkc"
    w = synth.WORKLOADS[name]
    m = synth.workload_mechanism(name)
    T, p, Y = synth.workload_states(name, m, cells=37)
    a, b = shard.shard_cells(37, world, rank)
    Yn, st, _, _ = oracle.integrate(oracle.Mech(m), T[a:b], p[a:b], Y[:, a:b], w["dt"], w["rtol"],
                                    w["atol"], w["method"], nthreads=1)
    # results only meet after integration (no exchange while integrating)
    out = [None] * world
    dist.all_gather_object(out, (a, b, Yn, st))
    if rank == 0:
        q.put(out)
    dist.destroy_process_group()


def test_two_rank_shards_equal_single_rank():
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    name = "h2co_13sp_rkc"
    w = synth.WORKLOADS[name]
    m = synth.workload_mechanism(name)
    T, p, Y = synth.workload_states(name, m, cells=37)
    Yref, st_ref, _, _ = oracle.integrate(oracle.Mech(m), T, p, Y, w["dt"], w["rtol"], w["atol"],
                                          w["method"], nthreads=1)
    got = np.concatenate([o[2] for o in sorted(out, key=lambda o: o[0])], axis=1)
    assert np.array_equal(got, Yref)


def _bench_worker(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    name = "h2co_13sp_rkc"
    m = synth.workload_mechanism(name)
    a, b, T, p, Y = bench.rank_states(name, m, 37, world, rank)
    out = [None] * world
    dist.all_gather_object(out, (a, b, T, Y))
    if rank == 0:
        q.put(out)
    dist.destroy_process_group()


def test_benchmark_ranks_cover_the_job_once_in_order():
    """bench.py's rank blocks under two gloo ranks: the job is 2 x 37 cells
    of one seeded draw; the blocks tile it once, in order, and hold exactly
    the single-rank draw's states."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    out = sorted(out, key=lambda o: o[0])
    assert [(o[0], o[1]) for o in out] == [(0, 37), (37, 74)]
    name = "h2co_13sp_rkc"
    T, p, Y = synth.workload_states(name, synth.workload_mechanism(name), cells=74)
    assert np.array_equal(np.concatenate([o[2] for o in out]), T)
    assert np.array_equal(np.concatenate([o[3] for o in out], axis=1), Y)
