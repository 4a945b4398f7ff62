"""The multi-GPU path of bench.py (weak scaling, one process per GPU) on CPU with gloo ranks.

Each rank classifies its own batch (seed + rank) and no collective touches the data path;
the only collectives are the barrier and the max over ranks of the timed region.  These tests
run that host-side logic with two gloo ranks on 127.0.0.1: every rank gets the slowest rank's
time, the per-rank batches have equal sizes but different data, and the whole-job value counts
the units of all ranks.
"""
import argparse
import os
import socket
import zlib

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist = bench.dist_setup(world, backend="gloo")
    try:
        t = bench.max_over_ranks(dist, 1.0 + 2.5 * rank, device="cpu")
        w = bench.make_workload("footprints", rank, 0.0005)
        total = bench.sum_over_ranks(dist, w.pair_tests(), device="cpu")
        sizes = torch.tensor([w.n_polys, w.n_candidates, w.pair_tests()], dtype=torch.float64)
        gathered = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, sizes)
        dist.barrier()
        q.put((rank, t, [g.tolist() for g in gathered], zlib.crc32(w.points.tobytes()), total))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    times = [r[1] for r in res]
    assert times == [3.5, 3.5]                         # every rank sees the slowest rank's time
    sizes = res[0][2]
    assert sizes[0][:2] == sizes[1][:2]                # same polygons and candidates per rank (weak scaling)
    assert res[0][3] != res[1][3]                      # ... but each rank's own data
    pairs = sizes[0][2] + sizes[1][2]
    assert res[0][4] == res[1][4] == pairs             # the job counts every rank's pair tests
    assert bench.job_rate(pairs, 2.0) == pytest.approx(pairs / 0.002)


def test_single_rank_has_no_collective():
    assert bench.dist_setup(1) is None
    assert bench.max_over_ranks(None, 4.25) == 4.25


def test_reference_arm_other_ranks_exit_without_work():
    args = argparse.Namespace(workload="footprints", steps=1, warmup=1)
    assert bench.run_reference(args, rank=1, world=2) == 0
