"""Sharding of one classification across ranks (paper_2306_04316_gb300.shard), on CPU.

The partitions are checked against the oracle: the polygon ranges cover every polygon once and
balance the pair tests; the edge pieces closed through R_0 give, XORed, exactly the polygon's
bits, boundary points included.  Two gloo ranks then run the combine steps: each rank's
partial bits come from the oracle on that rank's shard (the test is the checker), and the
combined bits must equal the oracle's bits for the whole batch.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2306_04316_gb300 import shard, workloads as W

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _csr_case():
    w = W.footprints(seed=91, n_polys=3000, pts_per_poly=9)
    return w


def _edge_case():
    """Star and self-intersecting polygons with lattice points, many on edges and vertices."""
    rng = np.random.default_rng(92)
    polys = []
    for k in range(12):
        m = int(rng.integers(3, 40))
        if k % 3 == 0:   # self-intersecting: random lattice vertices
            polys.append(rng.integers(0, 24, (m, 2)))
        else:
            ang = np.sort(rng.uniform(0, 2 * np.pi, m))
            r = rng.uniform(4, 11, m)
            polys.append(np.stack([12 + np.rint(r * np.cos(ang)), 12 + np.rint(r * np.sin(ang))], 1))
    po = np.zeros(len(polys) + 1, dtype=np.int64)
    po[1:] = np.cumsum([len(p) for p in polys])
    verts = np.concatenate(polys).astype(np.int32)
    xs, ys = np.meshgrid(np.arange(-1, 26), np.arange(-1, 26))
    pts = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    return pts, po.astype(np.int32), verts


def test_polygon_ranges_cover_and_balance():
    w = _csr_case()
    wt = shard.pair_weights(w.poly_offsets, w.cand_offsets)
    for world in (1, 2, 3, 5, 8):
        b = shard.polygon_ranges(w.poly_offsets, w.cand_offsets, world)
        assert b[0] == 0 and b[-1] == w.n_polys and np.all(np.diff(b) >= 0)
        loads = np.array([wt[b[r]:b[r + 1]].sum() for r in range(world)])
        assert loads.sum() == wt.sum()
        assert loads.max() <= wt.sum() / world + wt.max()   # a contiguous cut is off by < one polygon


def test_polygon_ranges_degenerate():
    po = np.array([0, 3, 3, 7], dtype=np.int32)
    co = np.array([0, 0, 0, 0], dtype=np.int32)   # no candidates at all
    b = shard.polygon_ranges(po, co, 4)
    assert b[0] == 0 and b[-1] == 3 and np.all(np.diff(b) >= 0)


def test_edge_pieces_xor_is_the_polygon():
    pts, po, verts = _edge_case()
    n_bits = (len(po) - 1) * 32 * ((len(pts) + 31) // 32)
    want = oracle.unpack_bits(oracle.classify(pts, po, verts), n_bits)
    for world in (1, 2, 3, 7):
        acc = np.zeros_like(want)
        pieces = shard.edge_pieces(po, verts, world)
        assert len(pieces) == world
        for ppo, pv in pieces:
            acc ^= oracle.unpack_bits(oracle.classify(pts, ppo, pv), len(want))
        assert np.array_equal(acc, want), f"world={world}"


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo")
    try:
        # polygon partition: this rank's range, its bits at their global positions, SUM all-reduce
        w = _csr_case()
        b = shard.polygon_ranges(w.poly_offsets, w.cand_offsets, world)
        p0, p1, po_v, co_v = shard.rank_views(b, rank, w.poly_offsets, w.cand_offsets)
        mine = oracle.classify(w.points, po_v, w.verts, co_v, w.cand_ids)      # absolute offsets
        words = np.zeros(w.n_words, dtype=np.uint32)
        words[:len(mine)] = mine
        t = torch.from_numpy(words.view(np.int32).copy())
        shard.combine_disjoint(t, dist)
        poly_bits = t.numpy().view(np.uint32).copy()
        # edge partition: this rank's pieces of every polygon, all-gather and XOR
        pts, po, verts = _edge_case()
        ppo, pv = shard.edge_pieces(po, verts, world)[rank]
        part = torch.from_numpy(oracle.classify(pts, ppo, pv).view(np.int32).copy())

        def xor_cpu(dst, src):
            dst.bitwise_xor_(src)
        shard.combine_xor(part, dist, xor_into=xor_cpu)
        q.put((rank, poly_bits, part.numpy().view(np.uint32).copy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_the_whole():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = _csr_case()
    want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
    pts, po, verts = _edge_case()
    want_e = oracle.classify(pts, po, verts)
    for rank, poly_bits, edge_bits in res:
        assert np.array_equal(poly_bits, want), f"rank {rank}: polygon partition"
        assert np.array_equal(edge_bits, want_e), f"rank {rank}: edge partition"
