"""Sharding of one classification across ranks (one process per GPU; not part of the paper).

The paper's only parallel axis is the points of one polygon (Algorithm 4 runs them in a
``prange``).  Across GPUs the work units are (polygon, candidate) pairs, and there are two ways
to split them, both host-side bookkeeping around the unchanged ``pip_classify`` call:

* by polygon (``polygon_ranges``): contiguous polygon ranges balanced by their pair tests
  (sum over the range of vertices x candidates).  A rank classifies its range with views of the
  global arrays (``poly_offsets[p0:p1+1]``, ``cand_offsets[p0:p1+1]``): candidate offsets are
  absolute, so its bits land at their global positions of a zeroed full-size output.  The
  ranks' bits are disjoint, so an integer SUM all-reduce of the words is their OR
  (``combine_disjoint``).
* by edge (``edge_pieces``): each polygon's edge chain is cut into one piece per rank, and each
  piece is closed through the polygon's first vertex R_0 (vertices R_0, R_a, ..., R_b).  Every
  added chord R_0 -> R_a is also the closing edge, reversed, of the previous piece, and an edge's
  crossing test does not depend on its direction, so each chord is counted twice and cancels:
  the XOR of the pieces' parities is the polygon's parity, bit for bit (boundary points
  included).  Every rank classifies all candidates against its pieces; NCCL has no XOR, so
  ``combine_xor`` all-gathers the ranks' words and XORs them locally.

The functions take numpy arrays (the partition is computed once per polygon set on the host)
and torch tensors for the combine step, with ``dist`` a ``torch.distributed`` module or None for
one rank.
"""
from __future__ import annotations

import numpy as np


def pair_weights(poly_offsets, cand_offsets):
    """Pair tests per polygon: vertices x candidates (int64)."""
    m = np.diff(np.asarray(poly_offsets, dtype=np.int64))
    n = np.diff(np.asarray(cand_offsets, dtype=np.int64))
    return m * n


def polygon_ranges(poly_offsets, cand_offsets, world: int) -> np.ndarray:
    """Boundaries p_0 = 0 <= p_1 <= ... <= p_world = P of contiguous polygon ranges whose pair
    tests are as equal as a contiguous cut allows: rank r takes polygons [p_r, p_{r+1}).  The cut
    for rank r is the first polygon at which the running total reaches r/world of the whole
    (one polygon more than the total can never be split by this partition)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = pair_weights(poly_offsets, cand_offsets)
    P = len(w)
    cum = np.concatenate([[0], np.cumsum(w)])
    total = int(cum[-1])
    b = np.zeros(world + 1, dtype=np.int64)
    b[-1] = P
    for r in range(1, world):
        # first boundary index whose prefix reaches the target share
        b[r] = int(np.searchsorted(cum, total * r / world, side="left"))
    b = np.maximum.accumulate(np.clip(b, 0, P))
    return b


def rank_views(bounds, rank: int, poly_offsets, cand_offsets):
    """(p0, p1, poly_offsets view, cand_offsets view) of one rank's range; both views have
    p1 - p0 + 1 entries and keep absolute values (vertex and candidate indices of the global
    arrays)."""
    p0, p1 = int(bounds[rank]), int(bounds[rank + 1])
    return p0, p1, poly_offsets[p0:p1 + 1], cand_offsets[p0:p1 + 1]


def edge_pieces(poly_offsets, verts, world: int):
    """Per rank, a polygon set whose k-th polygon is the rank's piece of polygon k: the chain of
    edges [a, b) of polygon k (m vertices, edge i from R_i to R_{i+1 mod m}) closed through R_0,
    i.e. the vertices R_0, R_a, ..., R_b (R_m read as R_0).  Rank r takes edges
    [floor(r m / world), floor((r + 1) m / world)); a rank whose chain is empty gets an empty
    polygon (no vertices).  Returns a list of (poly_offsets, verts) numpy pairs, int32."""
    po = np.asarray(poly_offsets, dtype=np.int64)
    v = np.asarray(verts)
    m = np.diff(po)
    out = []
    for r in range(world):
        a = (r * m) // world
        b = ((r + 1) * m) // world
        take = []
        sizes = np.zeros(len(m), dtype=np.int64)
        for k in range(len(m)):
            if b[k] <= a[k]:
                continue
            idx = np.arange(a[k], b[k] + 1) % m[k] + po[k]   # R_a .. R_b (R_m = R_0)
            if a[k] != 0:
                idx = np.concatenate([[po[k]], idx])          # closed through R_0
            take.append(idx)
            sizes[k] = len(idx)
        offs = np.zeros(len(m) + 1, dtype=np.int64)
        offs[1:] = np.cumsum(sizes)
        vv = v[np.concatenate(take)] if take else v[:0]
        out.append((offs.astype(np.int32), np.ascontiguousarray(vv, dtype=np.int32)))
    return out


def combine_disjoint(words, dist=None):
    """OR of the ranks' output words when every bit is set by at most one rank (polygon
    partition): an integer SUM all-reduce, which never carries because the bits are disjoint.
    ``words`` (int32 tensor, full output size) is reduced in place and returned."""
    if dist is not None and dist.get_world_size() > 1:
        dist.all_reduce(words, op=dist.ReduceOp.SUM)
    return words


def combine_xor(words, dist=None, xor_into=None):
    """XOR of the ranks' output words (edge partition): all-gather, then a local XOR of the
    gathered parts into this rank's words by ``xor_into(dst, src)`` (default: the library's
    ``pip_xor_words`` kernel, which needs CUDA tensors).  Returns ``words``, combined in place."""
    if dist is None or dist.get_world_size() <= 1:
        return words
    import torch
    if xor_into is None:
        from . import api
        xor_into = api.pip_xor_words
    parts = [torch.empty_like(words) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, words)
    me = dist.get_rank()
    for r, p in enumerate(parts):
        if r != me:
            xor_into(words, p)
    return words
