"""GPU parity at the full benchmark sizes, through the same calls and default launch
configuration that bench.py times; every bit is compared with the oracle (0 mismatches).

- footprints (1M polygons, 16M candidates), stress (1M polygons, 8M candidates), star
  (test_gpu_parity.test_star_full), the fractal batch (64 polygons of 1e4-1e6 vertices, 10M
  points, about 8e11 pair tests) and the paper-shaped country batch (17,097,823 points against
  one 100,000-vertex polygon, dense): all bits, both kernels;
- footprints and stress again under every small-polygon kernel shape of the autotuner's grid,
  fractal and country under every edge tile the bench may pick;
- the spatial join (100k polygons against one full 10M-point batch): the GPU candidate lists
  must equal the closed-box lists computed here from the definition on points sorted by x
  (that computation is itself checked against the oracle's brute-force join on 100 polygons),
  and every candidate's bit must equal the oracle's on those lists.
The sampled tests at the end of the file are quick checks of the same batches.
"""
import numpy as np
import pytest

import oracle
from paper_2306_04316_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import api, assert_same, check_full, gpu_bits  # noqa: E402,F401


def test_footprints_full_size(api):
    check_full(api, W.footprints(), "full size")


def test_stress_full_size(api):
    check_full(api, W.stress(), "full size")


@pytest.mark.parametrize("make", [W.footprints, W.stress], ids=["footprints", "stress"])
def test_full_size_every_small_kernel(api, make):
    """Every small-polygon kernel shape the autotuner may pick for the timed step (lockstep,
    compacting, thread per polygon; each slice size and CTA count of its grid) gives the oracle's
    bits on the full footprint and stress batches."""
    from paper_2306_04316_gb300 import tuning
    w = make()
    want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
    before = api.pip_get_small_tuning()
    try:
        for shape in tuning.SMALL_GRID:
            api.pip_set_small_tuning(*shape)
            assert_same(gpu_bits(api, w), want, w.n_bits, f"{w.name} full size small={shape}")
    finally:
        api.pip_set_small_tuning(*before)


@pytest.mark.parametrize("make", [W.fractal, W.country], ids=["fractal", "country"])
def test_large_polygons_full_size(api, make):
    """Every bit of the fractal and country batches, both kernels at the default tuning, and the
    filtered kernel again at every edge tile the bench's autotuner may pick for them (the smaller
    the tile, the more tiles take the exact int32 test instead of the FP32 filter)."""
    w = make()
    want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
    for exact in (False, True):
        assert_same(gpu_bits(api, w, exact), want, w.n_bits, f"{w.name} full size {'exact' if exact else 'filtered'}")
    before = api.pip_get_tuning()
    try:
        for t in ((256, 4, 3), (512, 4, 3), (4096, 4, 2)):
            api.pip_set_tuning(*t)
            assert_same(gpu_bits(api, w), want, w.n_bits, f"{w.name} full size tuning={t}")
    finally:
        api.pip_set_tuning(*before)


def _closed_box_lists(points, poly_offsets, verts):
    """Candidate lists by the closed-box definition (x0 <= p_x <= x1 and y0 <= p_y <= y1, ids
    ascending), evaluated on the points sorted by x: a polygon's x-range is a window of that
    order, whose points are then filtered by y."""
    po = poly_offsets.astype(np.int64)
    v = verts.astype(np.int64)
    m = np.diff(po)
    starts = np.minimum(po[:-1], max(len(v) - 1, 0))
    x0, x1 = np.minimum.reduceat(v[:, 0], starts), np.maximum.reduceat(v[:, 0], starts)
    y0, y1 = np.minimum.reduceat(v[:, 1], starts), np.maximum.reduceat(v[:, 1], starts)
    order = np.argsort(points[:, 0], kind="stable")
    xs, ys = points[order, 0], points[order, 1]
    lo, hi = np.searchsorted(xs, x0, "left"), np.searchsorted(xs, x1, "right")
    lists = []
    for k in range(len(m)):
        if m[k] == 0:
            lists.append(np.zeros(0, dtype=np.int64))
            continue
        yy = ys[lo[k]:hi[k]]
        lists.append(np.sort(order[lo[k]:hi[k]][(yy >= y0[k]) & (yy <= y1[k])]))
    co = np.zeros(len(m) + 1, dtype=np.int64)
    co[1:] = np.cumsum([len(t) for t in lists])
    return co, np.concatenate(lists).astype(np.int64)


def test_join_full_batch(api):
    """One full join batch: 100k polygons, 10M clustered points, binned and classified on the GPU."""
    w = W.join()
    want_co, want_ids = _closed_box_lists(w.points, w.poly_offsets, w.verts)
    # the window computation against the oracle's brute-force join, on 100 polygons
    polys = np.sort(np.random.default_rng(2306043160 + 80).choice(w.n_polys, 100, replace=False))
    counts, ids_o = oracle.bbox_join(w.points, w.poly_offsets, w.verts, polys)
    assert np.array_equal(counts, want_co[polys + 1] - want_co[polys])
    assert np.array_equal(ids_o, np.concatenate([want_ids[want_co[k]:want_co[k + 1]] for k in polys]))
    d = api.to_device(w)
    co, ids = api.bin_join(d["points"], d["poly_offsets"], d["verts"])
    n_c = int(co[-1].item())
    out = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], co, ids, n_cands=n_c)
    torch.cuda.synchronize()
    assert np.array_equal(co.cpu().numpy().astype(np.int64), want_co), "candidate offsets"
    assert np.array_equal(ids.cpu().numpy()[:n_c].astype(np.int64), want_ids), "candidate ids"
    want = oracle.classify(w.points, w.poly_offsets, w.verts, want_co, want_ids)
    assert_same(out.cpu().numpy().view(np.uint32)[:len(want)], want, n_c, "join full batch")


def test_fractal_full_size_sampled(api):
    w = W.fractal()
    rng = np.random.default_rng(2306043160 + 77)
    sample = np.unique(rng.integers(0, w.n_bits, 3000))
    want = oracle.classify_sample(w.points, w.poly_offsets, w.verts, sample, w.cand_offsets, w.cand_ids)
    for exact in (False, True):
        got = oracle.unpack_bits(gpu_bits(api, w, exact), w.n_bits)[sample]
        bad = np.nonzero(got != want)[0]
        assert len(bad) == 0, f"{'exact' if exact else 'filtered'}: {len(bad)} of {len(sample)} sampled bits differ"


def test_join_full_size_sampled(api):
    w = W.join()
    d = api.to_device(w)
    co, ids = api.bin_join(d["points"], d["poly_offsets"], d["verts"])
    n_c = int(co[-1].item())
    out = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], co, ids, n_cands=n_c)
    torch.cuda.synchronize()
    co, ids = co.cpu().numpy().astype(np.int64), ids.cpu().numpy()
    bits = oracle.unpack_bits(out.cpu().numpy().view(np.uint32), n_c)
    rng = np.random.default_rng(2306043160 + 78)
    polys = np.sort(rng.choice(w.n_polys, 300, replace=False))
    counts, want_ids = oracle.bbox_join(w.points, w.poly_offsets, w.verts, polys)
    # the sampled polygons alone, with the oracle's own candidate lists
    po = w.poly_offsets.astype(np.int64)
    sub_po = np.zeros(len(polys) + 1, dtype=np.int64)
    sub_po[1:] = np.cumsum(po[polys + 1] - po[polys])
    sub_v = np.concatenate([w.verts[po[k]:po[k + 1]] for k in polys])
    sub_co = np.zeros(len(polys) + 1, dtype=np.int64)
    sub_co[1:] = np.cumsum(counts)
    want_bits = oracle.unpack_bits(
        oracle.classify(w.points, sub_po, sub_v, sub_co, want_ids.astype(np.int64)), int(sub_co[-1]))
    for i, k in enumerate(polys):
        seg = slice(co[k], co[k + 1])
        order = np.argsort(ids[seg], kind="stable")
        assert np.array_equal(ids[seg][order], want_ids[sub_co[i]:sub_co[i + 1]]), f"candidates of polygon {k}"
        assert np.array_equal(bits[seg][order], want_bits[sub_co[i]:sub_co[i + 1]]), f"bits of polygon {k}"


def test_country_full_size_sampled(api):
    """The paper-shaped batch: 17,097,823 building-like points against one 100,000-vertex
    country-like polygon (dense mode), checked on 3,000 sampled points."""
    w = W.country()
    rng = np.random.default_rng(2306043160 + 79)
    sample = np.unique(rng.integers(0, w.n_points, 3000))
    want = oracle.classify_sample(w.points, w.poly_offsets, w.verts, sample)
    got = oracle.unpack_bits(gpu_bits(api, w), w.n_bits)[sample]
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, f"{len(bad)} of {len(sample)} sampled bits differ"
