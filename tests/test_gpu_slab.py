"""GPU parity of the y-slab edge index (pip_slab_build + pip_classify_slab) against the oracle.

The index changes which edges a point tests, never its answer, so every case below requires
the same bits as the oracle's full ray casting: fractal and star polygons, the paper-shaped
country batch (sampled), polygons whose tall edges span many slabs (comb teeth), full-range
coordinates, points on slab boundaries and outside the polygons' y-range, an index too small
to hold its entries (ignored), and small polygons mixed in (which never get slabs).
"""
import numpy as np
import pytest

import oracle
from paper_2306_04316_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import _concat, _star_polygon, api, assert_same, make  # noqa: E402,F401


def slab_bits(api, w, edges_per_slab=8, index=None):
    d = api.to_device(w)
    if index is None:
        index = api.slab_index(d["poly_offsets"], d["verts"], edges_per_slab)
    out = api.pip_classify_slab(d["points"], d["poly_offsets"], d["verts"], d.get("cand_offsets"),
                                d.get("cand_ids"), index=index, n_cands=None if w.dense else w.n_bits)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)[:w.n_words]


def check(api, w, what="", **kw):
    want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
    assert_same(slab_bits(api, w, **kw), want, w.n_bits, f"{w.name} {what} (slab index)")


@pytest.mark.parametrize("eps", [1, 8, 64])
def test_fractal_and_star(api, eps):
    check(api, W.fractal(seed=61, n_polys=6, m_lo=2_000, m_hi=30_000, n_points=100_000, cell=300_000, grid=3),
          f"edges_per_slab={eps}", edges_per_slab=eps)
    check(api, W.star(), f"edges_per_slab={eps}", edges_per_slab=eps)


def test_country_sampled(api):
    w = W.country()
    rng = np.random.default_rng(2306043160 + 83)
    sample = np.unique(rng.integers(0, w.n_points, 3000))
    want = oracle.classify_sample(w.points, w.poly_offsets, w.verts, sample)
    got = oracle.unpack_bits(slab_bits(api, w), w.n_bits)[sample]
    assert np.array_equal(got, want), f"{int((got != want).sum())} sampled bits differ"


def test_tall_edges_and_slab_boundaries(api):
    """A comb: long vertical teeth (tall edges in every polygon's tall list) joined by short
    steps; points on every slab boundary row, on the teeth, and above and below the comb."""
    rng = np.random.default_rng(2306043160 + 84)
    polys = []
    for c in range(3):
        teeth = 150 + 50 * c
        x = 0
        top = []
        for t in range(teeth):
            top += [(x, 0), (x, 10_000 + 7 * t), (x + 3, 10_000 + 7 * t), (x + 3, 0)]
            x += 5
        v = top + [(x, -500), (0, -500)]
        polys.append([(px + 100_000 * c, py) for px, py in v])
    ys = list(range(-600, 12_000, 37))
    pts = [(int(rng.integers(-10, 100_000 * 3)), y) for y in ys for _ in range(20)]
    # every row of the first comb's y-range (so every slab boundary) at a few columns
    pts += [(x, y) for x in (1, 3, 4, 9, 747) for y in range(-510, 11_060)]
    pts += [(v[0], v[1]) for p in polys for v in p[::7]]
    check(api, make("comb", polys, pts), "dense")
    ids = list(range(len(pts)))
    check(api, make("comb-csr", polys, pts, [ids, ids[::2], ids[1::3]]), "csr")


def test_full_range_polygons(api):
    rng = np.random.default_rng(2306043160 + 85)
    polys = [_star_polygon(rng, 3000, 2.0**31), _star_polygon(rng, 600, 2.0**29.95)]
    pts = [rng.integers(-2**31, 2**31, (4000, 2))]
    for v in polys:
        pts.append(v[rng.integers(0, len(v), 300)])
    lo, hi = -2**31, 2**31 - 1
    pts.append(np.array([(lo, lo), (hi, hi), (lo, hi), (hi, lo), (0, 0), (hi, 0), (0, lo)]))
    check(api, make("slab-full-range", [v.tolist() for v in polys], np.concatenate(pts).tolist()))


def test_index_too_small_is_ignored(api):
    w = W.fractal(seed=62, n_polys=4, m_lo=2_000, m_hi=8_000, n_points=40_000, cell=200_000, grid=2)
    d = api.to_device(w)
    lib = api._lib.load()
    n_polys, n_verts = w.n_polys, int(w.verts.shape[0])
    nbytes = int(lib.pip_slab_index_bytes(n_polys, n_verts, 8, 0))
    index = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    need = torch.zeros(1, dtype=torch.int64, device="cuda")
    api._lib.check("pip_slab_build", lib.pip_slab_build(api._ptr(d["poly_offsets"]), api._ptr(d["verts"]), n_polys,
                                                         n_verts, 8, api._ptr(index), nbytes, api._ptr(need),
                                                         api._stream(None)))
    torch.cuda.synchronize()
    assert int(need.item()) > 0
    check(api, w, "unusable index", index=index)


def test_small_polygons_mixed_in(api):
    parts = []
    for i in range(4):
        parts.append(W.footprints(seed=300 + i, n_polys=41 + 9 * i, pts_per_poly=5 + i))
        parts.append(W.fractal(seed=310 + i, n_polys=1, m_lo=300 + 900 * i, m_hi=301 + 900 * i,
                               n_points=900 + 77 * i, cell=100_000, grid=1))
    check(api, _concat(parts, "mixed"))
