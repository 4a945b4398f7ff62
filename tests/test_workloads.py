"""The seeded synthetic inputs match the recipes the benchmark and the design state (sizes,
vertex-count distributions, placement of points, coordinate boxes) and are reproducible.
CPU only, reduced sizes."""
import numpy as np

from paper_2306_04316_gb300 import workloads as W


def _boxes(w):
    po = w.poly_offsets.astype(np.int64)
    v = w.verts.astype(np.int64)
    return (np.minimum.reduceat(v[:, 0], po[:-1]), np.minimum.reduceat(v[:, 1], po[:-1]),
            np.maximum.reduceat(v[:, 0], po[:-1]), np.maximum.reduceat(v[:, 1], po[:-1]))


def test_generators_are_reproducible():
    a, b = W.footprints(n_polys=2000), W.footprints(n_polys=2000)
    for k in ("points", "poly_offsets", "verts", "cand_offsets", "cand_ids"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    c = W.footprints(seed=W.BASE_SEED + 99, n_polys=2000)
    assert not np.array_equal(a.verts, c.verts)


def test_star_recipe():
    w = W.star()
    assert w.dense and w.n_polys == 1 and w.verts.shape == (1024, 2)
    assert w.n_points == 101_000
    r = np.hypot(w.verts[:, 0].astype(np.float64), w.verts[:, 1].astype(np.float64))
    assert r.min() >= 0.5 * 1e5 - 1 and r.max() <= 1e5 + 1
    ang = np.arctan2(w.verts[:, 1], w.verts[:, 0]) % (2 * np.pi)
    assert (np.diff(ang) > -1e-4).all()                           # angles sorted (up to rounding)
    # at least the 500 points placed on vertices are vertices
    vset = {tuple(p) for p in w.verts.tolist()}
    assert sum(tuple(p) in vset for p in w.points.tolist()) >= 500


def test_footprints_recipe():
    w = W.footprints(n_polys=20_000)
    m = np.diff(w.poly_offsets.astype(np.int64))
    assert m.min() >= 4 and m.max() <= 64
    assert 6.5 < m.mean() < 7.5                                   # lognormal(ln 6, 0.5), rounded, clipped
    co = w.cand_offsets.astype(np.int64)
    assert (np.diff(co) == 16).all()
    assert np.array_equal(w.cand_ids, np.arange(16 * 20_000))      # CSR by construction
    x0, y0, x1, y1 = _boxes(w)
    k = np.repeat(np.arange(20_000), 16)
    px, py = w.points[:, 0].astype(np.int64), w.points[:, 1].astype(np.int64)
    cx, cy = (x0 + x1) / 2, (y0 + y1) / 2
    hw, hh = (x1 - x0) * 0.75 + 1, (y1 - y0) * 0.75 + 1            # 1.5x box (+ rounding)
    assert (np.abs(px - cx[k]) <= hw[k]).all() and (np.abs(py - cy[k]) <= hh[k]).all()
    inside = (px >= x0[k]) & (px <= x1[k]) & (py >= y0[k]) & (py <= y1[k])
    assert 0.35 < inside.mean() < 0.55                             # about 1 / 1.5^2
    assert x0.min() >= W.LON0 and x1.max() <= W.LON1 and y0.min() >= W.LAT0 and y1.max() <= W.LAT1
    side = np.maximum(x1 - x0, y1 - y0) / W.UNITS_PER_M_X
    assert side.max() < 80                                          # sides of 5-50 m, rotated


def test_stress_recipe():
    w = W.stress(n_polys=20_000)
    m = np.diff(w.poly_offsets.astype(np.int64))
    assert m.min() >= 3 and m.max() <= 32
    assert (np.diff(w.cand_offsets.astype(np.int64)) == 8).all()
    x0, y0, x1, y1 = _boxes(w)
    span = np.maximum(x1 - x0, y1 - y0)
    assert span.max() > 2**31                                       # boxes reaching the full range
    assert span.min() < 2**10
    v = w.verts.astype(np.int64)
    assert v.min() == W.I32_MIN or v.max() == W.I32_MAX             # vertices at the int32 limits


def test_join_recipe():
    w = W.join(n_polys=5000, n_points=200_000)
    m = np.diff(w.poly_offsets.astype(np.int64))
    assert m.min() >= 4 and m.max() <= 256
    assert w.cand_offsets is None                                   # the CSR comes from binning
    p = w.points.astype(np.int64)
    assert p[:, 0].min() >= W.LON0 and p[:, 0].max() <= W.LON1
    assert p[:, 1].min() >= W.LAT0 and p[:, 1].max() <= W.LAT1
    # 70 % clustered: cells of about two cluster sigmas hold several points in clusters and
    # almost never in a uniform spread (200,000 points over 1.8M such cells)
    cell = 40_000
    keys = (p[:, 0] // cell) * 10**6 + p[:, 1] // cell
    _, inv, counts = np.unique(keys, return_inverse=True, return_counts=True)
    dense = counts[inv] >= 5
    assert 0.6 < dense.mean() < 0.75


def test_fractal_recipe():
    w = W.fractal(n_polys=4, m_lo=1000, m_hi=3000, n_points=20_000, grid=2)
    m = np.diff(w.poly_offsets.astype(np.int64))
    assert len(m) == 4 and m.min() >= 1000 and m.max() <= 3000
    x0, y0, x1, y1 = _boxes(w)
    # polygons kept inside their own cells of the grid: boxes do not overlap
    for a in range(4):
        for b in range(a + 1, 4):
            assert x1[a] < x0[b] or x1[b] < x0[a] or y1[a] < y0[b] or y1[b] < y0[a]
    # the CSR lists exactly the points in each closed box, ascending
    co = w.cand_offsets.astype(np.int64)
    px, py = w.points[:, 0], w.points[:, 1]
    for k in range(4):
        want = np.nonzero((px >= x0[k]) & (px <= x1[k]) & (py >= y0[k]) & (py <= y1[k]))[0]
        assert np.array_equal(w.cand_ids[co[k]:co[k + 1]], want)


def test_country_recipe():
    w = W.country(m=2000, n_points=50_000)
    assert w.dense and w.n_polys == 1 and w.verts.shape == (2000, 2)
    v = w.verts.astype(np.int64)
    assert v[:, 0].min() >= W.LON0 and v[:, 0].max() <= W.LON1
    assert v[:, 1].min() >= W.LAT0 and v[:, 1].max() <= W.LAT1
    assert W.PAPER_N_POINTS == 17_097_823                            # the paper's point count
