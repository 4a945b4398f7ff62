"""Seeded synthetic workloads (numpy only; none of the point-in-polygon arithmetic).

Shared by the tests, the benchmark and the oracle checks.  Coordinates are int32
fixed point in 1e-7 degree units.  The paper's own data (Google Open Buildings points
for Ghana against the GADM Ghana polygon, Simulation section) is not available, so
these generators stand in for it with the shapes, sizes and distributions of the six
workloads listed in ``WORKLOADS``:

1. ``star``        one 1,024-vertex star polygon, R = 1e5 units; 100,000 uniform points in
                   its bbox plus 1% placed exactly on vertices and on lattice points of edges;
                   dense mode (every point against the polygon).
2. ``footprints``  1M building-footprint polygons (rotated rectangles and L-shapes with
                   extra jittered edge vertices, 4-64 vertices, log-normal counts) in Ghana's
                   lon/lat box; 16 points per polygon uniform in its 1.5x bbox; CSR by
                   construction.
3. ``join``        100k footprints of 4-256 vertices and 10M points, 70% of both drawn from
                   1,000 Gaussian clusters (sigma 200 m); the CSR comes from the GPU binning
                   pass (or the oracle's closed-bbox join in tests).
4. ``fractal``     64 midpoint-displacement polygons (Hurst 0.7) of 1e4-1e6 vertices on an
                   8x8 grid of cells and 10M uniform points; CSR = closed-bbox candidates.
5. ``stress``      1M polygons of 3-32 vertices spanning the whole int32 range (needle
                   triangles, collinear runs, random stars), 8 points per polygon, half of
                   them placed on or within 1-3 units of the boundary.
6. ``country``     the paper's experiment in shape: 17,097,823 building-like points (70% in
                   1,000 settlements) against one 100,000-vertex fractal country-like polygon
                   spanning the box; dense mode.

Seeds: ``seed_k = 2306043160 + k`` (numpy PCG64) unless a test passes its own.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

I32_MIN = -2**31
I32_MAX = 2**31 - 1
BASE_SEED = 2306043160

# Ghana's approximate bounding box (lon -3.3..1.2 deg, lat 4.7..11.2 deg) in 1e-7 deg units
LON0, LON1 = -33_000_000, 12_000_000
LAT0, LAT1 = 47_000_000, 112_000_000
UNITS_PER_M_X = 90.7   # 1 m in lon units at 8 deg N
UNITS_PER_M_Y = 89.8   # 1 m in lat units


@dataclasses.dataclass
class Workload:
    name: str
    points: np.ndarray                 # int32 [N, 2]
    poly_offsets: np.ndarray           # int32 [P + 1]
    verts: np.ndarray                  # int32 [V, 2]
    cand_offsets: Optional[np.ndarray] = None   # int32 [P + 1] or None (dense)
    cand_ids: Optional[np.ndarray] = None       # int32 [C] or None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return int(self.points.shape[0])

    @property
    def n_polys(self) -> int:
        return int(self.poly_offsets.shape[0] - 1)

    @property
    def dense(self) -> bool:
        return self.cand_offsets is None

    @property
    def n_bits(self) -> int:
        if self.dense:
            return self.n_polys * 32 * ((self.n_points + 31) // 32)
        return int(self.cand_offsets[-1])

    @property
    def n_words(self) -> int:
        if self.dense:
            return self.n_polys * ((self.n_points + 31) // 32)
        return (self.n_bits + 31) // 32

    @property
    def n_candidates(self) -> int:
        return self.n_polys * self.n_points if self.dense else self.n_bits

    def pair_tests(self) -> int:
        """T = sum over candidates of the vertex count of the candidate's polygon."""
        m = np.diff(self.poly_offsets.astype(np.int64))
        if self.dense:
            return int(m.sum()) * self.n_points
        n = np.diff(self.cand_offsets.astype(np.int64))
        return int((m * n).sum())

    def algorithmic_bytes(self) -> int:
        """Bytes the classify pass must move at least once: vertices, offsets, the gathered
        point per candidate, candidate ids and the output bits."""
        V = int(self.verts.shape[0])
        P = self.n_polys
        if self.dense:
            return 8 * V + 4 * (P + 1) + 8 * self.n_points * P + self.n_words * 4
        C = self.n_bits
        return 8 * V + 8 * (P + 1) + 12 * C + self.n_words * 4

    def prefix(self, n_polys: int) -> "Workload":
        """The first n_polys polygons with their candidates (CSR mode; points kept whole)."""
        n = max(0, min(int(n_polys), self.n_polys))
        po = self.poly_offsets[:n + 1]
        v = self.verts[:int(po[-1])] if n else self.verts[:0]
        if self.dense:
            return dataclasses.replace(self, poly_offsets=po, verts=v)
        co = self.cand_offsets[:n + 1]
        return dataclasses.replace(self, poly_offsets=po, verts=v, cand_offsets=co,
                                   cand_ids=self.cand_ids[:int(co[-1])] if n else self.cand_ids[:0])

    def bounded(self, max_pairs: float) -> "Workload":
        """A leading part of the batch with at most about max_pairs pair tests (at least one
        polygon or point): the first polygons (CSR), or the first points (dense)."""
        T = self.pair_tests()
        if T <= max_pairs:
            return self
        if self.dense:
            n = max(1, int(self.n_points * max_pairs / T))
            return dataclasses.replace(self, points=self.points[:n])
        return self.prefix(max(1, int(self.n_polys * max_pairs / T)))

    def with_csr(self, cand_offsets, cand_ids, name=None):
        return dataclasses.replace(self, name=name or self.name,
                                   cand_offsets=np.ascontiguousarray(cand_offsets, dtype=np.int32),
                                   cand_ids=np.ascontiguousarray(cand_ids, dtype=np.int32))


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _clip32(a):
    return np.clip(np.rint(a), I32_MIN, I32_MAX).astype(np.int64)


def _offsets(counts):
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


def _bboxes(poly_offsets, verts):
    """Per polygon (xmin, ymin, xmax, ymax) for polygons with >= 1 vertex (int64)."""
    starts = poly_offsets[:-1]
    x, y = verts[:, 0].astype(np.int64), verts[:, 1].astype(np.int64)
    return (np.minimum.reduceat(x, starts), np.minimum.reduceat(y, starts),
            np.maximum.reduceat(x, starts), np.maximum.reduceat(y, starts))


# ---------------------------------------------------------------------------------------------
# 1. single star polygon, dense mode
# ---------------------------------------------------------------------------------------------

def star(seed=BASE_SEED + 1, m=1024, R=100_000, n_uniform=100_000, n_special=1_000) -> Workload:
    rng = _rng(seed)
    ang = np.sort(rng.uniform(0.0, 2 * np.pi, m))
    rad = rng.uniform(0.5, 1.0, m) * R
    v = np.stack([np.rint(rad * np.cos(ang)), np.rint(rad * np.sin(ang))], 1).astype(np.int64)
    x0, y0 = v.min(0)
    x1, y1 = v.max(0)
    uni = np.stack([rng.integers(x0, x1, n_uniform, endpoint=True),
                    rng.integers(y0, y1, n_uniform, endpoint=True)], 1)
    n_vert = n_special // 2
    n_edge = n_special - n_vert
    on_vert = v[rng.integers(0, m, n_vert)]
    # lattice points strictly inside edges (where gcd(|dx|, |dy|) > 1), else a vertex
    e = rng.integers(0, m, n_edge)
    a, b = v[e], v[(e + 1) % m]
    d = b - a
    g = np.gcd(np.abs(d[:, 0]), np.abs(d[:, 1]))
    k = np.where(g > 1, 1 + (rng.integers(0, 2**62, n_edge) % np.maximum(g - 1, 1)), 0)
    step = d // np.maximum(g, 1)[:, None]
    on_edge = a + step * k[:, None]
    pts = np.concatenate([uni, on_vert, on_edge])
    pts = pts[rng.permutation(len(pts))]
    return Workload("star", pts.astype(np.int32), np.array([0, m], dtype=np.int32),
                    v.astype(np.int32), meta=dict(seed=seed, m=m, R=R, n_special=n_special,
                                                  edge_lattice=int((g > 1).sum())))


# ---------------------------------------------------------------------------------------------
# footprint shapes (rotated rectangles and L-shapes with jittered extra edge vertices)
# ---------------------------------------------------------------------------------------------

def _footprint_shapes(rng, m_arr, centres_xy):
    """Vertices (in units) of footprint polygons with the given vertex counts and centres.

    m == 4 -> rotated rectangle; m == 6 -> L-shape; other m -> rectangle (or L for m >= 6,
    half the time) with m - base extra vertices on its edges, jittered by <= 0.1 m.  Sides
    U[5, 50] m, rotation U[0, pi), every vertex jittered by up to +-0.3 m."""
    n = len(m_arr)
    use_l = (m_arr == 6) | ((m_arr > 6) & (rng.random(n) < 0.5))
    offs = _offsets(m_arr)
    out = np.zeros((int(offs[-1]), 2), dtype=np.int64)
    a = rng.uniform(5.0, 50.0, n)
    b = rng.uniform(5.0, 50.0, n)
    a1 = rng.uniform(0.3, 0.7, n)
    b1 = rng.uniform(0.3, 0.7, n)
    theta = rng.uniform(0.0, np.pi, n)
    for m in np.unique(m_arr):
        for lshape in (False, True):
            sel = np.nonzero((m_arr == m) & (use_l == lshape))[0]
            if len(sel) == 0:
                continue
            A, B = a[sel], b[sel]
            if lshape:
                base = np.stack([
                    np.stack([np.zeros_like(A), np.zeros_like(A)], 1),
                    np.stack([A, np.zeros_like(A)], 1),
                    np.stack([A, B * b1[sel]], 1),
                    np.stack([A * a1[sel], B * b1[sel]], 1),
                    np.stack([A * a1[sel], B], 1),
                    np.stack([np.zeros_like(A), B], 1)], 1)
            else:
                base = np.stack([
                    np.stack([np.zeros_like(A), np.zeros_like(A)], 1),
                    np.stack([A, np.zeros_like(A)], 1),
                    np.stack([A, B], 1),
                    np.stack([np.zeros_like(A), B], 1)], 1)
            base = base - np.stack([A / 2, B / 2], 1)[:, None, :]
            nb = base.shape[1]
            extra = int(m) - nb
            if extra > 0:
                ekey = rng.integers(0, nb, (len(sel), extra)) + rng.uniform(0.05, 0.95, (len(sel), extra))
                keys = np.concatenate([np.broadcast_to(np.arange(nb, dtype=np.float64), (len(sel), nb)), ekey], 1)
                order = np.argsort(keys, axis=1, kind="stable")
                keys = np.take_along_axis(keys, order, 1)
                j = np.floor(keys).astype(np.int64)
                t = keys - j
                p0 = np.take_along_axis(base, j[:, :, None].repeat(2, 2), 1)
                p1 = np.take_along_axis(base, ((j + 1) % nb)[:, :, None].repeat(2, 2), 1)
                shape = p0 + (p1 - p0) * t[:, :, None]
                is_extra = t > 0
                shape = shape + is_extra[:, :, None] * rng.uniform(-0.1, 0.1, shape.shape)
            else:
                shape = base
            shape = shape + rng.uniform(-0.3, 0.3, shape.shape)
            c, s = np.cos(theta[sel]), np.sin(theta[sel])
            xr = shape[:, :, 0] * c[:, None] - shape[:, :, 1] * s[:, None]
            yr = shape[:, :, 0] * s[:, None] + shape[:, :, 1] * c[:, None]
            X = centres_xy[sel, 0][:, None] + xr * UNITS_PER_M_X
            Y = centres_xy[sel, 1][:, None] + yr * UNITS_PER_M_Y
            idx = offs[sel][:, None] + np.arange(int(m))[None, :]
            out[idx.ravel(), 0] = _clip32(X).ravel()
            out[idx.ravel(), 1] = _clip32(Y).ravel()
    return offs, out


def _points_in_bboxes(rng, poly_offsets, verts, per_poly, grow=1.5):
    x0, y0, x1, y1 = _bboxes(poly_offsets, verts)
    cx, cy = (x0 + x1) / 2.0, (y0 + y1) / 2.0
    hx, hy = (x1 - x0) * grow / 2.0, (y1 - y0) * grow / 2.0
    n = len(x0)
    ux = rng.uniform(-1.0, 1.0, (n, per_poly))
    uy = rng.uniform(-1.0, 1.0, (n, per_poly))
    px = _clip32(cx[:, None] + ux * hx[:, None])
    py = _clip32(cy[:, None] + uy * hy[:, None])
    return np.stack([px.ravel(), py.ravel()], 1)


# ---------------------------------------------------------------------------------------------
# 2. building-footprint batch
# ---------------------------------------------------------------------------------------------

def footprints(seed=BASE_SEED + 2, n_polys=1_000_000, pts_per_poly=16) -> Workload:
    rng = _rng(seed)
    m_arr = np.clip(np.rint(rng.lognormal(np.log(6.0), 0.5, n_polys)), 4, 64).astype(np.int64)
    centres = np.stack([rng.uniform(LON0 + 10_000, LON1 - 10_000, n_polys),
                        rng.uniform(LAT0 + 10_000, LAT1 - 10_000, n_polys)], 1)
    offs, v = _footprint_shapes(rng, m_arr, centres)
    pts = _points_in_bboxes(rng, offs, v, pts_per_poly)
    co = np.arange(n_polys + 1, dtype=np.int64) * pts_per_poly
    ids = np.arange(n_polys * pts_per_poly, dtype=np.int64)
    return Workload("footprints", pts.astype(np.int32), offs.astype(np.int32), v.astype(np.int32),
                    co.astype(np.int32), ids.astype(np.int32),
                    meta=dict(seed=seed, n_polys=n_polys, pts_per_poly=pts_per_poly,
                              mean_m=float(m_arr.mean())))


# ---------------------------------------------------------------------------------------------
# 3. spatial join (the CSR is produced by binning)
# ---------------------------------------------------------------------------------------------

def _clustered(rng, n, centres, sigma_m, frac_clustered):
    k = rng.random(n) < frac_clustered
    which = rng.integers(0, len(centres), n)
    x = np.where(k, centres[which, 0] + rng.normal(0, sigma_m * UNITS_PER_M_X, n), rng.uniform(LON0, LON1, n))
    y = np.where(k, centres[which, 1] + rng.normal(0, sigma_m * UNITS_PER_M_Y, n), rng.uniform(LAT0, LAT1, n))
    return np.stack([np.clip(x, LON0, LON1), np.clip(y, LAT0, LAT1)], 1)


def join_polygons(seed=BASE_SEED + 3, n_polys=100_000, n_clusters=1_000):
    rng = _rng(seed)
    clusters = np.stack([rng.uniform(LON0, LON1, n_clusters), rng.uniform(LAT0, LAT1, n_clusters)], 1)
    m_arr = np.clip(np.rint(rng.lognormal(np.log(7.0), 0.8, n_polys)), 4, 256).astype(np.int64)
    centres = _clustered(rng, n_polys, clusters, 200.0, 0.7)
    offs, v = _footprint_shapes(rng, m_arr, centres)
    return clusters, offs.astype(np.int32), v.astype(np.int32)


def join_points(clusters, seed, n_points=10_000_000):
    rng = _rng(seed)
    return _clip32(_clustered(rng, n_points, clusters, 200.0, 0.7)).astype(np.int32)


def join(seed=BASE_SEED + 3, n_polys=100_000, n_points=10_000_000, batch=0) -> Workload:
    """Polygons and the points of one batch; ``cand_offsets``/``cand_ids`` are left empty."""
    clusters, offs, v = join_polygons(seed, n_polys)
    pts = join_points(clusters, seed + 1000 + batch, n_points)
    return Workload("join", pts, offs, v, meta=dict(seed=seed, batch=batch, n_polys=n_polys,
                                                     n_points=n_points))


# ---------------------------------------------------------------------------------------------
# 4. fractal coastline polygons
# ---------------------------------------------------------------------------------------------

def _midpoint_displacement(rng, m, centre, radius, sigma0, hurst=0.7):
    ang = np.arange(8) * (2 * np.pi / 8) + rng.uniform(0, 2 * np.pi / 8)
    pts = np.stack([centre[0] + radius * np.cos(ang), centre[1] + radius * np.sin(ang)], 1)
    level = 0
    while len(pts) < m:
        n = len(pts)
        nxt = np.roll(pts, -1, axis=0)
        mid = (pts + nxt) / 2.0
        d = nxt - pts
        perp = np.stack([-d[:, 1], d[:, 0]], 1)
        norm = np.maximum(np.hypot(perp[:, 0], perp[:, 1]), 1e-9)
        sig = sigma0 * 2.0 ** (-hurst * level)
        mid = mid + perp / norm[:, None] * rng.normal(0.0, sig, n)[:, None]
        need = m - n
        if need >= n:
            take = np.ones(n, dtype=bool)
        else:
            take = np.zeros(n, dtype=bool)
            take[rng.choice(n, need, replace=False)] = True
        out = np.empty((n + int(take.sum()), 2))
        pos = np.arange(n) + np.concatenate([[0], np.cumsum(take)[:-1]])
        out[pos] = pts
        out[pos[take] + 1] = mid[take]
        pts = out
        level += 1
    return pts


def fractal(seed=BASE_SEED + 4, n_polys=64, m_lo=10_000, m_hi=1_000_000, n_points=10_000_000,
            cell=5_000_000, grid=8) -> Workload:
    rng = _rng(seed)
    m_arr = np.rint(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), n_polys))).astype(np.int64)
    ox, oy = LON0 + 1_000_000, LAT0 + 1_000_000
    polys = []
    for k in range(n_polys):
        gx, gy = k % grid, (k // grid) % grid
        cx, cy = ox + (gx + 0.5) * cell, oy + (gy + 0.5) * cell
        p = _midpoint_displacement(rng, int(m_arr[k]), (cx, cy), 0.3 * cell, 0.04 * cell)
        lo = np.array([ox + gx * cell + 1, oy + gy * cell + 1])
        hi = lo + cell - 2
        polys.append(np.clip(np.rint(p), lo, hi).astype(np.int64))
    offs = _offsets(m_arr)
    v = np.concatenate(polys)
    ext = grid * cell
    pts = np.stack([rng.integers(ox, ox + ext, n_points), rng.integers(oy, oy + ext, n_points)], 1)
    co, ids = bbox_csr(offs, v, pts)
    return Workload("fractal", pts.astype(np.int32), offs.astype(np.int32), v.astype(np.int32),
                    co.astype(np.int32), ids.astype(np.int32),
                    meta=dict(seed=seed, n_polys=n_polys, m=[int(t) for t in m_arr]))


def bbox_csr(poly_offsets, verts, points):
    """Closed-bbox candidate lists (ascending point id per polygon) for few polygons."""
    x0, y0, x1, y1 = _bboxes(np.asarray(poly_offsets, dtype=np.int64), np.asarray(verts))
    px, py = points[:, 0], points[:, 1]
    lists = []
    for k in range(len(x0)):
        lists.append(np.nonzero((px >= x0[k]) & (px <= x1[k]) & (py >= y0[k]) & (py <= y1[k]))[0])
    co = _offsets(np.array([len(t) for t in lists], dtype=np.int64))
    ids = np.concatenate(lists) if lists else np.zeros(0, dtype=np.int64)
    return co, ids


# ---------------------------------------------------------------------------------------------
# 5. precision stress at the full int32 range
# ---------------------------------------------------------------------------------------------

def stress(seed=BASE_SEED + 5, n_polys=1_000_000, pts_per_poly=8) -> Workload:
    rng = _rng(seed)
    kind = rng.integers(0, 3, n_polys)                 # 0 needle, 1 collinear runs, 2 star
    m_arr = rng.integers(3, 33, n_polys)
    m_arr = np.where(kind == 0, 3, m_arr)
    m_arr = np.where(kind == 1, np.maximum(m_arr, 5), m_arr)
    scale = 2.0 ** rng.uniform(4, 32, n_polys)
    centre = np.stack([rng.uniform(I32_MIN, I32_MAX, n_polys), rng.uniform(I32_MIN, I32_MAX, n_polys)], 1)
    offs = _offsets(m_arr)
    V = int(offs[-1])
    v = np.zeros((V, 2), dtype=np.int64)
    # needle triangles: A, B at distance ~scale; C = a lattice-rounded point of AB moved 1-3 units
    sel = np.nonzero(kind == 0)[0]
    if len(sel):
        A = centre[sel] + rng.uniform(-0.5, 0.5, (len(sel), 2)) * scale[sel, None]
        B = centre[sel] + rng.uniform(-0.5, 0.5, (len(sel), 2)) * scale[sel, None]
        A, B = _clip32(A), _clip32(B)
        t = rng.uniform(0.1, 0.9, len(sel))
        C = np.rint(A + (B - A) * t[:, None]).astype(np.int64)
        C += rng.integers(1, 4, (len(sel), 2)) * rng.choice([-1, 1], (len(sel), 2))
        C = np.clip(C, I32_MIN, I32_MAX)
        base = offs[sel]
        v[base] = A
        v[base + 1] = B
        v[base + 2] = C
    # collinear runs: an axis-aligned box whose sides carry extra lattice vertices and whose
    # first corner is cut by an exact 45-degree diagonal carrying a lattice vertex
    sel = np.nonzero(kind == 1)[0]
    for m in np.unique(m_arr[sel]):
        s2 = sel[m_arr[sel] == m]
        n = len(s2)
        w = np.maximum(np.rint(scale[s2] * rng.uniform(0.3, 1.0, n)), 8).astype(np.int64)
        h = np.maximum(np.rint(scale[s2] * rng.uniform(0.3, 1.0, n)), 8).astype(np.int64)
        cut = np.maximum(np.minimum(w, h) // 4, 2)
        x0 = np.rint(centre[s2, 0] - w / 2).astype(np.int64)
        y0 = np.rint(centre[s2, 1] - h / 2).astype(np.int64)
        # ring (CCW): (x0+cut, y0) -> (x0+w, y0) -> (x0+w, y0+h) -> (x0, y0+h) -> (x0, y0+cut)
        #             -> diagonal lattice point (x0+cut/2, y0+cut/2 - ...)
        corners = np.stack([
            np.stack([x0 + cut, y0], 1), np.stack([x0 + w, y0], 1), np.stack([x0 + w, y0 + h], 1),
            np.stack([x0, y0 + h], 1), np.stack([x0, y0 + cut], 1)], 1)
        extra = int(m) - 5
        diag = np.stack([x0 + cut // 2, y0 + cut - cut // 2], 1)[:, None, :]
        # extra vertices on the 4 axis sides at integer positions, plus the diagonal point
        n_side = max(extra - 1, 0)
        which = rng.integers(0, 4, (n, n_side))
        frac = rng.uniform(0.05, 0.95, (n, n_side))
        keys = which + frac
        order = np.argsort(keys, 1)
        keys = np.take_along_axis(keys, order, 1)
        which = np.floor(keys).astype(np.int64)
        frac = keys - which
        p0 = np.take_along_axis(corners, which[:, :, None].repeat(2, 2), 1)
        p1 = np.take_along_axis(corners, (which + 1)[:, :, None].repeat(2, 2), 1)
        pe = np.rint(p0 + (p1 - p0) * frac[:, :, None]).astype(np.int64)   # axis sides: exact
        allk = np.concatenate([np.broadcast_to(np.arange(5.0), (n, 5)), keys], 1)
        allp = np.concatenate([corners, pe], 1)
        o2 = np.argsort(allk, 1, kind="stable")
        ring = np.take_along_axis(allp, o2[:, :, None].repeat(2, 2), 1)
        if extra >= 1:
            ring = np.concatenate([ring, diag], 1)
        ring = np.clip(ring, I32_MIN, I32_MAX)
        idx = offs[s2][:, None] + np.arange(int(m))[None, :]
        v[idx.ravel()] = ring.reshape(-1, 2)
    # random star polygons
    sel = np.nonzero(kind == 2)[0]
    for m in np.unique(m_arr[sel]):
        s2 = sel[m_arr[sel] == m]
        n = len(s2)
        ang = np.sort(rng.uniform(0, 2 * np.pi, (n, int(m))), 1)
        rad = rng.uniform(0.2, 1.0, (n, int(m))) * scale[s2, None] / 2
        X = centre[s2, 0][:, None] + rad * np.cos(ang)
        Y = centre[s2, 1][:, None] + rad * np.sin(ang)
        idx = offs[s2][:, None] + np.arange(int(m))[None, :]
        v[idx.ravel(), 0] = _clip32(X).ravel()
        v[idx.ravel(), 1] = _clip32(Y).ravel()
    # points: half hard (vertex, edge lattice point, y of a vertex, 1-3 units off an edge),
    # half uniform in the 1.5x bbox, all clamped to int32
    hard = pts_per_poly // 2
    uni = _points_in_bboxes(rng, offs, v, pts_per_poly - hard).reshape(n_polys, -1, 2)
    mp = m_arr[:, None]
    e = rng.integers(0, 2**62, (n_polys, hard)) % mp
    a = v[offs[:-1, None] + e]
    b = v[offs[:-1, None] + (e + 1) % mp]
    d = b - a
    g = np.gcd(np.abs(d[..., 0]), np.abs(d[..., 1]))
    kk = np.where(g > 1, 1 + rng.integers(0, 2**62, g.shape) % np.maximum(g - 1, 1), 0)
    lattice = a + (d // np.maximum(g, 1)[..., None]) * kk[..., None]
    t = rng.uniform(0, 1, g.shape)
    near = np.rint(a + d * t[..., None]).astype(np.int64) + rng.integers(-3, 4, a.shape)
    x0, y0, x1, y1 = _bboxes(offs, v)
    same_y = np.stack([rng.integers(0, 2**62, g.shape) % np.maximum(x1 - x0 + 1, 1)[:, None] + x0[:, None],
                       a[..., 1]], -1)
    pick = rng.integers(0, 4, g.shape)
    hardp = np.where((pick == 0)[..., None], a, np.where((pick == 1)[..., None], lattice,
                     np.where((pick == 2)[..., None], same_y, near)))
    hardp = np.clip(hardp, I32_MIN, I32_MAX)
    pts = np.concatenate([hardp, uni], 1).reshape(-1, 2)
    co = np.arange(n_polys + 1, dtype=np.int64) * pts_per_poly
    ids = np.arange(n_polys * pts_per_poly, dtype=np.int64)
    return Workload("stress", pts.astype(np.int32), offs.astype(np.int32), v.astype(np.int32),
                    co.astype(np.int32), ids.astype(np.int32),
                    meta=dict(seed=seed, n_polys=n_polys, pts_per_poly=pts_per_poly))


# ---------------------------------------------------------------------------------------------
# 6. paper-shaped: all building points of the country against its boundary polygon
# ---------------------------------------------------------------------------------------------

PAPER_N_POINTS = 17_097_823   # building points left in Ghana's box (Simulation section)


def country(seed=BASE_SEED + 6, m=100_000, n_points=PAPER_N_POINTS, n_clusters=1_000) -> Workload:
    """One country-like polygon against every building point in its box, as in the paper's
    experiment (Simulation section: the Open Buildings points inside Ghana's box against the
    GADM boundary of Ghana).  Neither data set is available, so: the polygon is a fractal
    coastline (midpoint displacement from an octagon, Hurst 0.7) with m vertices (the paper
    does not state the boundary's vertex count; 1e5 is an assumption) spanning most of the
    lon/lat box; the points are building-like, 70 % in 1,000 Gaussian settlements of sigma
    200 m and 30 % uniform in the box.  Dense mode: every point is a candidate."""
    rng = _rng(seed)
    cx, cy = (LON0 + LON1) / 2.0, (LAT0 + LAT1) / 2.0
    r = 0.45 * min(LON1 - LON0, LAT1 - LAT0)
    p = _midpoint_displacement(rng, m, (cx, cy), r, 0.05 * r)
    v = _clip32(np.clip(np.rint(p), [LON0, LAT0], [LON1, LAT1])).astype(np.int64)
    clusters = np.stack([rng.uniform(LON0, LON1, n_clusters), rng.uniform(LAT0, LAT1, n_clusters)], 1)
    pts = _clip32(_clustered(rng, n_points, clusters, 200.0, 0.7))
    return Workload("country", pts.astype(np.int32), np.array([0, m], dtype=np.int32), v.astype(np.int32),
                    meta=dict(seed=seed, m=m, n_points=n_points, n_clusters=n_clusters))


WORKLOADS = {
    "star": star,
    "footprints": footprints,
    "join": join,
    "fractal": fractal,
    "stress": stress,
    "country": country,
}


def scattered_points(w: Workload, seed=7) -> Workload:
    """Same (polygon, point) pairs with the points stored in a random order, so that the
    candidate gather becomes random access instead of a stream."""
    rng = _rng(seed)
    perm = rng.permutation(w.n_points)
    pts = np.empty_like(w.points)
    pts[perm] = w.points
    return dataclasses.replace(w, name=w.name + "-scattered", points=pts,
                               cand_ids=perm[w.cand_ids].astype(np.int32))
