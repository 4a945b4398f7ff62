"""The oracle's pins P1-P9, written so that any compiled copy of the oracle can be checked.

Each ``pin_*`` function takes an oracle library handle (``oracle.open_library``) and
returns a list of failure strings (empty = pinned).  ``test_oracle_pins`` runs them on
the real oracle; ``test_oracle_mutants`` runs them on deliberately broken copies to show
that each plausible slip is caught by at least one pin.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

import oracle
import pins

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dense_one(lib, points, verts) -> np.ndarray:
    """Oracle bits of many points against one polygon (dense mode), as 0/1 uint8."""
    pts = np.asarray(points, dtype=np.int64).reshape(-1, 2)
    v = np.asarray(verts, dtype=np.int64).reshape(-1, 2)
    words = oracle.classify(pts, np.array([0, len(v)]), v, lib=lib, threads=1)
    return oracle.unpack_bits(words, len(pts))


def _fail(out, name, pt, got, want, extra=""):
    if len(out) < 8:
        out.append(f"{name}: point {tuple(int(t) for t in pt)} got {int(got)} want {int(want)} {extra}")


def pin_golden(lib):
    out = []
    d = json.load(open(os.path.join(GOLDEN, "diamond.json")))
    got = dense_one(lib, [d["point"]], d["verts"])[0]
    if got != d["inside_half_open"]:
        _fail(out, "diamond", d["point"], got, d["inside_half_open"])
    s = json.load(open(os.path.join(GOLDEN, "square.json")))
    pts = [c[0] for c in s["cases"]]
    got = dense_one(lib, pts, s["verts"])
    for (p, want), g in zip(s["cases"], got):
        if g != want:
            _fail(out, "square", p, g, want)
    return out


def pin_rectangles(lib, seed=1):
    """P1: axis-aligned rectangles, exhaustive on a small lattice and random at full range."""
    out = []
    rng = np.random.default_rng(seed)
    for _ in range(60):
        x0, x1 = sorted(rng.integers(-6, 7, 2))
        y0, y1 = sorted(rng.integers(-6, 7, 2))
        if x0 == x1 or y0 == y1:
            continue
        start = int(rng.integers(0, 4))
        ring = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
        if rng.random() < 0.5:
            ring = ring[::-1]
        ring = ring[start:] + ring[:start]
        xs, ys = np.meshgrid(np.arange(x0 - 2, x1 + 3), np.arange(y0 - 2, y1 + 3))
        pts = np.stack([xs.ravel(), ys.ravel()], 1)
        got = dense_one(lib, pts, ring)
        for p, g in zip(pts, got):
            w = pins.rect_inside(p[0], p[1], x0, y0, x1, y1)
            if g != w:
                _fail(out, "rect", p, g, w)
    lo, hi = -2**31, 2**31 - 1
    for _ in range(40):
        x0, x1 = sorted(int(t) for t in rng.integers(lo, hi, 2, endpoint=True))
        y0, y1 = sorted(int(t) for t in rng.integers(lo, hi, 2, endpoint=True))
        if x0 == x1 or y0 == y1:
            continue
        ring = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
        cand = []
        for _k in range(200):
            px = int(rng.choice([x0, x1, x0 - 1, x1 - 1, x0 + 1, int(rng.integers(x0, x1))]))
            py = int(rng.choice([y0, y1, y0 - 1, y1 - 1, y0 + 1, int(rng.integers(y0, y1))]))
            if lo <= px <= hi and lo <= py <= hi:
                cand.append((px, py))
        got = dense_one(lib, cand, ring)
        for p, g in zip(cand, got):
            w = pins.rect_inside(p[0], p[1], x0, y0, x1, y1)
            if g != w:
                _fail(out, "rect-full", p, g, w)
    return out


def pin_triangles(lib, seed=2):
    """P2: triangle closed form (first-order expansion of the three orientations)."""
    out = []
    rng = np.random.default_rng(seed)
    for _ in range(120):
        tri = [tuple(int(t) for t in rng.integers(-5, 6, 2)) for _ in range(3)]
        xs, ys = np.meshgrid(np.arange(-6, 7), np.arange(-6, 7))
        pts = np.stack([xs.ravel(), ys.ravel()], 1)
        got = dense_one(lib, pts, tri)
        for p, g in zip(pts, got):
            w = pins.triangle_inside((int(p[0]), int(p[1])), *tri)
            if g != w:
                _fail(out, f"tri {tri}", p, g, w)
    lo, hi = -2**31, 2**31 - 1
    for _ in range(60):
        tri = [tuple(int(t) for t in rng.integers(lo, hi, 2, endpoint=True)) for _ in range(3)]
        if rng.random() < 0.3:  # needle: third vertex a few units off the long side
            (ax, ay), (bx, by) = tri[0], tri[1]
            t = rng.random()
            cx = int(ax + t * (bx - ax)) + int(rng.integers(-3, 4))
            cy = int(ay + t * (by - ay)) + int(rng.integers(-3, 4))
            tri[2] = (min(max(cx, lo), hi), min(max(cy, lo), hi))
        pts = []
        for _k in range(150):
            a, b = tri[int(rng.integers(0, 3))], tri[int(rng.integers(0, 3))]
            t = rng.random()
            px = int(a[0] + t * (b[0] - a[0])) + int(rng.integers(-2, 3))
            py = int(a[1] + t * (b[1] - a[1])) + int(rng.integers(-2, 3))
            if rng.random() < 0.2:
                px, py = a
            pts.append((min(max(px, lo), hi), min(max(py, lo), hi)))
        got = dense_one(lib, pts, tri)
        for p, g in zip(pts, got):
            w = pins.triangle_inside(p, *tri)
            if g != w:
                _fail(out, "tri-full", p, g, w)
    return out


def _star(rng, m, R, cx=0, cy=0):
    ang = np.sort(rng.uniform(0, 2 * np.pi, m))
    rad = rng.uniform(0.5, 1.0, m) * R
    v = np.stack([np.rint(cx + rad * np.cos(ang)), np.rint(cy + rad * np.sin(ang))], 1).astype(np.int64)
    return [tuple(int(t) for t in r) for r in v]


def pin_star(lib, seed=3):
    """P3: star polygon sector form at off-boundary points."""
    out = []
    rng = np.random.default_rng(seed)
    for m, R in ((16, 50), (64, 1000), (256, 100000)):
        v = _star(rng, m, R)
        pts = rng.integers(-R - 2, R + 3, size=(1500, 2))
        got = dense_one(lib, pts, v)
        for p, g in zip(pts, got):
            px, py = int(p[0]), int(p[1])
            if pins.on_boundary(px, py, v):
                continue
            w = pins.star_inside(px, py, 0, 0, v)
            if g != w:
                _fail(out, f"star m={m}", p, g, w)
    return out


def _random_poly(rng, m, lo, hi):
    return [tuple(int(t) for t in rng.integers(lo, hi + 1, 2)) for _ in range(m)]


def pin_winding(lib, seed=4):
    """P4: winding number mod 2 equals the oracle at off-boundary points (self-intersecting
    polygons included)."""
    out = []
    rng = np.random.default_rng(seed)
    for scale in (20, 10**4, 2**30):
        for _ in range(25):
            m = int(rng.integers(3, 14))
            v = _random_poly(rng, m, -scale, scale)
            pts = rng.integers(-scale - 2, scale + 3, size=(200, 2))
            # add points sharing a vertex's y (on the ray through a vertex)
            extra = [(int(rng.integers(-scale, scale + 1)), v[int(rng.integers(0, m))][1])
                     for _ in range(50)]
            pts = np.concatenate([pts, np.array(extra, dtype=np.int64)])
            got = dense_one(lib, pts, v)
            for p, g in zip(pts, got):
                px, py = int(p[0]), int(p[1])
                if pins.on_boundary(px, py, v):
                    continue
                w = pins.winding_number(px, py, v) & 1
                if g != w:
                    _fail(out, f"winding scale={scale}", p, g, w)
    return out


def pin_bruteforce(lib, seed=5, n_polys=150):
    """P5: tiny lattice polygons with every degeneracy, every lattice point of [-1, 17]^2,
    against the scaled-perturbation winding number."""
    out = []
    rng = np.random.default_rng(seed)
    xs, ys = np.meshgrid(np.arange(-1, 18), np.arange(-1, 18))
    pts = np.stack([xs.ravel(), ys.ravel()], 1)
    for t in range(n_polys):
        m = int(rng.integers(3, 9))
        v = _random_poly(rng, m, 0, 16)
        kind = t % 5
        if kind == 1:  # repeated vertex
            i = int(rng.integers(0, m))
            v = v[:i + 1] + [v[i]] + v[i + 1:]
        elif kind == 2:  # horizontal and vertical runs
            i = int(rng.integers(0, m))
            x, y = v[i]
            v = v[:i + 1] + [(int(rng.integers(0, 17)), y), (int(rng.integers(0, 17)), y)] + v[i + 1:]
        elif kind == 3:  # collinear run along a lattice diagonal
            x, y = v[0]
            k = int(rng.integers(1, 4))
            v = [(x, y), (min(x + k, 16), min(y + k, 16)), (min(x + 2 * k, 16), min(y + 2 * k, 16))] + v[1:]
        elif kind == 4:  # explicit closing vertex R_n = R_0
            v = v + [v[0]]
        got = dense_one(lib, pts, v)
        for p, g in zip(pts, got):
            w = pins.perturbed_inside(int(p[0]), int(p[1]), v)
            if g != w:
                _fail(out, f"brute {v}", p, g, w)
    return out


def pin_tiling(lib, seed=6):
    """P6: a tiling of a box assigns every lattice point of the half-open box to exactly one
    tile and points outside to none."""
    out = []
    rng = np.random.default_rng(seed)
    # jittered quad mesh over [0, 40] x [0, 40]; boundary vertices stay on the box
    n = 5
    g = np.zeros((n + 1, n + 1, 2), dtype=np.int64)
    for i in range(n + 1):
        for j in range(n + 1):
            x, y = 8 * i, 8 * j
            if 0 < i < n:
                x += int(rng.integers(-3, 4))
            if 0 < j < n:
                y += int(rng.integers(-3, 4))
            g[i, j] = (x, y)
    polys = []
    for i in range(n):
        for j in range(n):
            quad = [g[i, j], g[i + 1, j], g[i + 1, j + 1], g[i, j + 1]]
            polys.append([tuple(int(t) for t in q) for q in quad])
    # a triangulated fan inside [100, 140]^2 around (120, 120) (a convex 8-gon, 8 triangles)
    ring = [(110, 102), (130, 102), (138, 110), (138, 130), (130, 138), (110, 138), (102, 130), (102, 110)]
    fan = [[(120, 120), ring[k], ring[(k + 1) % 8]] for k in range(8)]
    xs, ys = np.meshgrid(np.arange(-2, 43), np.arange(-2, 43))
    pts = np.stack([xs.ravel(), ys.ravel()], 1)
    total = np.zeros(len(pts), dtype=np.int64)
    for poly in polys:
        total += dense_one(lib, pts, poly)
    for p, tcount in zip(pts, total):
        w = pins.rect_inside(p[0], p[1], 0, 0, 40, 40)
        if tcount != w:
            _fail(out, "quad-mesh", p, tcount, w)
    xs, ys = np.meshgrid(np.arange(100, 141), np.arange(100, 141))
    pts = np.stack([xs.ravel(), ys.ravel()], 1)
    total = np.zeros(len(pts), dtype=np.int64)
    for tri in fan:
        total += dense_one(lib, pts, tri)
    whole = dense_one(lib, pts, ring)
    for p, tcount, w in zip(pts, total, whole):
        if tcount != w or tcount > 1:
            _fail(out, "fan", p, tcount, w)
    return out


def pin_invariance_exact(lib, seed=7):
    """P7: transformations that leave every bit unchanged (boundary points included)."""
    out = []
    rng = np.random.default_rng(seed)
    for t in range(60):
        m = int(rng.integers(3, 10))
        v = _random_poly(rng, m, 0, 30)
        xs, ys = np.meshgrid(np.arange(-1, 32), np.arange(-1, 32))
        pts = np.stack([xs.ravel(), ys.ravel()], 1)
        base = dense_one(lib, pts, v)
        variants = {
            "reversed": v[::-1],
            "rotated": v[3 % m:] + v[:3 % m],
            "dup-vertex": v[:2] + [v[1]] + v[2:],
            "closed": v + [v[0]],
        }
        # split an edge at a lattice point on it
        for i in range(m):
            (ax, ay), (bx, by) = v[i], v[(i + 1) % m]
            gg = math.gcd(abs(bx - ax), abs(by - ay))
            if gg > 1:
                mid = (ax + (bx - ax) // gg, ay + (by - ay) // gg)
                variants["split-edge"] = v[:i + 1] + [mid] + v[i + 1:]
                break
        for name, w in variants.items():
            got = dense_one(lib, pts, w)
            bad = np.nonzero(got != base)[0]
            for b in bad[:2]:
                _fail(out, name, pts[b], got[b], base[b])
        # integer translation (points and polygon together)
        dxy = rng.integers(-2**30, 2**30, 2)
        got = dense_one(lib, pts + dxy, [(x + int(dxy[0]), y + int(dxy[1])) for x, y in v])
        bad = np.nonzero(got != base)[0]
        for b in bad[:2]:
            _fail(out, "translate", pts[b], got[b], base[b])
    return out


def pin_invariance_offboundary(lib, seed=8):
    """P8: reflections, axis swap and quarter turns preserve bits at off-boundary points."""
    out = []
    rng = np.random.default_rng(seed)
    for t in range(40):
        m = int(rng.integers(3, 12))
        v = _random_poly(rng, m, -1000, 1000)
        pts = rng.integers(-1002, 1003, size=(400, 2))
        keep = np.array([not pins.on_boundary(int(p[0]), int(p[1]), v) for p in pts])
        pts = pts[keep]
        base = dense_one(lib, pts, v)
        maps = {
            "mirror-x": (lambda x, y: (-x, y)),
            "mirror-y": (lambda x, y: (x, -y)),
            "swap": (lambda x, y: (y, x)),
            "rot90": (lambda x, y: (-y, x)),
        }
        for name, f in maps.items():
            w = [f(x, y) for x, y in v]
            q = np.array([f(int(p[0]), int(p[1])) for p in pts])
            got = dense_one(lib, q, w)
            bad = np.nonzero(got != base)[0]
            for b in bad[:2]:
                _fail(out, name, pts[b], got[b], base[b])
    return out


def pin_layouts(lib, seed=9):
    """CSR and dense layouts give the same bits for the same (polygon, point) pairs,
    including empty polygons, fewer than 3 vertices and empty candidate lists."""
    out = []
    rng = np.random.default_rng(seed)
    polys = [_random_poly(rng, int(rng.integers(3, 9)), 0, 20) for _ in range(9)]
    polys[2] = []
    polys[5] = [(3, 3), (9, 9)]
    po = np.concatenate([[0], np.cumsum([len(p) for p in polys])])
    verts = np.array([q for p in polys for q in p], dtype=np.int64).reshape(-1, 2)
    pts = rng.integers(-1, 22, size=(77, 2))
    dense = oracle.unpack_bits(oracle.classify(pts, po, verts, lib=lib, threads=3), 9 * 96)
    ids, offs = [], [0]
    for k in range(9):
        sel = [] if k == 4 else list(rng.choice(77, size=int(rng.integers(0, 40)), replace=False))
        ids += sel
        offs.append(len(ids))
    csr = oracle.unpack_bits(oracle.classify(pts, po, verts, np.array(offs), np.array(ids), lib=lib,
                                             threads=2), len(ids))
    for k in range(9):
        for c in range(offs[k], offs[k + 1]):
            if csr[c] != dense[k * 96 + ids[c]]:
                _fail(out, f"layout poly {k}", pts[ids[c]], csr[c], dense[k * 96 + ids[c]])
    for k in (2, 5):
        if dense[k * 96:(k + 1) * 96].any():
            out.append(f"degenerate polygon {k} has inside points")
    return out


ALL_PINS = [pin_golden, pin_rectangles, pin_triangles, pin_star, pin_winding, pin_bruteforce,
            pin_tiling, pin_invariance_exact, pin_invariance_offboundary, pin_layouts]
