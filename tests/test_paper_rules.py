"""The oracle's literal evaluation of the paper's printed Algorithms 1 and 2 (rules 1, 2 of
``oracle.classify_rule``), used to measure how often their boundary and on-ray decisions
differ from the half-open rule.

Pins: hand-worked cases (tests/golden/paper_rules.json) on the ray and on the boundary, where
the rules differ; agreement with the independently pinned half-open oracle at generic points (y
different from every vertex's y, not on any edge), where all three rules coincide because no
candidate edge is horizontal or touched at a vertex; and a second literal evaluation of both
printed rules in plain Python (integers for Algorithm 1, float64 operation by operation for
Algorithm 2) on every lattice point of [-1, 17]^2 against 120 small lattice polygons, boundary
and on-ray points included.
"""
import json
import os

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _one(verts, point, rule):
    v = np.asarray(verts, dtype=np.int32)
    po = np.array([0, len(v)], dtype=np.int32)
    out = oracle.classify_rule(np.asarray([point], dtype=np.int32), po, v, rule)
    return int(out[0] & 1)


def test_golden_paper_rules():
    g = json.load(open(os.path.join(HERE, "golden", "paper_rules.json")))
    for c in g["cases"]:
        for rule, key in ((0, "half_open"), (1, "alg1"), (2, "alg2")):
            assert _one(c["verts"], c["point"], rule) == c[key], (c["name"], key)


def _on_some_edge(p, v):
    m = len(v)
    for i in range(m):
        a, b = v[i], v[(i + 1) % m]
        cross = (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])
        if cross == 0 and min(a[0], b[0]) <= p[0] <= max(a[0], b[0]) and min(a[1], b[1]) <= p[1] <= max(a[1], b[1]):
            return True
    return False


def test_rules_agree_at_generic_points():
    rng = np.random.default_rng(2306043160 + 91)
    checked = 0
    for _ in range(300):
        m = int(rng.integers(3, 9))
        v = rng.integers(0, 17, (m, 2))
        ys = set(v[:, 1].tolist())
        pts = [(x, y) for x in range(-1, 18) for y in range(-1, 18)
               if y not in ys and not _on_some_edge((x, y), v.tolist())]
        if not pts:
            continue
        pts = np.array(pts, dtype=np.int32)
        po = np.array([0, m], dtype=np.int32)
        ref = oracle.unpack_bits(oracle.classify(pts, po, v.astype(np.int32)), len(pts))
        for rule in (1, 2):
            got = oracle.unpack_bits(oracle.classify_rule(pts, po, v.astype(np.int32), rule), len(pts))
            assert np.array_equal(got, ref), (rule, v.tolist())
        checked += len(pts)
    assert checked > 10_000


def test_rules_differ_on_the_boundary():
    """On a lattice square every boundary point is decided by the half-open rule alone; the
    literal rules disagree with it on some of them (counted, not fixed: the paper's rule is
    what it is)."""
    v = np.array([[0, 0], [6, 0], [6, 6], [0, 6]], dtype=np.int32)
    pts = np.array([(x, y) for x in range(-1, 8) for y in range(-1, 8)], dtype=np.int32)
    po = np.array([0, 4], dtype=np.int32)
    n = len(pts)
    ref = oracle.unpack_bits(oracle.classify(pts, po, v), n)
    for rule in (1, 2):
        got = oracle.unpack_bits(oracle.classify_rule(pts, po, v, rule), n)
        diff = np.nonzero(got != ref)[0]
        assert len(diff) > 0
        assert all(_on_some_edge(tuple(pts[i]), v.tolist()) or pts[i][1] in (0, 6) for i in diff)


# ------------------------------------------------------------------------------------------
# A second, independent literal evaluation of the printed rules in plain Python, compared with
# the oracle's on every lattice point (boundary and on-ray points included, where the rules
# differ from the half-open one).  Algorithm 1: exact integers.  Algorithm 2: IEEE float64, one
# rounding per operation as the printed array code performs them: int differences converted to
# float64, the division (0/0 is NaN, x/0 is +-inf), the product, the sum.
# ------------------------------------------------------------------------------------------

import math  # noqa: E402


def _alg1_literal(px, py, v):
    """Constraint 1: an edge is a candidate when f_i f_(i+1) <= 0 (f = y - p_y); its normal
    (d_y, -d_x) is negated when its x component is negative; it counts when (p - R_i) . n <= 0."""
    m, count = len(v), 0
    for i in range(m):
        (xi, yi), (xj, yj) = v[i], v[(i + 1) % m]
        if (yi - py) * (yj - py) > 0:
            continue
        nx, ny = yj - yi, -(xj - xi)
        if nx < 0:
            nx, ny = -nx, -ny
        if (px - xi) * nx + (py - yi) * ny <= 0:
            count += 1
    return count & 1


def _f64_div(a, b):
    if b == 0.0:
        if a == 0.0 or math.isnan(a):
            return math.nan
        return math.copysign(math.inf, a) * math.copysign(1.0, b)
    return a / b


def _alg2_literal(px, py, v):
    """Constraint 2: the same candidates; an edge counts when x_i + ((p_y - y_i) / d_y) d_x > p_x
    in float64 (a NaN never counts)."""
    m, count = len(v), 0
    for i in range(m):
        (xi, yi), (xj, yj) = v[i], v[(i + 1) % m]
        if (yi - py) * (yj - py) > 0:
            continue
        lam = _f64_div(float(py - yi), float(yj - yi))
        x_new = float(xi) + lam * float(xj - xi)
        if x_new > float(px):
            count += 1
    return count & 1


def _lattice_polygons(rng, n):
    """Tiny polygons on the [0, 16]^2 lattice: random vertices (self-intersections, repeated
    vertices), axis-aligned runs (horizontal edges on many rays) and an explicit closing vertex."""
    out = []
    for k in range(n):
        m = int(rng.integers(3, 9))
        v = rng.integers(0, 17, (m, 2)).tolist()
        if k % 4 == 1:      # a horizontal run
            v.insert(1, [v[0][0] + 3, v[0][1]])
        if k % 4 == 2:      # a repeated vertex
            v.insert(2, list(v[1]))
        if k % 4 == 3:      # the closing copy R_n = R_0
            v.append(list(v[0]))
        out.append(v)
    return out


def test_printed_rules_match_a_literal_python_evaluation_everywhere():
    rng = np.random.default_rng(2306043160 + 92)
    pts = [(x, y) for x in range(-1, 18) for y in range(-1, 18)]
    P = np.array(pts, dtype=np.int32)
    checked = 0
    for v in _lattice_polygons(rng, 120):
        V = np.array(v, dtype=np.int32)
        po = np.array([0, len(v)], dtype=np.int32)
        for rule, lit in ((1, _alg1_literal), (2, _alg2_literal)):
            got = oracle.unpack_bits(oracle.classify_rule(P, po, V, rule), len(pts))
            want = np.array([lit(x, y, v) for x, y in pts], dtype=np.uint8)
            bad = np.nonzero(got != want)[0]
            assert len(bad) == 0, (rule, v, [pts[i] for i in bad[:5]])
        checked += len(pts)
    assert checked == 120 * 361
