"""Independent checks that pin the oracle to the mathematics (no crossing-parity code).

Nothing here counts ray crossings: every function below reaches the inside/outside
answer by a different route, so that a slip in the oracle (a dropped term, a wrong
sign, a swapped index, the wrong boundary rule) makes at least one pin fail.

The oracle defines inside(p, R) as: the point p + (eps, delta), 0 < delta << eps
infinitesimal, lies in the even-odd interior of R (the half-open reading of the
Method section's sign-change step and of Constraint 1's side test).

* ``rect_inside``      closed form for an axis-aligned rectangle (half-open box).
* ``triangle_inside``  closed form for a triangle, from a first-order expansion of
                       the three orientation tests at p + (eps, delta).
* ``winding_number``   exact winding number by quadrant counting (angle summation
                       in quarter turns) at any point off the boundary.
* ``perturbed_inside`` brute force for small lattice polygons: winding number, mod
                       2, at the scaled point (K p_x + 64, K p_y + 1) against K R,
                       K = 4096, which lies in the same face as p + (eps, delta).
* ``on_boundary``      exact test of p lying on an edge.
* ``star_inside``      sector form for a polygon star-shaped about a centre c.
* ``literal_paper_count`` the paper's printed rule taken literally (f_i f_{i+1} <= 0
                       and line_pos <= 0, Algorithm 1) -- used to document where the
                       half-open reading deviates from it (the diamond example).
All arithmetic is Python integers, hence exact.
"""
from __future__ import annotations


def orient(ax, ay, bx, by, cx, cy) -> int:
    """(b - a) x (c - a): > 0 when c is left of a->b."""
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)


def rect_inside(px, py, x0, y0, x1, y1) -> int:
    """Axis-aligned rectangle [x0, x1] x [y0, y1]: p + (eps, delta) inside the open box
    iff x0 <= p_x < x1 and y0 <= p_y < y1 (integers)."""
    return int(x0 <= px < x1 and y0 <= py < y1)


def triangle_inside(p, a, b, c) -> int:
    """Triangle closed form.  Orient CCW; edge U->V accepts p iff orient(U, V, p) > 0,
    or orient = 0 and (dy < 0, or dy = 0 and dx > 0) -- the sign of
    orient(U, V, p + (eps, delta)) = o + dx*delta - dy*eps to first order."""
    area = orient(*a, *b, *c)
    if area == 0:
        return 0
    if area < 0:
        b, c = c, b
    for (ux, uy), (vx, vy) in ((a, b), (b, c), (c, a)):
        o = orient(ux, uy, vx, vy, p[0], p[1])
        dx, dy = vx - ux, vy - uy
        if o > 0:
            continue
        if o == 0 and (dy < 0 or (dy == 0 and dx > 0)):
            continue
        return 0
    return 1


def _quadrant(x, y) -> int:
    # half-open quarter planes by angle: [0, 90), [90, 180), [180, 270), [270, 360)
    if x > 0 and y >= 0:
        return 0
    if x <= 0 and y > 0:
        return 1
    if x < 0 and y <= 0:
        return 2
    return 3


def winding_number(px, py, verts) -> int:
    """Exact winding number of the closed polyline about p (p must be off the boundary)."""
    m = len(verts)
    total = 0
    for i in range(m):
        ax, ay = verts[i][0] - px, verts[i][1] - py
        bx, by = verts[(i + 1) % m][0] - px, verts[(i + 1) % m][1] - py
        if (ax, ay) == (0, 0) or (bx, by) == (0, 0):
            raise ValueError("point on a vertex")
        qa, qb = _quadrant(ax, ay), _quadrant(bx, by)
        d = (qb - qa) % 4
        if d == 3:
            d = -1
        elif d == 2:
            cr = ax * by - ay * bx
            if cr == 0:
                raise ValueError("point on an edge")
            d = 2 if cr > 0 else -2
        total += d
    assert total % 4 == 0
    return total // 4


def on_boundary(px, py, verts) -> bool:
    m = len(verts)
    for i in range(m):
        ax, ay = verts[i]
        bx, by = verts[(i + 1) % m]
        if orient(ax, ay, bx, by, px, py) == 0 and min(ax, bx) <= px <= max(ax, bx) \
                and min(ay, by) <= py <= max(ay, by):
            return True
    return False


K_SCALE = 4096


def perturbed_inside(px, py, verts) -> int:
    """Brute force for lattice polygons with coordinates in [0, 16]: parity of the winding
    number at (K p_x + 64, K p_y + 1) against the polygon scaled by K = 4096.

    The offset (1/64, 1/4096) is shorter than the distance 1/(16 sqrt 2) from any lattice
    point to an edge line not through it, and its angle atan(1/64) is below the smallest
    positive lattice direction angle atan(1/16), so the scaled point sits in the same face
    as p + (eps, delta) with delta << eps.  It is never on an axis through a scaled vertex
    (64 and 1 are not multiples of K), so the quadrant count is well defined."""
    K = K_SCALE
    sv = [(K * x, K * y) for x, y in verts]
    return winding_number(K * px + 64, K * py + 1, sv) & 1


def star_inside(px, py, cx, cy, verts) -> int:
    """Polygon star-shaped about c with vertices in strictly increasing angle (CCW, each
    sector under 180 degrees).  For p off the boundary: p is inside iff p = c or p lies
    strictly inside the triangle (c, v_i, v_{i+1}) of its sector or on the shared rays."""
    if (px, py) == (cx, cy):
        return 1
    m = len(verts)
    rx, ry = px - cx, py - cy
    for i in range(m):
        ax, ay = verts[i][0] - cx, verts[i][1] - cy
        bx, by = verts[(i + 1) % m][0] - cx, verts[(i + 1) % m][1] - cy
        # p in the sector [a, b): cross(a, r) >= 0 and cross(r, b) > 0 (sector < 180 deg)
        if ax * ry - ay * rx >= 0 and rx * by - ry * bx > 0:
            if ax * ry - ay * rx == 0 and ax * rx + ay * ry < 0:
                continue  # opposite ray
            return int(orient(verts[i][0], verts[i][1], verts[(i + 1) % m][0],
                              verts[(i + 1) % m][1], px, py) > 0)
    raise ValueError("sector not found")


def literal_paper_count(px, py, verts) -> int:
    """Crossing count under the paper's rule read literally (Algorithm 1): candidate edges
    where f_i f_{i+1} <= 0, normal n = (dy, -dx) flipped to n_x >= 0, counted when
    (p - r_i) . n <= 0.  As in the paper, the vertex array is R_0 .. R_n with R_n = R_0
    (appended here when missing) and only consecutive rows form edges."""
    rows = [tuple(v) for v in verts]
    if rows[0] != rows[-1]:
        rows.append(rows[0])
    cnt = 0
    for i in range(len(rows) - 1):
        xi, yi = rows[i]
        xj, yj = rows[i + 1]
        if (yi - py) * (yj - py) > 0:
            continue
        nx, ny = yj - yi, xi - xj
        if nx < 0:
            nx, ny = -nx, -ny
        if (px - xi) * nx + (py - yi) * ny <= 0:
            cnt += 1
    return cnt
