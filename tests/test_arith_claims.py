"""Host checks of the arithmetic facts the exact fast paths of the kernels rest on (Method section,
Constraint 1: the straddle test and the sign of det decide each pair).  They run on numpy's IEEE
FP32 and wrapping int32 arithmetic, the same rounding and wrap-around rules the GPU applies.

- A point clamped to [x0 - 1, x1] x [y0 - 1, y1] of a box with (W + 1)(H + 1) <= 2^30 has
  |det| < 2^31 against every edge inside the box, so the int32 record c + p_x a + p_y b
  evaluated with wrap-around equals -sign(d_y) det exactly on every edge with d_y != 0 (the only
  ones that can straddle).
- Below 2^24 the FP32 difference of two integers is exact and its sign bit is set exactly when
  the first is smaller (an exact zero is +0), so the straddle test may run in FP32 there; at
  2^24 + 1 it is no longer exact.
"""
import numpy as np


def _int32_record(xi, yi, xj, yj):
    """(c, a, b) with c + p_x a + p_y b = -sign(d_y) det modulo 2^32 (uint32 arithmetic)."""
    u = np.uint32
    dx, dy = (xj.astype(u) - xi.astype(u)), (yj.astype(u) - yi.astype(u))
    c = xi.astype(u) * dy - yi.astype(u) * dx
    pos = dy.view(np.int32) > 0
    a = np.where(pos, dy, u(0) - dy)
    b = np.where(pos, u(0) - dx, dx)
    c = np.where(pos, u(0) - c, c)
    return c, a, b


def test_int32_record_exact_for_clamped_points():
    rng = np.random.default_rng(2306043160 + 300)
    with np.errstate(over="ignore"):
        for trial in range(200):
            # a box with (W + 1)(H + 1) <= 2^30 anywhere in the int32 range, often at its limits
            w = int(rng.integers(0, 2**15)) if trial % 3 else int(rng.integers(0, 2**30 // 2 - 1))
            h = (2**30 // (w + 1)) - 1
            h = int(rng.integers(0, h + 1)) if trial % 2 else h
            x0 = int(rng.integers(-2**31 + 1, 2**31 - 1 - w))
            y0 = int(rng.integers(-2**31 + 1, 2**31 - 1 - h))
            if trial % 7 == 0:
                x0, y0 = -2**31 + 1, 2**31 - 1 - h
            n = 4000
            xi, xj = rng.integers(x0, x0 + w + 1, n), rng.integers(x0, x0 + w + 1, n)
            yi, yj = rng.integers(y0, y0 + h + 1, n), rng.integers(y0, y0 + h + 1, n)
            px = rng.integers(x0 - 1, x0 + w + 1, n)
            py = rng.integers(y0 - 1, y0 + h + 1, n)
            det = (xi - px) * (yj - yi) - (yi - py) * (xj - xi)            # exact in int64
            assert np.abs(det).max() < 2**31
            want = -np.sign(yj - yi) * det
            c, a, b = _int32_record(*(v.astype(np.int32) for v in (xi, yi, xj, yj)))
            nt = (c + px.astype(np.int32).astype(np.uint32) * a
                  + py.astype(np.int32).astype(np.uint32) * b).view(np.int32)
            live = yj != yi                      # a horizontal edge never straddles: nt unused
            assert np.array_equal(nt.astype(np.int64)[live], want[live]), trial


def test_fp32_straddle_difference_below_2_24():
    rng = np.random.default_rng(2306043160 + 301)
    lim = 2**24
    a = np.concatenate([rng.integers(-1, lim + 1, 200_000), np.array([0, lim, lim, -1, 0, lim - 1])])
    b = np.concatenate([rng.integers(0, lim + 1, 200_000), np.array([0, lim, 0, lim, lim, lim])])
    # operands as the kernel forms them (clamped p_y - y0 in [-1, H], y - y0 in [0, H], H < 2^24)
    keep = (np.abs(a - b) <= lim)
    a, b = a[keep], b[keep]
    d = a.astype(np.float32) - b.astype(np.float32)
    assert np.array_equal(d.astype(np.int64), a - b)                       # exact
    sign = (d.view(np.uint32) >> 31).astype(bool)
    assert np.array_equal(sign, a < b)                                      # sign bit <=> a < b
    assert not np.signbit(np.float32(5) - np.float32(5))                   # exact zero is +0


def test_fp32_straddle_not_exact_above_2_24():
    """The bound is tight: one past 2^24 an integer no longer converts exactly, so the kernels
    keep the integer subtraction for taller tiles."""
    big = 2**24 + 1
    assert int(np.float32(big)) != big
    assert not (np.float32(big) - np.float32(2**24) > 0)                   # the difference is lost
