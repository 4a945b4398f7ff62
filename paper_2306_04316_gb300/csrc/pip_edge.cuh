// Per-edge records, exact fallbacks and output helpers shared by the small-polygon kernels
// (pip_filtered.cu, pip_small.cu) of pip_classify.
//
// Method section, steps 2-7 with Constraint 1: the straddle test (y_i > p_y) != (y_j > p_y) and
// the side test sign(d_y) det > 0 with det = (x_i - p_x) d_y - (y_i - p_y) d_x.  The records
// below hold per-edge terms so that a (point, edge) pair costs a few multiply-adds: exact int32
// for small boxes, exact int64 products below 2^31, FP32 with a forward-error bound above.
#pragma once

#include "pip_device.cuh"

namespace pipdev {

// Bound factor of the FP32 records: rounding the four record inputs, the product Y d_x and the
// fused X d_y - Y d_x, then P_x, P_y and the two per-pair fused operations, costs at most
// 5u|X d_y| + 6u|Y d_x| + 4u|P_x d_y| + 3u|P_y d_x| (+ O(u^2)) <= 12u (M_x H + M_y W), with H, W
// the polygon's height and width (>= |d_y|, |d_x| of every edge).
constexpr float PM_BOUND_K = 7.748603820800781e-07f;     // 13 * 2^-24 (exact in FP32)
constexpr int WP_V = 256;           // most vertices of a small polygon (and of a staged run)
constexpr long long LARGE_W = 1LL << 18;   // (candidates x vertices) above which a polygon is large
// Arithmetic of a polygon's pair tests: exact int32 when its box is small enough that every
// value fits (width, height < 2^30 and width * height < 2^30); exact int64 products of int32
// differences when the box is below 2^31 on both sides; else the FP32 filter, with int64/double
// records when the box is 2^30 or more from its centre.
constexpr int MODE_INT32 = 0, MODE_INT64 = 1, MODE_FP32 = 2, MODE_WIDE = 3;

// A polygon goes to k_pip_large when it has more vertices than a run holds or more
// (candidate, edge) pairs than one warp should walk.
__device__ __forceinline__ bool is_large_polygon(long long m, long long n)
{
    return m > WP_V || m * n > LARGE_W;
}

// c' = s (X_i d_y - Y_i d_x) rounded to FP32 (s = sign(d_y)).
__device__ __forceinline__ float edge_c(int2 ri, long long dx, long long dy, int ox, int oy, int wide)
{
    const long long X = (long long)ri.x - ox, Y = (long long)ri.y - oy;
    float c;
    if (!wide) {
        c = __ll2float_rn(X * dy - Y * dx);              // |X dy|, |Y dx| < 2^61: exact int64
    } else {
        c = __double2float_rn(__dmul_rn((double)X, (double)dy) - __dmul_rn((double)Y, (double)dx));
    }
    return dy > 0 ? c : -c;
}

// Edge record of a frame 2^30 or more wide (int64 and double arithmetic; rare, out of line).
static __device__ __noinline__ float4 wide_record(int2 ri, int2 rj, int ox, int oy)
{
    const long long dx = (long long)rj.x - ri.x, dy = (long long)rj.y - ri.y;
    const float c = dy == 0 ? 0.f : edge_c(ri, dx, dy, ox, oy, 1);
    return dy > 0 ? make_float4(c, __ll2float_rn(dy), __ll2float_rn(dx), __int_as_float(rj.y))
                  : make_float4(c, __ll2float_rn(-dy), __ll2float_rn(-dx), __int_as_float(rj.y));
}

// Exact parity of p over the edges e0..e1-1 of staged vertices v, edge e running from v[e]
// to v[e + 1], or to v[e0] for the last edge when `wrap`.  Rare path: kept out of line.
static __device__ __noinline__ int exact_parity(const int2 *v, int e0, int e1, bool wrap, int2 p)
{
    int parity = 0;
    for (int e = e0; e < e1; ++e) {
        const int nx = (wrap && e + 1 == e1) ? e0 : e + 1;
        const int2 ri = v[e], rj = v[nx];
        if ((ri.y > p.y) != (rj.y > p.y)) parity ^= exact_edge_counts(p.x, p.y, ri.x, ri.y, rj.x, rj.y);
    }
    return parity;
}

// Exact parity of p over the edges e0..e1-1 of a polygon of m vertices read straight from global
// memory (edge e runs from v[e] to v[(e + 1) mod m]).  Used by a large-polygon CTA whose wait for
// a staged tile gave up: it no longer trusts or touches its shared tile buffer.
static __device__ __noinline__ int global_exact_parity(const int2 *__restrict__ v, int m, int e0, int e1, int2 p)
{
    int parity = 0;
    int2 ri = __ldg(v + e0);
    for (int e = e0; e < e1; ++e) {
        const int2 rj = __ldg(v + (e + 1 == m ? 0 : e + 1));
        if ((ri.y > p.y) != (rj.y > p.y)) parity ^= exact_edge_counts(p.x, p.y, ri.x, ri.y, rj.x, rj.y);
        ri = rj;
    }
    return parity;
}

// Exact parity of the point (px, py) over the same edges, computed by the 32 lanes of a warp
// together (lane l takes edges e0 + l, e0 + l + 32, ...); every lane returns it.  All lanes must
// call it.  The rare recheck of one lane's candidate over a large polygon's tile then costs its
// warp about (e1 - e0) / 32 exact tests instead of e1 - e0.  (The small-polygon kernel keeps the
// per-lane exact_parity: its polygons have at most 256 edges, and the warp-wide form there
// measured more instructions on the footprint batch, whose polygons never take this path.)
__device__ __forceinline__ int warp_exact_parity(const int2 *v, int e0, int e1, bool wrap, int px, int py, int lane)
{
    int part = 0;
    for (int e = e0 + lane; e < e1; e += 32) {
        const int nx = (wrap && e + 1 == e1) ? e0 : e + 1;
        const int2 ri = v[e], rj = v[nx];
        if ((ri.y > py) != (rj.y > py)) part ^= exact_edge_counts(px, py, ri.x, ri.y, rj.x, rj.y);
    }
    return __popc(__ballot_sync(FULL, part)) & 1;
}

// Sets exactly the bits `mask` of *word to `bits` (other bits untouched, no zero-fill needed).
__device__ __forceinline__ void masked_store(uint32_t *word, unsigned mask, unsigned bits)
{
    if (mask == 0xffffffffu) {
        *word = bits;
    } else if (mask) {
        atomicAnd(word, ~mask | bits);
        atomicOr(word, bits & mask);
    }
}

__device__ __forceinline__ unsigned range_mask(int lo, int hi)   // bits [lo, hi), 0 <= lo <= hi <= 32
{
    return (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
}

// Bits [c0, c1) of the output to 0, by the 32 lanes of a warp.
__device__ __forceinline__ void zero_bits(uint32_t *out, long long c0, long long c1, int lane)
{
    if (c1 <= c0) return;
    const long long w0 = c0 >> 5, w1 = (c1 + 31) >> 5;
    for (long long wd = w0 + lane; wd < w1; wd += 32) {
        const int lo = (int)(max(c0, wd * 32) - wd * 32), hi = (int)(min(c1, wd * 32 + 32) - wd * 32);
        masked_store(out + wd, range_mask(lo, hi), 0u);
    }
}

// 16-byte shared-memory load at a 32-bit shared address.
__device__ __forceinline__ int4 lds128(unsigned addr)
{
    int4 v;
    asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}

// Integer record of the edge ri -> rj for the exact int32 test (origin-free):
// x + p_x y + p_y z = -sign(d_y) det modulo 2^32, w = y_j.
__device__ __forceinline__ int4 int32_record(int2 ri, int2 rj)
{
    const unsigned dx = (unsigned)rj.x - (unsigned)ri.x, dy = (unsigned)rj.y - (unsigned)ri.y;
    const unsigned c = (unsigned)ri.x * dy - (unsigned)ri.y * dx;
    return (int)dy > 0 ? make_int4((int)(0u - c), (int)dy, (int)(0u - dx), rj.y)
                       : make_int4((int)c, (int)(0u - dy), (int)dx, rj.y);
}

// FP32 record of the edge ri -> rj in the frame with origin (ox, oy) (see PM_BOUND_K).
__device__ __forceinline__ float4 fp32_record(int2 ri, int2 rj, int ox, int oy)
{
    const int dx = rj.x - ri.x, dy = rj.y - ri.y;
    const float fdx = __int2float_rn(dx), fdy = __int2float_rn(dy);
    const float X = __int2float_rn(ri.x - ox), Y = __int2float_rn(ri.y - oy);
    const float c = __fmaf_rn(X, fdy, -__fmul_rn(Y, fdx));
    return dy > 0 ? make_float4(c, fdy, fdx, __int_as_float(rj.y)) : make_float4(-c, -fdy, -fdx, __int_as_float(rj.y));
}

// The same FP32 record from int64 differences, for frames of 2^31 or more (where the int32
// differences of fp32_record would wrap): the four inputs are rounded from exact integers as in
// fp32_record, so the same bound holds.  (c, a, b) = s (X d_y - Y d_x), |d_y|, s d_x.
__device__ __forceinline__ float3 fp32_record_ll(int2 ri, int2 rj, int ox, int oy)
{
    const long long dx = (long long)rj.x - ri.x, dy = (long long)rj.y - ri.y;
    const float fdx = __ll2float_rn(dx), fdy = __ll2float_rn(dy);
    const float X = __ll2float_rn((long long)ri.x - ox), Y = __ll2float_rn((long long)ri.y - oy);
    const float c = __fmaf_rn(X, fdy, -__fmul_rn(Y, fdx));
    return dy > 0 ? make_float3(c, fdy, fdx) : make_float3(-c, -fdy, -fdx);
}

}  // namespace pipdev
