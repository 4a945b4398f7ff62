// FP32-filtered classification with an exact integer recheck (pip_classify).
//
// Method section, steps 2-7 with Constraint 1.  For the edge R_i -> R_j of a polygon and a
// candidate point p, the crossing counts when the straddle test (y_i > p_y) != (y_j > p_y)
// holds (int32, exact) and sign(d_y) * det > 0, where det = (x_i - p_x) d_y - (y_i - p_y) d_x
// is the paper's side test (p - R_i) . n up to the sign fixed by orienting n so that
// n_x >= 0.  Parity of the count = inside bit.
//
// Local frame and FP32 evaluation.  A polygon (or one tile of a large polygon together with
// the tile's candidate points) gets an integer origin o at the centre of a box holding every
// vertex and point used with it; M_x, M_y bound |x - o_x|, |y - o_y| over that box.  Per
// edge the staging pass stores
//     c' = s (X_i d_y - Y_i d_x)   (X = x - o_x, Y = y - o_y, s = sign(d_y))
//     a = |d_y|,  b = s d_x
// and per (point, edge) pair the kernel evaluates t = fma(P_y, b, fma(-P_x, a, c')) with
// P = p - o rounded to FP32, so that t approximates s * det.  The record is formed in FP32
// from the exact integer differences (int64 and double when the box is 2^30 or more wide):
// rounding the four record inputs, the product Y d_x and the fused X d_y - Y d_x, then P_x,
// P_y and the two per-pair fused operations, costs at most 5u|X d_y| + 6u|Y d_x| +
// 4u|P_x d_y| + 3u|P_y d_x| (+ O(u^2)) <= 12u (M_x H + M_y W), u = 2^-24, H and W the box's
// height and width (>= |d_y|, |d_x| of every edge in it).  The bound B = 13u (M_x H + M_y W),
// evaluated with upward rounding, dominates it: |t| > B implies sign(t) = sign(s det) and
// det != 0, and only a straddling pair with |t| <= B needs the exact 64/128-bit recheck,
// which runs in place.  A point outside its polygon's closed bounding box is outside the
// polygon (the number of straddling edges is even and every crossing lies on one side of
// p), so it skips the edge loop.
//
// Two kernels, launched back to back on the caller's stream:
//
// k_pip_pipe -- polygon-major, producer/consumer.  A CTA takes chunks of 128 consecutive
//   polygons, so that every array it reads is one contiguous range: the chunk's vertex and
//   candidate offsets, its vertices and its candidate ids; only the candidate points are
//   gathered.  One producer warp cuts each chunk into passes (runs of whole polygons with at
//   most 1,024 vertices and 1,024 candidates) and stages a pass's offsets, vertices and
//   gathered points into one of two shared-memory stages with cp.async, while seven consumer
//   warps classify the previous pass: bounding box, frame and bound per polygon, FP32 edge
//   records per edge, then a queue of the candidates inside their polygon's box (polygons of
//   at most 8 edges from the front, longer ones from the back, so that a warp's lanes walk
//   similar edge counts) and the edge loop.  Named barriers hand stages back and forth.
//   Results are packed into shared words and written out; the first and last word of a pass
//   may be shared with a neighbouring pass, so those are written with a masked AND/OR pair
//   that sets exactly the pass's own bits (no zero-fill pass is needed).  Polygons with more
//   than 1,024 vertices or more than 2^18 (candidate, edge) pairs get bit 0 here and go on a
//   device-side list.
//
// k_pip_large -- the listed polygons.  Work items (polygon, block of 256*PPT candidates,
//   slice of edges) are taken from the list by atomic counters; the CTA streams the slice
//   through shared memory in tiles of T edges, each tile framed by the union of its vertices
//   and the block's candidate points, and XORs the partial parities into the output words
//   (stream order puts it after the first kernel's writes).  Its last CTA empties the list for
//   the next call.  With more large polygons than the list holds, it falls back to a scan over
//   all polygons.
#include <algorithm>
#include <type_traits>

#include "pip_device.cuh"
#include "pip_launch.h"

namespace pipdev {


// large-polygon kernel geometry
constexpr int LG_THREADS = 256;

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
__device__ __noinline__ float4 wide_record(int2 ri, int2 rj, int ox, int oy)
{
    const long long dx = (long long)rj.x - ri.x, dy = (long long)rj.y - ri.y;
    const float c = dy == 0 ? 0.f : edge_c(ri, dx, dy, ox, oy, 1);
    return dy > 0 ? make_float4(c, __ll2float_rn(dy), __ll2float_rn(dx), __int_as_float(rj.y))
                  : make_float4(c, __ll2float_rn(-dy), __ll2float_rn(-dx), __int_as_float(rj.y));
}


// Exact parity of p over the edges e0..e1-1 of staged vertices v, edge e running from v[e]
// to v[e + 1], or to v[e0] for the last edge when `wrap`.  Rare path: kept out of line.
__device__ __noinline__ int exact_parity(const int2 *v, int e0, int e1, bool wrap, int2 p)
{
    int parity = 0;
    for (int e = e0; e < e1; ++e) {
        const int nx = (wrap && e + 1 == e1) ? e0 : e + 1;
        const int2 ri = v[e], rj = v[nx];
        if ((ri.y > p.y) != (rj.y > p.y)) parity ^= exact_edge_counts(p.x, p.y, ri.x, ri.y, rj.x, rj.y);
    }
    return parity;
}

// =============================================================================================
// k_pip_pipe -- small polygons, polygon-major, producer/consumer
// =============================================================================================

// Bound factor of the FP32 records: rounding the four record inputs, the product Y d_x and the
// fused X d_y - Y d_x, then P_x, P_y and the two per-pair fused operations, costs at most
// 5u|X d_y| + 6u|Y d_x| + 4u|P_x d_y| + 3u|P_y d_x| (+ O(u^2)) <= 12u (M_x H + M_y W), with H, W
// the polygon's height and width (>= |d_y|, |d_x| of every edge).
constexpr float PM_BOUND_K = 7.748603820800781e-07f;     // 13 * 2^-24 (exact in FP32)
constexpr int PM_THREADS = 256;     // warps 0-6 consume, warp 7 produces
constexpr int PM_CONS = 224;
constexpr int PM_NP = 128;          // polygons per chunk (and at most per pass)
constexpr int PM_TV = 1024;         // staged vertices per pass
constexpr int PM_TC = 1024;         // staged candidates per pass
constexpr int PM_SHORT = 8;         // polygons of at most this many edges share warps
constexpr int PM_LARGE_M = 1024;    // polygons above this many vertices go to k_pip_large
constexpr long long PM_LARGE_W = 1LL << 18;   // ... and those with more (candidates x vertices)
// named barriers (0 is __syncthreads)
constexpr int BAR_CONS = 1, BAR_FULL = 2, BAR_EMPTY = 4;

__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }

template <typename CI>
struct __align__(16) PipeStage {
    int2 v[PM_TV + 2];              // the pass's vertices
    int2 pts[PM_TC];                // the pass's candidate points
    CI co[PM_NP + 1];               // candidate offsets of the pass's polygons
    int po[PM_NP + 1];              // vertex offsets (global)
    int kind;                       // 0 end, 1 run of small polygons, 2 one large polygon
    int kg0;                        // global index of the pass's polygon 0
    int np;                         // polygons in the pass
    int nc;                         // candidates [cb0, cb0 + nc)
    CI cb0;
};

template <typename CI>
struct __align__(16) PipeSmem {
    PipeStage<CI> st[2];
    // consumer-private
    float4 rec[PM_TV];
    int4 pbox[PM_NP];
    int4 pfr[PM_NP];                // ox, oy, bound (float bits), wide
    unsigned short vp[PM_TV];
    unsigned short cp[PM_TC];
    unsigned short queue[PM_TC];
    unsigned words[PM_TC / 32 + 2];
    // producer-private
    int ids[PM_TC];
    int ppo[PM_NP + 1];
    CI pco[PM_NP + 1];
    unsigned plg[PM_NP / 32];
};

__device__ __forceinline__ bool pm_is_large(long long m, long long n)
{
    return m > PM_LARGE_M || m * n > PM_LARGE_W;
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

template <bool DENSE>
__global__ void __launch_bounds__(PM_THREADS, 3) k_pip_pipe(ClassifyArgs a, long long total_bits, LargeList *ll,
                                                            int lcap)
{
    using CI = typename std::conditional<DENSE, long long, int>::type;
    extern __shared__ __align__(16) unsigned char dsm[];
    PipeSmem<CI> &sm = *reinterpret_cast<PipeSmem<CI> *>(dsm);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int P = a.n_polys;
    const CI W32 = (CI)(a.words_per_poly * 32);
    const CI NPTS = (CI)a.n_points;
    const int nchunk = (P + PM_NP - 1) / PM_NP;

    if (wid == 7) {
        // ================================ producer ================================
        if (!DENSE && blockIdx.x == 0 && lane == 0 && P > 0) {
            // bits past the last candidate in the final word are 0
            const long long C = __ldg(a.cand_offsets + P);
            if (C & 31) masked_store(a.out_bits + (C >> 5), ~((1u << (C & 31)) - 1u), 0u);
        }
        int j = 0;   // pass counter
        // claim stage j & 1 (after the consumers released pass j - 2)
        auto begin = [&]() -> PipeStage<CI> & {
            if (j >= 2) bar_sync(BAR_EMPTY + (j & 1), PM_THREADS);
            return sm.st[j & 1];
        };
        auto publish = [&]() {
            cp_async_wait_all();
            __threadfence_block();
            __syncwarp();
            bar_arrive(BAR_FULL + (j & 1), PM_THREADS);
            ++j;
        };
        // fill a stage with polygons [p, q) of the chunk and candidates [cb0, cb0 + nc)
        auto fill = [&](PipeStage<CI> &S, int k0, int p, int q, int kind, CI cb0, int nc) {
            if (lane == 0) { S.kind = kind; S.kg0 = k0 + p; S.np = q - p; S.nc = nc; S.cb0 = cb0; }
            for (int t = lane; t <= q - p; t += 32) { S.po[t] = sm.ppo[p + t]; S.co[t] = sm.pco[p + t]; }
            if (kind != 1) return;
            const int vb = sm.ppo[p], nv = sm.ppo[q] - vb;
            for (int i = lane; i < nv; i += 32) cp_async8(&S.v[i], a.verts + vb + i);
            if (!DENSE) {
                for (int i = lane; i < nc; i += 32) cp_async4(&sm.ids[i], a.cand_ids + cb0 + i);
                cp_async_commit();
                cp_async_wait_all();
                __syncwarp();
            }
            for (int i = lane; i < nc; i += 32) {
                CI pid;
                if (DENSE) {
                    const CI c = cb0 + i;
                    pid = c - (c / W32) * W32;
                } else {
                    pid = sm.ids[i];
                }
                if (pid < NPTS) cp_async8(&S.pts[i], a.points + pid);
            }
            cp_async_commit();
        };
        for (int ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
            const int k0 = ch * PM_NP;
            const int np = min(PM_NP, P - k0);
            for (int t = lane; t <= np; t += 32) {
                cp_async4(&sm.ppo[t], a.poly_offsets + k0 + t);
                if (!DENSE) cp_async4(&sm.pco[t], a.cand_offsets + k0 + t);
            }
            cp_async_commit();
            cp_async_wait_all();
            __syncwarp();
            if (DENSE)
                for (int t = lane; t <= np; t += 32) sm.pco[t] = (CI)(k0 + t) * W32;
            __syncwarp();
            #pragma unroll
            for (int b = 0; b < PM_NP / 32; ++b) {
                const int q = 32 * b + lane;
                bool lg = false;
                if (q < np) {
                    const long long n = DENSE ? min((long long)NPTS, (long long)W32) : (long long)(sm.pco[q + 1] - sm.pco[q]);
                    lg = pm_is_large(sm.ppo[q + 1] - sm.ppo[q], n);
                }
                const unsigned m = __ballot_sync(FULL, lg);
                if (lane == 0) sm.plg[b] = m;
            }
            __syncwarp();
            int p = 0;
            while (p < np) {
                if ((sm.plg[p >> 5] >> (p & 31)) & 1u) {
                    PipeStage<CI> &S = begin();
                    fill(S, k0, p, p + 1, 2, (CI)sm.pco[p], 0);
                    publish();
                    ++p;
                    continue;
                }
                // run [p, q): small polygons, vertices <= PM_TV, candidates <= PM_TC
                int q = p + 1;
                for (int base = p + 1; base <= np; base += 32) {
                    const int e = base + lane;
                    const bool ok = e <= np && sm.ppo[e] - sm.ppo[p] <= PM_TV &&
                                    (long long)(sm.pco[e] - sm.pco[p]) <= PM_TC &&
                                    !((sm.plg[(e - 1) >> 5] >> ((e - 1) & 31)) & 1u);
                    const unsigned bm = __ballot_sync(FULL, ok);
                    const int run = bm == FULL ? 32 : __ffs(~bm) - 1;
                    if (run > 0) q = base + run - 1;
                    if (run < 32) break;
                }
                q = max(q, p + 1);
                const CI c0 = (CI)sm.pco[p], c1 = (CI)sm.pco[q];
                if (c1 - c0 <= PM_TC) {
                    PipeStage<CI> &S = begin();
                    fill(S, k0, p, q, 1, c0, (int)(c1 - c0));
                    publish();
                } else {   // one polygon with more candidates than a pass holds
                    for (CI cb = c0; cb < c1; cb += PM_TC) {
                        PipeStage<CI> &S = begin();
                        fill(S, k0, p, p + 1, 1, cb, (int)min((CI)PM_TC, c1 - cb));
                        publish();
                    }
                }
                p = q;
            }
        }
        {
            PipeStage<CI> &S = begin();
            if (lane == 0) S.kind = 0;
            publish();
        }
        // the consumers' release of the last real pass (j - 2 after the end marker's ++j)
        if (j >= 2) bar_sync(BAR_EMPTY + (j & 1), PM_THREADS);
        return;
    }

    // ================================ consumers ================================
    unsigned st_cand = 0, st_rej = 0, st_fbp = 0;
    for (int j = 0;; ++j) {
        bar_sync(BAR_FULL + (j & 1), PM_THREADS);
        PipeStage<CI> &S = sm.st[j & 1];
        const int kind = S.kind;
        if (kind == 0) break;
        const int np = S.np, nc = S.nc;
        const CI cb0 = S.cb0;
        if (kind == 2) {
            // bits 0 here (k_pip_large XORs the parities in later); the list gets the polygon
            const CI cbeg = S.co[0], cfin = S.co[1];
            if (tid == 0 && cfin > cbeg && NPTS > 0) {
                const int idx = atomicAdd(&ll->count, 1);
                if (idx < lcap) {
                    large_entries(ll)[idx] = S.kg0;
                    large_taken(ll, lcap)[idx] = 0;
                } else {
                    atomicExch(&ll->overflow, 1);
                }
            }
            const CI w0 = cbeg >> 5, w1 = (cfin + 31) >> 5;
            for (CI wd = w0 + tid; wd < w1; wd += PM_CONS) {
                const int lo = (int)(max(cbeg, wd * 32) - wd * 32), hi = (int)(min(cfin, wd * 32 + 32) - wd * 32);
                masked_store(a.out_bits + wd, range_mask(lo, hi), 0u);
            }
            __threadfence_block();
            bar_arrive(BAR_EMPTY + (j & 1), PM_THREADS);
            continue;
        }
        const int vbase = S.po[0];
        const int nv = S.po[np] - vbase;
        // ---- bounding boxes and frames, one thread per polygon
        for (int q = tid; q < np; q += PM_CONS) {
            const int e0 = S.po[q] - vbase, e1 = S.po[q + 1] - vbase;
            int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
            for (int i = e0; i < e1; ++i) {
                const int2 v = S.v[i];
                x0 = min(x0, v.x); y0 = min(y0, v.y); x1 = max(x1, v.x); y1 = max(y1, v.y);
                sm.vp[i] = (unsigned short)q;
            }
            const unsigned W = (unsigned)x1 - (unsigned)x0, H = (unsigned)y1 - (unsigned)y0;
            const unsigned Mx = W - (W >> 1), My = H - (H >> 1);
            const float B = __fmul_ru(PM_BOUND_K, __fadd_ru(__fmul_ru(__uint2float_ru(Mx), __uint2float_ru(H)),
                                                             __fmul_ru(__uint2float_ru(My), __uint2float_ru(W))));
            sm.pfr[q] = make_int4(x0 + (int)(W >> 1), y0 + (int)(H >> 1), __float_as_int(B),
                                  (Mx >= (1u << 30)) | (My >= (1u << 30)));
            sm.pbox[q] = make_int4(x0, y0, x1, y1);
            // candidate slots of this polygon in the pass
            const int s0 = (int)(max(S.co[q], cb0) - cb0);
            const int s1 = (int)(min(S.co[q + 1], cb0 + (CI)nc) - cb0);
            int s1v = s1;
            if (DENSE) s1v = (int)max((CI)s0, min((CI)s1 + cb0, S.co[q] + NPTS) - cb0);
            for (int s = s0; s < s1v; ++s) sm.cp[s] = (unsigned short)q;
            for (int s = s1v; s < s1; ++s) sm.cp[s] = 0xffff;   // dense padding
        }
        for (int t = tid; t < PM_TC / 32 + 2; t += PM_CONS) sm.words[t] = 0;
        bar_sync(BAR_CONS, PM_CONS);
        // ---- edge records, one thread per edge (FP32 unless the frame is 2^30 wide)
        for (int i = tid; i < nv; i += PM_CONS) {
            const int q = sm.vp[i];
            const int nx = (i + 1 == S.po[q + 1] - vbase) ? S.po[q] - vbase : i + 1;
            const int2 ri = S.v[i], rj = S.v[nx];
            const int4 f = sm.pfr[q];
            float4 rec;
            if (!f.w) {
                const int dx = rj.x - ri.x, dy = rj.y - ri.y;
                const float fdx = __int2float_rn(dx), fdy = __int2float_rn(dy);
                const float X = __int2float_rn(ri.x - f.x), Y = __int2float_rn(ri.y - f.y);
                const float c = __fmaf_rn(X, fdy, -__fmul_rn(Y, fdx));
                rec = dy > 0 ? make_float4(c, fdy, fdx, __int_as_float(rj.y))
                             : make_float4(-c, -fdy, -fdx, __int_as_float(rj.y));
            } else {
                rec = wide_record(ri, rj, f.x, f.y);
            }
            sm.rec[i] = rec;
        }
        bar_sync(BAR_CONS, PM_CONS);
        // ---- the edge loop, candidates in order (one per thread): lanes of a warp share one or
        //      two polygons.  A point outside its polygon's closed box is outside: its y is
        //      replaced by INT_MAX, so no edge straddles its ray and the loop leaves 0.
        const int sh = (int)(cb0 & 31);   // bit of candidate cb0 within its word
        for (int i0 = 0; i0 < nc; i0 += PM_CONS) {   // warp-uniform rounds (ballot below)
            const int i = i0 + tid;
            const int q = i < nc ? sm.cp[i] : 0xffff;
            int parity = 0;
            if (q != 0xffff) {
                const int2 p = S.pts[i];
                const int4 b = sm.pbox[q];
                const bool in = p.x >= b.x && p.x <= b.z && p.y >= b.y && p.y <= b.w;
                ++st_cand;
                st_rej += !in;
                const int py = in ? p.y : INT_MAX;
                const int4 f = sm.pfr[q];
                const int e0 = S.po[q] - vbase, e1 = S.po[q + 1] - vbase;
                const float B = __int_as_float(f.z);
                const float Px = __ll2float_rn((long long)p.x - f.x), Py = __ll2float_rn((long long)p.y - f.y);
                bool sp = S.v[e0].y > py;
                bool unc = false;
                #pragma unroll 2
                for (int e = e0; e < e1; ++e) {
                    const float4 q4 = sm.rec[e];
                    const bool sn = __float_as_int(q4.w) > py;
                    const bool st = sn != sp;
                    sp = sn;
                    float tt = __fmaf_rn(-Px, q4.y, q4.x);
                    tt = __fmaf_rn(Py, q4.z, tt);
                    parity ^= (int)(st & (tt > 0.f));
                    unc |= st & (fabsf(tt) <= B);
                }
                if (unc) {
                    ++st_fbp;
                    parity = exact_parity(S.v, e0, e1, true, p);
                }
            }
            // pack: this warp's 32 consecutive candidates start at bit sh + i0 + 32 wid
            const unsigned bits = __ballot_sync(FULL, parity);
            if (lane == 0 && bits) {
                const int bpos = sh + i0 + 32 * wid;
                atomicOr(&sm.words[bpos >> 5], bits << (bpos & 31));
                if (bpos & 31) atomicOr(&sm.words[(bpos >> 5) + 1], bits >> (32 - (bpos & 31)));
            }
        }
        // the stage's data is no longer needed
        __threadfence_block();
        bar_arrive(BAR_EMPTY + (j & 1), PM_THREADS);
        bar_sync(BAR_CONS, PM_CONS);
        // ---- write the pass's words: bits [sh, sh + nc) of words cb0 >> 5 ...
        const int nwd = (sh + nc + 31) >> 5;
        for (int t = tid; t < nwd; t += PM_CONS)
            masked_store(a.out_bits + (cb0 >> 5) + t, range_mask(t == 0 ? sh : 0, min(32, sh + nc - 32 * t)),
                         sm.words[t]);
    }
    if (a.stats) {
        st_rej += st_cand;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st_cand += __shfl_down_sync(FULL, st_cand, o);
            st_rej += __shfl_down_sync(FULL, st_rej, o);
            st_fbp += __shfl_down_sync(FULL, st_fbp, o);
        }
        if (lane == 0) {
            if (st_cand) atomicAdd(a.stats + ST_CANDIDATES, (unsigned long long)st_cand);
            if (st_rej) atomicAdd(a.stats + ST_BBOX_REJECTS, (unsigned long long)st_rej);
            if (st_fbp) atomicAdd(a.stats + ST_FALLBACK_POINTS, (unsigned long long)st_fbp);
        }
    }
}

// =============================================================================================
// k_pip_large
// =============================================================================================

size_t filtered_smem_bytes(int T)
{
    // records float4[T], vertices int2[T + 1]
    size_t b = (size_t)T * 16 + (size_t)(T + 1) * 8;
    return (b + 15) & ~(size_t)15;
}

// Parities of a thread's PPT candidates over the tile's edges 0..nt-1 (edge e from s_v[e] to
// s_v[e + 1]; record e holds the edge's bound in .w): one shared record load serves every
// candidate, and the PPT chains are independent.  Candidates whose FP32 sign came within the
// bound of zero are redone exactly.
template <int PPT>
__device__ __forceinline__ void tile_parity_multi(const float4 *__restrict__ s_rec, const int2 *__restrict__ s_v,
                                                  int nt, const int2 (&p)[PPT], const bool (&ok)[PPT], int ox,
                                                  int oy, int (&par)[PPT], unsigned long long &n_fb_pts)
{
    // one candidate at a time: the side of the previous vertex is carried in one predicate
    #pragma unroll 1
    for (int r = 0; r < PPT; ++r) {
        if (!ok[r]) continue;
        const float Px = __ll2float_rn((long long)p[r].x - ox);
        const float Py = __ll2float_rn((long long)p[r].y - oy);
        const int py = p[r].y;
        bool sp = s_v[0].y > py;
        int pr = 0, unc = 0;
        #pragma unroll 2
        for (int e = 0; e < nt; ++e) {
            const float4 q = s_rec[e];
            const bool sn = s_v[e + 1].y > py;
            const bool st = sn != sp;
            sp = sn;
            float t = __fmaf_rn(-Px, q.y, q.x);
            t = __fmaf_rn(Py, q.z, t);
            pr ^= (int)(st & (t > 0.f));
            unc += (int)(st & (fabsf(t) <= q.w));
        }
        if (unc) {
            ++n_fb_pts;
            pr = exact_parity(s_v, 0, nt, false, p[r]);
        }
        par[r] ^= pr;
    }
}

// Edges per work item of a large polygon with m edges and nb candidate blocks: slices short
// enough that the listed polygons give every CTA about two items, never below 256 edges or
// above 16,384, a multiple of 32.  Every CTA derives the same value.
__device__ __forceinline__ int slice_edges(long long m, long long nb, int nlarge, int grid)
{
    const long long want = (2LL * grid + max(nlarge, 1) - 1) / max(nlarge, 1);
    const long long ns = max(1LL, (want + nb - 1) / max(nb, 1LL));
    long long es = (m + ns - 1) / ns;
    es = min(16384LL, max(256LL, es));
    return (int)((es + 31) & ~31LL);
}

template <int PPT>
__global__ void __launch_bounds__(LG_THREADS) k_pip_large(ClassifyArgs a, long long total_bits, LargeList *ll,
                                                         int lcap, int T)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *s_rec = reinterpret_cast<float4 *>(dsm);
    int2 *s_v = reinterpret_cast<int2 *>(s_rec + T);
    __shared__ int s_item[4];          // polygon, candidate block, edge slice, valid
    __shared__ int s_pb[4], s_tb[4];
    __shared__ int s_tf[4];            // tile frame: ox, oy, bound (float bits), wide

    constexpr int CB = LG_THREADS * PPT;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool dense = a.cand_offsets == nullptr;
    const int P = a.n_polys;
    const long long W32 = a.words_per_poly * 32;
    unsigned long long st_cand = 0, st_fbp = 0;
    const int count = *((volatile int *)&ll->count);
    const bool scan = *((volatile int *)&ll->overflow) != 0;
    long long scan_k = blockIdx.x;   // overflow mode: polygons blockIdx.x, + gridDim.x, ...
    int scan_item = 0;

    while (true) {
        if (tid == 0) {
            s_item[3] = 0;
            if (!scan) {
                while (true) {
                    const int e = *((volatile int *)&ll->cursor);
                    if (e >= min(count, lcap)) break;
                    const int k = large_entries(ll)[e];
                    const long long cs = dense ? k * W32 : (long long)a.cand_offsets[k];
                    const long long ce = dense ? cs + W32 : (long long)a.cand_offsets[k + 1];
                    const long long m = (long long)a.poly_offsets[k + 1] - a.poly_offsets[k];
                    const long long nb = (ce - cs + CB - 1) / CB;
                    const int ES = slice_edges(m, nb, count, gridDim.x);
                    const long long ns = (m + ES - 1) / ES;
                    const int it = atomicAdd(large_taken(ll, lcap) + e, 1);
                    if ((long long)it < nb * ns) {
                        s_item[0] = k; s_item[1] = (int)(it / ns); s_item[2] = (int)(it % ns); s_item[3] = ES;
                        break;
                    }
                    atomicCAS(&ll->cursor, e, e + 1);
                }
            } else {
                while (scan_k < P) {
                    const int k = (int)scan_k;
                    const long long cs = dense ? k * W32 : (long long)a.cand_offsets[k];
                    const long long ce = dense ? cs + W32 : (long long)a.cand_offsets[k + 1];
                    const long long m = (long long)a.poly_offsets[k + 1] - a.poly_offsets[k];
                    const long long n = dense ? min((long long)a.n_points, W32) : ce - cs;
                    const long long nb = pm_is_large(m, n) ? (ce - cs + CB - 1) / CB : 0;
                    const int ES = slice_edges(m, nb, count, gridDim.x);
                    const long long ns = (m + ES - 1) / ES;
                    if (scan_item < nb * ns) {
                        s_item[0] = k; s_item[1] = (int)(scan_item / ns); s_item[2] = (int)(scan_item % ns);
                        s_item[3] = ES;
                        ++scan_item;
                        break;
                    }
                    scan_k += gridDim.x;
                    scan_item = 0;
                }
            }
        }
        __syncthreads();
        if (!s_item[3]) break;
        const int k = s_item[0];
        const long long cs = dense ? k * W32 : (long long)a.cand_offsets[k];
        const long long ce = dense ? cs + W32 : (long long)a.cand_offsets[k + 1];
        const long long cb0 = cs + (long long)s_item[1] * CB, cb1 = min(cb0 + CB, ce);
        const int base = a.poly_offsets[k];
        const int m = a.poly_offsets[k + 1] - base;
        const int ES = s_item[3];
        const int ea = s_item[2] * ES, eb = min(m, ea + ES);
        int2 pt[PPT];
        bool ok[PPT];
        int par[PPT];
        if (tid == 0) { s_pb[0] = INT_MAX; s_pb[1] = INT_MAX; s_pb[2] = INT_MIN; s_pb[3] = INT_MIN; }
        __syncthreads();
        #pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const long long c = cb0 + tid + r * LG_THREADS;
            ok[r] = c < cb1;
            par[r] = 0;
            pt[r] = make_int2(0, 0);
            if (ok[r]) {
                long long pid = dense ? c - (long long)k * W32 : (long long)__ldg(a.cand_ids + c);
                if (pid >= a.n_points) ok[r] = false;
                else pt[r] = __ldg(a.points + pid);
            }
            if (ok[r]) {
                atomicMin(&s_pb[0], pt[r].x); atomicMin(&s_pb[1], pt[r].y);
                atomicMax(&s_pb[2], pt[r].x); atomicMax(&s_pb[3], pt[r].y);
                if (s_item[2] == 0) ++st_cand;
            }
        }
        __syncthreads();
        for (int e0 = ea; s_pb[0] <= s_pb[2] && e0 < eb; e0 += T) {
            const int nt = min(T, eb - e0);
            if (tid == 0) { s_tb[0] = s_pb[0]; s_tb[1] = s_pb[1]; s_tb[2] = s_pb[2]; s_tb[3] = s_pb[3]; }
            for (int i = tid; i <= nt; i += LG_THREADS) {
                int g = e0 + i;
                if (g >= m) g -= m;
                s_v[i] = __ldg(a.verts + base + g);
            }
            __syncthreads();
            int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
            for (int i = tid; i <= nt; i += LG_THREADS) {
                const int2 v = s_v[i];
                x0 = min(x0, v.x); y0 = min(y0, v.y); x1 = max(x1, v.x); y1 = max(y1, v.y);
            }
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x0 = min(x0, __shfl_xor_sync(FULL, x0, o)); y0 = min(y0, __shfl_xor_sync(FULL, y0, o));
                x1 = max(x1, __shfl_xor_sync(FULL, x1, o)); y1 = max(y1, __shfl_xor_sync(FULL, y1, o));
            }
            if (lane == 0) {
                atomicMin(&s_tb[0], x0); atomicMin(&s_tb[1], y0); atomicMax(&s_tb[2], x1); atomicMax(&s_tb[3], y1);
            }
            __syncthreads();
            if (tid == 0) {
                // box of the tile's vertices and the block's points, origin at its centre
                const unsigned W = (unsigned)s_tb[2] - (unsigned)s_tb[0], H = (unsigned)s_tb[3] - (unsigned)s_tb[1];
                const unsigned Mx = W - (W >> 1), My = H - (H >> 1);
                s_tf[0] = s_tb[0] + (int)(W >> 1);
                s_tf[1] = s_tb[1] + (int)(H >> 1);
                s_tf[2] = (int)Mx;   // as unsigned
                s_tf[3] = (int)My;
            }
            __syncthreads();
            const int ox = s_tf[0], oy = s_tf[1];
            const unsigned Mx = (unsigned)s_tf[2], My = (unsigned)s_tf[3];
            const bool wide = (Mx >= (1u << 30)) | (My >= (1u << 30));
            const float fMx = __uint2float_ru(Mx), fMy = __uint2float_ru(My);
            for (int i = tid; i < nt; i += LG_THREADS) {
                const int2 ri = s_v[i], rj = s_v[i + 1];
                float4 rec;
                if (!wide) {
                    const int dx = rj.x - ri.x, dy = rj.y - ri.y;
                    const float fdx = __int2float_rn(dx), fdy = __int2float_rn(dy);
                    const float X = __int2float_rn(ri.x - ox), Y = __int2float_rn(ri.y - oy);
                    const float c = __fmaf_rn(X, fdy, -__fmul_rn(Y, fdx));
                    rec = dy > 0 ? make_float4(c, fdy, fdx, 0.f) : make_float4(-c, -fdy, -fdx, 0.f);
                } else {
                    rec = wide_record(ri, rj, ox, oy);
                }
                // the edge's own bound 13u (M_x |d_y| + M_y |d_x|) (see PM_BOUND_K)
                const long long ady = llabs((long long)rj.y - ri.y), adx = llabs((long long)rj.x - ri.x);
                rec.w = __fmul_ru(PM_BOUND_K, __fadd_ru(__fmul_ru(fMx, __ll2float_ru(ady)), __fmul_ru(fMy, __ll2float_ru(adx))));
                s_rec[i] = rec;
            }
            __syncthreads();
            tile_parity_multi<PPT>(s_rec, s_v, nt, pt, ok, ox, oy, par, st_fbp);
            __syncthreads();
        }
        // XOR the partial parities into the output words (the block need not be word-aligned)
        #pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const long long cw = cb0 + (tid & ~31) + r * LG_THREADS;   // candidate of lane 0
            const unsigned bits = __ballot_sync(FULL, ok[r] && par[r]);
            if (lane == 0 && bits) {
                const int sh = (int)(cw & 31);
                atomicXor(a.out_bits + (cw >> 5), bits << sh);
                if (sh) {
                    const unsigned hi = bits >> (32 - sh);
                    if (hi) atomicXor(a.out_bits + (cw >> 5) + 1, hi);
                }
            }
        }
        __syncthreads();
    }
    if (a.stats) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st_cand += __shfl_down_sync(FULL, st_cand, o);
            st_fbp += __shfl_down_sync(FULL, st_fbp, o);
        }
        if (lane == 0) {
            if (st_cand) atomicAdd(a.stats + ST_CANDIDATES, st_cand);
            if (st_fbp) atomicAdd(a.stats + ST_FALLBACK_POINTS, st_fbp);
        }
    }
    // the last CTA to finish empties the list for the next call
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&ll->done, 1) == (int)gridDim.x - 1) {
            ll->count = 0;
            ll->cursor = 0;
            ll->overflow = 0;
            ll->done = 0;
            __threadfence();
        }
    }
}

// =============================================================================================
// launch
// =============================================================================================

template <typename K>
static int ensure_smem(K kernel, size_t smem, size_t *configured)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && configured[dev] < smem) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        configured[dev] = smem;
    }
    return 0;
}

template <bool DENSE>
static int launch_pipe_d(const ClassifyArgs &a, long long total_bits, LargeList *ll, int lcap, int n_sm,
                         cudaStream_t stream)
{
    using CI = typename std::conditional<DENSE, long long, int>::type;
    static size_t configured[64] = {0};
    static int blocks_per_sm[64] = {0};
    const size_t smem = sizeof(PipeSmem<CI>);
    int e = ensure_smem(k_pip_pipe<DENSE>, smem, configured);
    if (e) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && blocks_per_sm[dev] == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pip_pipe<DENSE>, PM_THREADS, smem) != cudaSuccess)
            nb = 1;
        blocks_per_sm[dev] = std::max(nb, 1);
    }
    const int bps = (dev >= 0 && dev < 64) ? blocks_per_sm[dev] : 1;
    const long long nchunk = ((long long)a.n_polys + PM_NP - 1) / PM_NP;
    const int grid = (int)std::max(1LL, std::min((long long)n_sm * bps, nchunk));
    k_pip_pipe<DENSE><<<grid, PM_THREADS, smem, stream>>>(a, total_bits, ll, lcap);
    return (int)cudaGetLastError();
}

template <int PPT>
static int launch_large_ppt(const ClassifyArgs &a, long long total_bits, LargeList *ll, int lcap, int T, int grid,
                            cudaStream_t stream)
{
    static size_t configured[64] = {0};
    const size_t smem = filtered_smem_bytes(T);
    int e = ensure_smem(k_pip_large<PPT>, smem, configured);
    if (e) return e;
    k_pip_large<PPT><<<grid, LG_THREADS, smem, stream>>>(a, total_bits, ll, lcap, T);
    return (int)cudaGetLastError();
}

int launch_filtered(const ClassifyArgs &a, long long total_bits, const Tuning &t, int n_sm, LargeList *ll, int lcap,
                    cudaStream_t stream)
{
    int e = a.cand_offsets ? launch_pipe_d<false>(a, total_bits, ll, lcap, n_sm, stream)
                           : launch_pipe_d<true>(a, total_bits, ll, lcap, n_sm, stream);
    if (e) return e;
    const int grid = n_sm * t.ctas_per_sm;
    switch (t.pts_per_thread) {
        case 1: return launch_large_ppt<1>(a, total_bits, ll, lcap, t.edge_tile, grid, stream);
        case 4: return launch_large_ppt<4>(a, total_bits, ll, lcap, t.edge_tile, grid, stream);
        default: return launch_large_ppt<2>(a, total_bits, ll, lcap, t.edge_tile, grid, stream);
    }
}

}  // namespace pipdev
