// Filtered classification (pip_classify): exact int32 or int64 tests for polygons whose box is
// below 2^31, an FP32 filter with an exact integer recheck for the rest.
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
// Exact int32 evaluation.  When a polygon's box is small (width, height < 2^30 and width x
// height < 2^30), det = (X_i - P_x) d_y - (Y_i - P_y) d_x of an in-box point is below 2^31 in
// magnitude, so the same record evaluated with wrapping 32-bit integer multiply-adds gives
// -sign(d_y) det exactly; the straddle test is the sign bit of (P_y - Y_j) XOR (P_y - Y_i).
// No filter and no recheck are needed for such polygons (building footprints, parcels).
//
// Exact int64 evaluation.  When the box is below 2^31 on both sides but too large for int32,
// the record (X_i, |d_y|, -s d_x, Y_j) holds int32 values in the box-centre frame and
// nt = (P_x - X_i)|d_y| + (P_y - Y_i)(-s d_x) = -s det is formed exactly from two 32 x 32 -> 64-bit
// products (every factor below 2^31; P_y - Y_i is the previous step's P_y - Y_j): again no filter
// and no recheck.  A run with any polygon
// outside the int32 test puts all its polygons on the int64 or FP32 test, so the lanes of a
// round walk at most two kinds of loop.  Only boxes of 2^31 or more use the FP32 filter.
//
// Two kernels, launched back to back on the caller's stream:
//
// k_pip_warp -- polygon-major, every warp on its own.  A warp takes chunks of 32 consecutive
//   polygons (lane = polygon, offsets in registers, the next chunk's loaded ahead) and cuts each
//   into runs of consecutive polygons with at most 256 vertices in all.  Per run it copies the
//   vertices into its own shared memory (cp.async) and forms the edge records (lane per edge)
//   and each polygon's box and arithmetic (lane per polygon).  The run's candidates are then
//   classified in slices of 256: the points are gathered into shared memory (cp.async; the next
//   slice's ids are loaded ahead), each candidate's polygon is found from a bitmap of polygon
//   starts, and 32 candidates at a time, one per lane, walk their polygons' edges in lockstep;
//   ballots pack the parities.  No barrier spans more than one warp, so the warps of an SM hide
//   one another's memory latency.  The first and last word of a slice may be shared with a
//   neighbouring slice, so those are written with a masked AND/OR pair that sets exactly the
//   slice's own bits (no zero-fill pass is needed).  Polygons with more than 256 vertices or
//   more than 2^18 (candidate, edge) pairs get bit 0 here and go on a device-side list.
//
// k_pip_large -- the listed polygons.  Work items (polygon, block of 256*PPT candidates,
//   slice of edges) are taken from the list by atomic counters; the CTA streams the slice
//   through shared memory in tiles of T edges (each tile's vertices by one bulk copy of the
//   tensor memory accelerator, completed on an mbarrier with a bounded wait; a CTA whose wait gives
//   up decides the rest of its pairs exactly from global memory), each tile framed
//   by the union of its vertices
//   and the block's candidate points (records scaled per edge by a power of two, so that one
//   uniform test flags the uncertain FP32 signs), and XORs the partial parities into the output
//   words (stream order puts it after the first kernel's writes).  With a y-slab index
//   (pip_classify_slab) an item is a candidate block whose points walk only their slab's edges.
//   Its last CTA empties the list for the next call.  With more large polygons than the list
//   holds, it falls back to a scan over all polygons.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "pip_device.cuh"
#include "pip_edge.cuh"
#include "pip_launch.h"

namespace pipdev {

// large-polygon kernel geometry
constexpr int LG_THREADS = 256;

// =============================================================================================
// k_pip_warp -- small polygons; every warp works on its own runs of consecutive polygons
// =============================================================================================

constexpr int WP_THREADS = 128;     // 4 independent warps per CTA
constexpr int WP_CTAS = 5;          // CTAs per SM (shared memory: 4 x 9.8 KB per CTA)

// WP_R: candidate rounds of 32 per slice (4 or 8; a tuning choice), WP_C = 32 WP_R candidates
template <int WP_R, int WP_C = 32 * WP_R>
struct __align__(16) WarpSmem {
    float4 rec[WP_V];               // edge records of the run (int32, int64 or FP32, per polygon)
    int2 v[WP_V];                   // the run's vertices
    int4 box[32];                   // per chunk polygon: closed bounding box
    int4 fr[32];                    // ox, oy, bound (float bits), e0 | e1 << 9 | mode << 18
    int2 pt[WP_C];                  // candidate points of the slice
    unsigned vstart[WP_V / 32 + 1]; // bit i: vertex i starts a polygon of the run, or i == nv
    unsigned char sp[WP_C];         // first candidate slot of a polygon -> chunk polygon
    unsigned char vp[WP_V];         // vertex -> chunk polygon
};

template <bool DENSE, bool VERIFY, int WP_R>
__global__ void __launch_bounds__(WP_THREADS, WP_CTAS) k_pip_warp(ClassifyArgs a, LargeList *ll, int lcap)
{
    using CI = typename std::conditional<DENSE, long long, int>::type;
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr int WP_C = 32 * WP_R;     // candidates of a slice
    WarpSmem<WP_R> &S = reinterpret_cast<WarpSmem<WP_R> *>(dsm)[threadIdx.x >> 5];
    pdl_trigger();   // the large-polygon kernel may launch now; it waits for this grid to finish
    const unsigned rec_base = (unsigned)__cvta_generic_to_shared(S.rec);
    const int lane = threadIdx.x & 31;
    const unsigned lemask = 0xffffffffu >> (31 - lane);   // lanes 0..lane
    const int P = a.n_polys;
    const CI W32 = (CI)(a.words_per_poly * 32);
    const long long NPTS = a.n_points;
    const int nchunk = (P + 31) >> 5;
    const int gw = blockIdx.x * (WP_THREADS / 32) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (WP_THREADS / 32);
    unsigned st_cand = 0, st_rej = 0, st_fbp = 0, st_err = 0, st_ver = 0;
    if (!DENSE && gw == 0 && lane == 0 && P > 0) {
        // bits past the last candidate in the final word are 0
        const long long C = __ldg(a.cand_offsets + P);
        if (C & 31) masked_store(a.out_bits + (C >> 5), ~((1u << (C & 31)) - 1u), 0u);
    }

    // offsets of a chunk (polygons k0 + lane), loaded one chunk ahead
    int f_pb = 0, f_pe = 0;
    CI f_cb = 0, f_ce = 0;
    auto fetch_chunk = [&](int c) {
        const int kk = (c << 5) + lane;
        if (c < nchunk && kk < P) {
            f_pb = __ldg(a.poly_offsets + kk);
            f_pe = __ldg(a.poly_offsets + kk + 1);
            if (DENSE) {
                f_cb = (CI)kk * W32;
                f_ce = f_cb + W32;
            } else {
                f_cb = __ldg(a.cand_offsets + kk);
                f_ce = __ldg(a.cand_offsets + kk + 1);
            }
        }
    };
    // candidate ids of the slice that starts at candidate nid_c0 (CSR), loaded one slice ahead
    const CI C_total = (!DENSE && P > 0) ? (CI)__ldg(a.cand_offsets + P) : 0;
    CI nid[WP_R];
    CI nid_c0 = -1;
    fetch_chunk(gw);

    for (int ch = gw; ch < nchunk; ch += nw) {
        // ---- the chunk: polygons k0 + lane, offsets in registers
        const int k0 = ch << 5, np = min(32, P - k0);
        const bool has = lane < np;
        const int pb = has ? f_pb : 0, pe = has ? f_pe : 0;
        const CI cb = has ? f_cb : 0, ce = has ? f_ce : 0;
        fetch_chunk(ch + nw);
        const long long nlen = DENSE ? min(NPTS, (long long)W32) : (long long)(ce - cb);
        const bool lg = has && is_large_polygon(pe - pb, nlen);
        const unsigned lgm = __ballot_sync(FULL, lg);
        if (lg && ce > cb && NPTS > 0) {
            const int idx = atomicAdd(&ll->count, 1);
            if (idx < lcap) {
                large_entries(ll)[idx] = k0 + lane;
                large_taken(ll, lcap)[idx] = 0;
            } else {
                atomicExch(&ll->overflow, 1);
            }
        }
        // large polygons' bits are 0 here; k_pip_large XORs their parities in afterwards (a dense
        // output is zeroed before this kernel)
        if (!DENSE)
            for (unsigned m = lgm; m; m &= m - 1) {
                const int l = __ffs(m) - 1;
                zero_bits(a.out_bits, (long long)__shfl_sync(FULL, cb, l), (long long)__shfl_sync(FULL, ce, l), lane);
            }

        int p = 0;
        while (p < np) {
            if ((lgm >> p) & 1u) { ++p; continue; }
            // ---- run [p, q): consecutive small polygons with <= WP_V vertices in all; their
            //      candidates are classified in slices of WP_C
            const int vb = __shfl_sync(FULL, pb, p);
            const CI cbp = __shfl_sync(FULL, cb, p);
            const bool ok = lane >= p && has && !lg && pe - vb <= WP_V;
            const unsigned okm = __ballot_sync(FULL, ok) >> p;
            const int q = p + max(1, __clz(__brev(~okm)));     // trailing ones of okm, at least 1
            const int nv = __shfl_sync(FULL, pe, q - 1) - vb;
            const CI cq = __shfl_sync(FULL, ce, q - 1);
            const bool mine = lane >= p && lane < q;            // this lane's polygon is in the run
            if (cq <= cbp) { p = q; continue; }                 // no candidates: nothing to write
            for (int i = lane; i < nv; i += 32) cp_async8(&S.v[i], a.verts + vb + i);
            cp_async_commit();
            // vertex i starts a polygon (or i == nv)
            if (lane <= WP_V / 32) S.vstart[lane] = 0;
            __syncwarp();
            if (mine && pe > pb) atomicOr(&S.vstart[(pb - vb) >> 5], 1u << ((pb - vb) & 31));
            if (lane == 0) atomicOr(&S.vstart[nv >> 5], 1u << (nv & 31));
            bool staged = false;
            bool run_all32 = true;   // every polygon of the run takes the int32 test

            for (CI c0 = cbp; c0 < cq; c0 += WP_C) {
                const int nc = (int)min((CI)WP_C, cq - c0);
                const CI dbase = DENSE ? (c0 - cbp) % W32 : 0;   // dense: polygon p starts at a multiple of W32
                // ---- candidate points of the slice to shared memory
                CI pid[WP_R];
                #pragma unroll
                for (int r = 0; r < WP_R; ++r) {
                    const int slot = 32 * r + lane;
                    pid[r] = -1;
                    if (slot < nc) {
                        if (DENSE) {
                            CI t = dbase + slot;               // (c0 + slot) mod W32
                            while (t >= W32) t -= W32;
                            pid[r] = t;
                        } else {
                            pid[r] = c0 == nid_c0 ? nid[r] : (CI)__ldg(a.cand_ids + c0 + slot);
                        }
                    }
                }
                unsigned validm = 0;
                #pragma unroll
                for (int r = 0; r < WP_R; ++r) {
                    if (pid[r] >= 0 && (long long)pid[r] < NPTS) {   // else past the slice, or dense padding
                        cp_async8(&S.pt[32 * r + lane], a.points + pid[r]);
                        validm |= 1u << r;
                    }
                }
                cp_async_commit();
                if (!DENSE) {   // the ids of the candidates that follow, for the next slice
                    nid_c0 = c0 + nc;
                    #pragma unroll
                    for (int r = 0; r < WP_R; ++r) {
                        const CI c = nid_c0 + 32 * r + lane;
                        nid[r] = c < C_total ? (CI)__ldg(a.cand_ids + c) : (CI)-1;
                    }
                }
                // ---- owners: a polygon whose candidates meet [c0, c0 + nc) marks its first slot;
                //      slot j belongs to the last mark at or before j
                int sword = -1;
                unsigned sbit = 0;
                if (mine && ce > c0 && cb < c0 + nc && ce > cb) {
                    const int s0 = (int)(max(cb, c0) - c0);
                    S.sp[s0] = (unsigned char)lane;
                    sword = s0 >> 5;
                    sbit = 1u << (s0 & 31);
                }
                if (!staged) {
                    staged = true;
                    asm volatile("cp.async.wait_group 1;\n" ::: "memory");     // the vertices
                    __syncwarp();
                    // ---- int32 records of the edges that do not close their polygon (lane per edge)
                    for (int i = lane; i + 1 < nv; i += 32)
                        if (!((S.vstart[(i + 1) >> 5] >> ((i + 1) & 31)) & 1u)) {
                            const int4 r4 = int32_record(S.v[i], S.v[i + 1]);
                            S.rec[i] = make_float4(__int_as_float(r4.x), __int_as_float(r4.y), __int_as_float(r4.z),
                                                   __int_as_float(r4.w));
                        }
                    __syncwarp();
                    // ---- per polygon (lane per polygon): box, arithmetic mode, closing edge; all of
                    //      its records in FP32 when the box is too large for the int32 test
                    int mode = MODE_INT32;
                    int4 fr4 = make_int4(0, 0, 0, 0), box4 = make_int4(0, 0, 0, 0);
                    const int e0 = pb - vb, e1 = pe - vb;
                    if (mine) {
                        int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
                        #pragma unroll 2
                        for (int i = e0; i < e1; ++i) {
                            const int2 v = S.v[i];
                            x0 = min(x0, v.x); y0 = min(y0, v.y); x1 = max(x1, v.x); y1 = max(y1, v.y);
                        }
                        const unsigned W = (unsigned)x1 - (unsigned)x0, H = (unsigned)y1 - (unsigned)y0;
                        const unsigned Mx = W - (W >> 1), My = H - (H >> 1);
                        int bound = 0;
                        if (!(W < (1u << 30) && H < (1u << 30) && (unsigned long long)W * H < (1ULL << 30))) {
                            if (W < (1u << 31) && H < (1u << 31)) {
                                mode = MODE_INT64;
                            } else {
                                mode = (Mx >= (1u << 30)) | (My >= (1u << 30)) ? MODE_WIDE : MODE_FP32;
                                bound = __float_as_int(__fmul_ru(
                                    PM_BOUND_K, __fadd_ru(__fmul_ru(__uint2float_ru(Mx), __uint2float_ru(H)),
                                                          __fmul_ru(__uint2float_ru(My), __uint2float_ru(W)))));
                            }
                        }
                        fr4 = make_int4(x0 + (int)(W >> 1), y0 + (int)(H >> 1), bound, e0 | (e1 << 9));
                        box4 = make_int4(x0, y0, x1, y1);
                    }
                    // a run with any polygon outside the int32 test puts its int32 polygons on the
                    // int64 test too, so that a round walks at most two kinds of loop
                    run_all32 = __all_sync(FULL, mode == MODE_INT32);
                    if (!run_all32 && mode == MODE_INT32) mode = MODE_INT64;
                    if (mine) {
                        S.fr[lane] = make_int4(fr4.x, fr4.y, fr4.z, fr4.w | (mode << 18));
                        S.box[lane] = box4;
                        if (mode == MODE_INT32 && e1 > e0) {
                            const int4 r4 = int32_record(S.v[e1 - 1], S.v[e0]);
                            S.rec[e1 - 1] = make_float4(__int_as_float(r4.x), __int_as_float(r4.y),
                                                        __int_as_float(r4.z), __int_as_float(r4.w));
                        }
                        if (!run_all32)
                            for (int i = e0; i < e1; ++i) S.vp[i] = (unsigned char)lane;
                    }
                    __syncwarp();
                    if (!run_all32) {
                        // int64 / FP32 / wide records, lane per edge, in each polygon's frame
                        for (int i = lane; i < nv; i += 32) {
                            const int4 f = S.fr[S.vp[i]];
                            const int e0 = f.w & 0x1ff, e1 = (f.w >> 9) & 0x1ff, md = f.w >> 18;
                            const int2 ri = S.v[i], rj = S.v[i + 1 == e1 ? e0 : i + 1];
                            if (md == MODE_INT64) {
                                // (X_i, |d_y|, -s d_x, Y_j), s = sign(d_y); every value below 2^31
                                const int dx = rj.x - ri.x, dy = rj.y - ri.y;
                                reinterpret_cast<int4 *>(S.rec)[i] =
                                    make_int4(ri.x - f.x, dy > 0 ? dy : -dy, dy > 0 ? -dx : dx, rj.y - f.y);
                            } else if (md == MODE_FP32) {
                                S.rec[i] = fp32_record(ri, rj, f.x, f.y);
                            } else {
                                S.rec[i] = wide_record(ri, rj, f.x, f.y);
                            }
                        }
                    }
                }
                cp_async_wait_all();
                __syncwarp();
                // ---- rounds: one candidate per lane; the lanes of a warp walk their polygons'
                //      edges in lockstep, a lane whose polygon has fewer edges repeating its last
                //      record (a repeated edge never straddles, so it adds nothing)
                const int sh = (int)(c0 & 31);
                unsigned mybits = 0;   // lane r keeps the ballot of round r
                int carry = 0;
                const int nr = (nc + 31) >> 5;
                #pragma unroll 1
                for (int r = 0; r < nr; ++r) {
                    const unsigned mk = __reduce_or_sync(FULL, sword == r ? sbit : 0u);
                    const unsigned below = mk & lemask;
                    const int own = below ? (int)S.sp[32 * r + 31 - __clz(below)] : carry;
                    carry = __shfl_sync(FULL, own, 31);
                    const bool valid = (validm >> r) & 1u;
                    const int2 p2 = S.pt[32 * r + lane];
                    const int4 b = S.box[own];
                    const int4 f = S.fr[own];
                    const bool in = valid && p2.x >= b.x && p2.x <= b.z && p2.y >= b.y && p2.y <= b.w;
                    st_cand += valid;
                    st_rej += valid && !in;
                    const int e0 = f.w & 0x1ff, e1 = (f.w >> 9) & 0x1ff, mode = f.w >> 18;
                    const bool go = in && e1 > e0;
                    int parity = 0;
                    const bool gi = go && mode == MODE_INT32;
                    const int ki = __reduce_max_sync(FULL, gi ? e1 - e0 : 0);
                    if (ki > 0) {
                        // nt = -sign(d_y) det exactly; the sign bit of (u_j ^ u_i) is the straddle
                        // test, u = p_y - y; a crossing counts when both sign bits are set
                        unsigned ad = rec_base + 16u * (unsigned)(gi ? e0 : 0);
                        const unsigned al = rec_base + 16u * (unsigned)(gi ? e1 - 1 : 0);
                        const unsigned px = (unsigned)p2.x, py = (unsigned)p2.y;
                        unsigned up = py - (unsigned)lds128(al).w;   // vertex e0
                        unsigned acc = 0;
                        #pragma unroll 4
                        for (int k = 0; k < ki; ++k) {
                            const unsigned acur = ad;
                            const int4 q4 = lds128(ad);
                            ad = __viaddmin_u32(ad, 16u, al);
                            const unsigned u = py - (unsigned)q4.w;
                            const unsigned nt = (unsigned)q4.x + px * (unsigned)q4.y + py * (unsigned)q4.z;
                            if (VERIFY && (int)(u ^ up) < 0) {   // a straddling edge: its exact test
                                const int e = (int)((acur - rec_base) >> 4);
                                const int2 ri = S.v[e], rj = S.v[e + 1 == e1 ? e0 : e + 1];
                                st_err += exact_edge_counts(p2.x, p2.y, ri.x, ri.y, rj.x, rj.y) != (int)(nt >> 31);
                                ++st_ver;
                            }
                            acc ^= (u ^ up) & nt;
                            up = u;
                        }
                        if (gi) parity = (int)(acc >> 31);
                    }
                    if (!run_all32) {
                        const bool g6 = go && mode == MODE_INT64;
                        const int k6 = __reduce_max_sync(FULL, g6 ? e1 - e0 : 0);
                        if (k6 > 0) {
                            // record (X_i, |d_y|, -s d_x, Y_j) in the frame; u = P_y - y, u_i carried from the
                            // step before and u_j from the record (so a repeated record adds nothing): the straddle
                            // test is the sign bit of u_i ^ u_j, and nt = (P_x - X_i)|d_y| + u_i (-s d_x) = -s det in
                            // int64 (every factor below 2^31); a crossing counts when both sign bits are set
                            unsigned ad = rec_base + 16u * (unsigned)(g6 ? e0 : 0);
                            const unsigned al = rec_base + 16u * (unsigned)(g6 ? e1 - 1 : 0);
                            const unsigned Px = (unsigned)p2.x - (unsigned)f.x, Py = (unsigned)p2.y - (unsigned)f.y;
                            unsigned up = Py - (unsigned)lds128(al).w;   // vertex e0 (end of the closing edge)
                            unsigned acc = 0;
                            #pragma unroll 2
                            for (int k = 0; k < k6; ++k) {
                                const int4 q4 = lds128(ad);
                                ad = __viaddmin_u32(ad, 16u, al);
                                const unsigned uj = Py - (unsigned)q4.w;   // P_y - Y_j; P_y - Y_i is up
                                const long long nt = (long long)(int)(Px - (unsigned)q4.x) * (long long)q4.y +
                                                     (long long)(int)up * (long long)q4.z;
                                acc ^= (up ^ uj) & (unsigned)((unsigned long long)nt >> 32);
                                up = uj;
                            }
                            if (g6) parity = (int)(acc >> 31);
                        }
                        const bool gf = go && mode >= MODE_FP32;
                        const int kf = __reduce_max_sync(FULL, gf ? e1 - e0 : 0);
                        if (kf > 0) {
                            unsigned ad = rec_base + 16u * (unsigned)(gf ? e0 : 0);
                            const unsigned al = rec_base + 16u * (unsigned)(gf ? e1 - 1 : 0);
                            const int py = p2.y;
                            const float B = __int_as_float(f.z);
                            const float Px = __ll2float_rn((long long)p2.x - f.x);
                            const float Py = __ll2float_rn((long long)p2.y - f.y);
                            bool sp = lds128(al).w > py;   // vertex e0
                            bool unc = false;
                            int par = 0;
                            #pragma unroll 2
                            for (int k = 0; k < kf; ++k) {
                                const unsigned acur = ad;
                                const int4 q4 = lds128(ad);
                                ad = __viaddmin_u32(ad, 16u, al);
                                const bool sn = q4.w > py;
                                const bool st = sn != sp;
                                sp = sn;
                                float tt = __fmaf_rn(-Px, __int_as_float(q4.y), __int_as_float(q4.x));
                                tt = __fmaf_rn(Py, __int_as_float(q4.z), tt);
                                if (VERIFY && gf && st && !(fabsf(tt) <= B)) {   // a trusted FP32 sign
                                    const int e = (int)((acur - rec_base) >> 4);
                                    const int2 ri = S.v[e], rj = S.v[e + 1 == e1 ? e0 : e + 1];
                                    st_err += exact_edge_counts(p2.x, p2.y, ri.x, ri.y, rj.x, rj.y) != (int)(tt > 0.f);
                                    ++st_ver;
                                }
                                par ^= (int)(st & (tt > 0.f));
                                unc |= st & (fabsf(tt) <= B);
                            }
                            if (gf) {
                                parity = par;
                                if (unc) {
                                    ++st_fbp;
                                    parity = exact_parity(S.v, e0, e1, true, p2);
                                }
                            }
                        }
                    }
                    const unsigned bits = __ballot_sync(FULL, parity);
                    if (lane == r) mybits = bits;
                }
                // ---- the slice's words: word k = bits_k << sh | bits_(k-1) >> (32 - sh), of which
                //      bits [sh, sh + nc) of words c0 >> 5 ... belong to the slice
                const unsigned prev = __shfl_up_sync(FULL, mybits, 1);
                unsigned myw = mybits << sh;
                if (sh && lane > 0) myw |= prev >> (32 - sh);
                const int nwd = (sh + nc + 31) >> 5;
                if (lane < nwd)
                    masked_store(a.out_bits + (c0 >> 5) + lane,
                                 range_mask(lane == 0 ? sh : 0, min(32, sh + nc - 32 * lane)), myw);
                __syncwarp();   // S.sp and S.pt are rewritten by the next slice
            }
            p = q;
        }
    }
    cp_async_wait_all();
    if (a.stats) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st_cand += __shfl_down_sync(FULL, st_cand, o);
            st_rej += __shfl_down_sync(FULL, st_rej, o);
            st_fbp += __shfl_down_sync(FULL, st_fbp, o);
            if (VERIFY) st_err += __shfl_down_sync(FULL, st_err, o);
            if (VERIFY) st_ver += __shfl_down_sync(FULL, st_ver, o);
        }
        if (lane == 0) {
            if (VERIFY && st_ver) atomicAdd(a.stats + ST_VERIFIED, (unsigned long long)st_ver);
            if (st_cand) atomicAdd(a.stats + ST_CANDIDATES, (unsigned long long)st_cand);
            if (st_rej) atomicAdd(a.stats + ST_BBOX_REJECTS, (unsigned long long)st_rej);
            if (st_fbp) atomicAdd(a.stats + ST_FALLBACK_POINTS, (unsigned long long)st_fbp);
            if (VERIFY && st_err) atomicAdd(a.stats + ST_FILTER_ERRORS, (unsigned long long)st_err);
        }
    }
}

// =============================================================================================
// k_pip_large
// =============================================================================================

size_t filtered_smem_bytes(int T)
{
    // records float4[T], vertices int2[T + 3] (a tile's T + 1 vertices, shifted by one when the
    // tile starts at an odd vertex so that the bulk copy lands on a 16-byte boundary)
    size_t b = (size_t)T * 16 + (size_t)(T + 3) * 8;
    return (b + 15) & ~(size_t)15;
}

// Parities of a thread's PPT candidates over the tile's edges 0..nt-1 (edge e from s_v[e] to
// s_v[e + 1]; record e holds the edge's bound in .w): one shared record load serves every
// candidate, and the PPT chains are independent.  Candidates whose FP32 sign came within the
// bound of zero are redone exactly.
template <int PPT, bool VERIFY>
__device__ __forceinline__ void tile_parity_multi(const float4 *__restrict__ s_rec, const int2 *__restrict__ s_v,
                                                  int nt, const int2 (&p)[PPT], const bool (&ok)[PPT], int ox,
                                                  int oy, int (&par)[PPT], unsigned long long &n_fb_pts,
                                                  unsigned long long &n_err, unsigned long long &n_ver)
{
    // one candidate at a time: the side of the previous vertex is carried in one predicate (the
    // loop is unrolled so that the thread's candidate arrays stay in registers)
    #pragma unroll
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
            if (VERIFY && st && !(fabsf(t) <= q.w)) {   // a trusted FP32 sign: its exact test
                const int2 ri = s_v[e], rj = s_v[e + 1];
                n_err += exact_edge_counts(p[r].x, p[r].y, ri.x, ri.y, rj.x, rj.y) != (int)(t > 0.f);
                ++n_ver;
            }
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

// Parities of a thread's PPT candidates over a tile whose vertices span a box x0..x1, y0..y1 with
// (W + 1)(H + 1) <= 2^30: every point is clamped to [x0 - 1, x1] x [y0 - 1, y1] first.  Each
// edge's crossing of a horizontal line lies in [x0, x1], so a point left of the box has every
// straddling edge's crossing strictly to its right before and after the clamp, a point at or right
// of x1 none, and a point below y0 or at or above y1 straddles no edge: every edge's decision is
// unchanged.  For the clamped point |det| <= (W + 1)|d_y| + (H + 1)|d_x| < 2 (W + 1)(H + 1) <=
// 2^31, so the int32 record (c, a, b, y_j) of pip_edge.cuh evaluated with wrapping arithmetic gives
// nt = -sign(d_y) det exactly, and the straddle test is the sign bit of (p_y - y_e) ^ (p_y - y_{e+1}):
// no filter and no uncertainty.  All PPT candidates share each record load.
// FY (a tile less than 2^24 high): the records hold y_{e+1} - y0 as an FP32 number and the
// straddle subtraction runs in FP32 on the clamped p_y - y0; both operands and their difference
// are integers of magnitude at most 2^24, so it is exact, and an exact zero is +0 (sign bit clear,
// as for the integer difference).  That moves one of the three integer-pipe operations of a pair
// to the FMA pipe, which the pair's two multiply-adds share with it.
template <int PPT, bool VERIFY, bool FY>
__device__ __forceinline__ void tile_parity_i32(const int4 *__restrict__ s_rec, const int2 *__restrict__ s_v,
                                                int nt, const int2 (&p)[PPT], const bool (&ok)[PPT], int x0, int y0,
                                                int x1, int y1, int (&par)[PPT], unsigned long long &n_err,
                                                unsigned long long &n_ver)
{
    unsigned px[PPT], py[PPT], up[PPT], acc[PPT];
    float fpy[PPT];
    const unsigned yv0 = (unsigned)s_v[0].y;
    const float fyv0 = __int2float_rn(s_v[0].y - y0);
    #pragma unroll
    for (int r = 0; r < PPT; ++r) {
        px[r] = (unsigned)min(p[r].x < x0 ? x0 - 1 : p[r].x, x1);
        py[r] = (unsigned)min(p[r].y < y0 ? y0 - 1 : p[r].y, y1);
        fpy[r] = __int2float_rn((int)(py[r] - (unsigned)y0));
        up[r] = FY ? __float_as_uint(__fsub_rn(fpy[r], fyv0)) : py[r] - yv0;
        acc[r] = 0;
    }
    #pragma unroll 4
    for (int e = 0; e < nt; ++e) {
        const int4 q = s_rec[e];
        #pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const unsigned u = FY ? __float_as_uint(__fsub_rn(fpy[r], __int_as_float(q.w))) : py[r] - (unsigned)q.w;
            const unsigned x = u ^ up[r];
            up[r] = u;
            const unsigned ntv = (unsigned)q.x + px[r] * (unsigned)q.y + py[r] * (unsigned)q.z;
            if (VERIFY && ok[r] && (int)x < 0) {   // a straddling edge: its exact test on the raw point
                const int2 ri = s_v[e], rj = s_v[e + 1];
                n_err += exact_edge_counts(p[r].x, p[r].y, ri.x, ri.y, rj.x, rj.y) != (int)(ntv >> 31);
                ++n_ver;
            }
            acc[r] ^= x & ntv;
        }
    }
    #pragma unroll
    for (int r = 0; r < PPT; ++r)
        if (ok[r]) par[r] ^= (int)(acc[r] >> 31);
}

// The same for a tile whose frame is below 2^30 from its centre, with scaled records: edge e is
// (-c' s_e, |d_y| s_e, -s d_x s_e, y_{e+1}) with s_e = 2^-k_e >= 1 / (M_x |d_y| + M_y |d_x|), so
// that nt = fma(P_y, ., fma(P_x, ., .)) = -s det s_e (rounded) and the edge's bound scaled by
// s_e is at most 13u whatever the edge: |nt| < 13u is the one uncertainty test.  The straddle
// test is the sign bit of (p_y - y_e) ^ (p_y - y_{e+1}) (the frame is under 2^31 tall), and an
// edge counts when that bit and nt's sign bit are both set.  All PPT candidates share each record
// load; each keeps its parity and its uncertainty in a sign bit.
template <int PPT, bool VERIFY>
__device__ __forceinline__ void tile_parity_scaled(const int4 *__restrict__ s_rec, const int2 *__restrict__ s_v,
                                                   int nt, const int2 (&p)[PPT], const bool (&ok)[PPT], int ox,
                                                   int oy, int (&par)[PPT], unsigned long long &n_fb_pts,
                                                   unsigned long long &n_err, unsigned long long &n_ver)
{
    float Px[PPT], Py[PPT];
    unsigned py[PPT], up[PPT], acc[PPT], unc[PPT];
    const unsigned y0 = (unsigned)s_v[0].y;
    #pragma unroll
    for (int r = 0; r < PPT; ++r) {
        Px[r] = __int2float_rn(p[r].x - ox);
        Py[r] = __int2float_rn(p[r].y - oy);
        py[r] = (unsigned)p[r].y;
        up[r] = py[r] - y0;
        acc[r] = 0;
        unc[r] = 0;
    }
    #pragma unroll 4
    for (int e = 0; e < nt; ++e) {
        const int4 q = s_rec[e];
        const float rc = __int_as_float(q.x), ra = __int_as_float(q.y), rb = __int_as_float(q.z);
        #pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const unsigned u = py[r] - (unsigned)q.w;
            const unsigned x = u ^ up[r];
            up[r] = u;
            const float ntf = __fmaf_rn(Py[r], rb, __fmaf_rn(Px[r], ra, rc));
            const float d = fabsf(ntf) - PM_BOUND_K;   // negative exactly when |nt| < 13u
            if (VERIFY && ok[r] && (int)x < 0 && d >= 0.f) {   // a trusted FP32 sign: its exact test
                const int2 ri = s_v[e], rj = s_v[e + 1];
                n_err += exact_edge_counts(p[r].x, p[r].y, ri.x, ri.y, rj.x, rj.y) != (int)(__float_as_uint(ntf) >> 31);
                ++n_ver;
            }
            acc[r] ^= x & __float_as_uint(ntf);
            unc[r] |= x & __float_as_uint(d);
        }
    }
    // candidates whose FP32 sign came within the bound of zero: the tile's exact parity, each by
    // the whole warp (every thread of the CTA is here)
    const int lane = threadIdx.x & 31;
    #pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const bool u = ok[r] && (unc[r] >> 31);
        int pr = (int)(acc[r] >> 31);
        for (unsigned um = __ballot_sync(FULL, u); um; um &= um - 1) {
            const int src = __ffs(um) - 1;
            const int q = warp_exact_parity(s_v, 0, nt, false, __shfl_sync(FULL, p[r].x, src),
                                            __shfl_sync(FULL, p[r].y, src), lane);
            if (lane == src) pr = q;
        }
        if (u) ++n_fb_pts;
        if (ok[r]) par[r] ^= pr;
    }
}

// Parity of p against polygon k through its y-slab index: the edges of p's slab and the tall
// list are exactly the edges whose y-range [min y, max y) contains p_y, i.e. every edge that can
// straddle p's ray; each straddling one is decided with the exact 64/128-bit test.
__device__ __forceinline__ int slab_parity(const unsigned char *ix, const SlabHeader *sh, int k, int2 p)
{
    const int4 g = reinterpret_cast<const int4 *>(ix + sh->off_geom)[k];
    if (p.y < g.x) return 0;
    const unsigned s = ((unsigned)p.y - (unsigned)g.x) / (unsigned)g.y;
    if (s >= (unsigned)g.z) return 0;                 // above the polygon: no edge straddles
    const unsigned *so = reinterpret_cast<const unsigned *>(ix + sh->off_slab);
    const unsigned *eo = reinterpret_cast<const unsigned *>(ix + sh->off_entry);
    const int4 *en = reinterpret_cast<const int4 *>(ix + sh->off_entries);
    const unsigned b = __ldg(so + k);
    int parity = 0;
    #pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {            // p's slab, then the tall list
        const unsigned sl = b + (pass == 0 ? s : (unsigned)g.z);
        const unsigned e1 = __ldg(eo + sl + 1);
        for (unsigned e = __ldg(eo + sl); e < e1; ++e) {
            const int4 q = __ldg(en + e);
            if ((q.y > p.y) != (q.w > p.y)) parity ^= exact_edge_counts(p.x, p.y, q.x, q.y, q.z, q.w);
        }
    }
    return parity;
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

template <int PPT, bool VERIFY>
__global__ void __launch_bounds__(LG_THREADS, PPT == 4 ? 3 : 4) k_pip_large(ClassifyArgs a, long long total_bits, LargeList *ll,
                                                         int lcap, int T)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *s_rec = reinterpret_cast<float4 *>(dsm);
    int2 *const s_vraw = reinterpret_cast<int2 *>(s_rec + T);   // 16-byte aligned
    __shared__ __align__(8) unsigned long long s_bar;           // completion of the tile's bulk copy
    __shared__ int s_fail;
    __shared__ int s_item[4];          // polygon, candidate block, edge slice, valid
    __shared__ int s_pb[4], s_tb[4];
    __shared__ int s_tf[4];            // tile frame: ox, oy, bound (float bits), wide
    __shared__ int s_vb[4];            // box of the tile's vertices alone

    constexpr int CB = LG_THREADS * PPT;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool dense = a.cand_offsets == nullptr;
    const int P = a.n_polys;
    const long long W32 = a.words_per_poly * 32;
    unsigned long long st_cand = 0, st_fbp = 0, st_err = 0, st_ver = 0;
    pdl_wait();   // the small-polygon kernel before it on the stream has filled the list
    const int count = *((volatile int *)&ll->count);
    const bool scan = *((volatile int *)&ll->overflow) != 0;
    if (count == 0 && !scan) return;   // nothing listed: the header is already clear for the next call
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        s_fail = 0;
    }
    unsigned bar_phase = 0;
    // A tile wait that gave up leaves the CTA "degraded": the copy may still land in its shared
    // tile buffer, so from then on the CTA neither issues copies nor touches that buffer and
    // decides every remaining pair exactly from global memory (same bits, slower); before it
    // exits it waits, again with a limit, for the copy that was late.
    bool degraded = false;
    unsigned fail_phase = 0;
    long long scan_k = blockIdx.x;   // overflow mode: polygons blockIdx.x, + gridDim.x, ...
    const SlabHeader *sh = reinterpret_cast<const SlabHeader *>(a.slab);
    const bool slab_ok = sh && sh->valid && sh->n_polys == P;
    // polygons with a y-slab index: one item per candidate block, no edge slices
    auto slabbed = [&](int k) {
        return slab_ok && reinterpret_cast<const int4 *>(a.slab + sh->off_geom)[k].z > 0;
    };
    // candidates per slab item: PPT per thread while the listed polygons give every CTA several
    // items that way, else one per thread (more, smaller items)
    auto slab_block = [&](long long n_cand) -> long long {
        return (n_cand / CB) * max(count, 1) >= 2LL * gridDim.x ? CB : LG_THREADS;
    };
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
                    const bool sl = slabbed(k);
                    const long long cbk = sl ? slab_block(ce - cs) : CB;
                    const long long nb = (ce - cs + cbk - 1) / cbk;
                    const int ES = sl ? (int)max(m, 1LL) : slice_edges(m, nb, count, gridDim.x);
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
                    const bool sl = slabbed(k);
                    const long long cbk = sl ? slab_block(ce - cs) : CB;
                    const long long nb = is_large_polygon(m, n) ? (ce - cs + cbk - 1) / cbk : 0;
                    const int ES = sl ? (int)max(m, 1LL) : slice_edges(m, nb, count, gridDim.x);
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
        const bool use_slabs = slabbed(k);
        const long long cbk = use_slabs ? slab_block(ce - cs) : CB;
        const long long cb0 = cs + (long long)s_item[1] * cbk, cb1 = min(cb0 + cbk, ce);
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
                if (pid < 0 || pid >= a.n_points) ok[r] = false;   // an id outside the points: no candidate
                else pt[r] = __ldg(a.points + pid);
            }
            if (ok[r]) {
                atomicMin(&s_pb[0], pt[r].x); atomicMin(&s_pb[1], pt[r].y);
                atomicMax(&s_pb[2], pt[r].x); atomicMax(&s_pb[3], pt[r].y);
                if (s_item[2] == 0) ++st_cand;
            }
        }
        if (use_slabs) {
            #pragma unroll
            for (int r = 0; r < PPT; ++r)
                if (ok[r]) par[r] = slab_parity(a.slab, sh, k, pt[r]);
        }
        __syncthreads();
        for (int e0 = ea; !use_slabs && s_pb[0] <= s_pb[2] && e0 < eb; e0 += T) {
            const int nt = min(T, eb - e0);
            if (degraded) {   // CTA-uniform: no barrier below is skipped by only some threads
                #pragma unroll
                for (int r = 0; r < PPT; ++r)
                    if (ok[r]) par[r] ^= global_exact_parity(a.verts + base, m, e0, e0 + nt, pt[r]);
                continue;
            }
            if (tid == 0) {
                s_tb[0] = s_pb[0]; s_tb[1] = s_pb[1]; s_tb[2] = s_pb[2]; s_tb[3] = s_pb[3];
                s_vb[0] = INT_MAX; s_vb[1] = INT_MAX; s_vb[2] = INT_MIN; s_vb[3] = INT_MIN;
            }
            // the tile's vertices e0 .. e0 + nt (the last one is vertex 0 when the tile closes the
            // polygon): the 16-byte-aligned interior of the contiguous run by one bulk copy, the
            // at most one vertex before and after it and the closing vertex by plain loads
            const int ncont = e0 + nt < m ? nt + 1 : nt;
            const unsigned long long src_lo = (unsigned long long)(a.verts + base + e0);
            const unsigned long long src_hi = src_lo + 8ull * (unsigned long long)ncont;
            const unsigned long long A = (src_lo + 15) & ~15ull, Bnd = src_hi & ~15ull;
            int2 *s_v = s_vraw + ((src_lo & 15) ? 1 : 0);     // s_v[i] = vertex e0 + i
            const bool bulk = Bnd > A;
            if (bulk && tid == 0)
                bulk_copy_g2s(s_v + (A - src_lo) / 8, reinterpret_cast<const void *>(A), (unsigned)(Bnd - A), &s_bar);
            const int ia = bulk ? (int)((A - src_lo) / 8) : ncont;        // first vertex of the copy
            const int ib = bulk ? (int)((Bnd - src_lo) / 8) : ncont;      // first vertex after it
            for (int i = tid; i <= nt; i += LG_THREADS) {
                if (bulk && i >= ia && i < ib) continue;
                int g = e0 + i;
                if (g >= m) g -= m;
                s_v[i] = __ldg(a.verts + base + g);
            }
            if (bulk && !mbar_wait(&s_bar, bar_phase, 1 << 22) && !mbar_wait(&s_bar, bar_phase, 1 << 22)) s_fail = 1;
            __syncthreads();
            if (s_fail) {   // read after the barrier, so every thread sees the same value
                degraded = true;
                fail_phase = bar_phase;
                #pragma unroll
                for (int r = 0; r < PPT; ++r)
                    if (ok[r]) par[r] ^= global_exact_parity(a.verts + base, m, e0, e0 + nt, pt[r]);
                continue;
            }
            if (bulk) bar_phase ^= 1u;
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
                atomicMin(&s_vb[0], x0); atomicMin(&s_vb[1], y0); atomicMax(&s_vb[2], x1); atomicMax(&s_vb[3], y1);
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
            // a tile whose own vertices span a box with (W + 1)(H + 1) <= 2^30 takes the exact int32
            // test on points clamped to [x0 - 1, x1] x [y0 - 1, y1] of that box (each edge's
            // decision unchanged), whatever the spread of the block's points
            const int vx0 = s_vb[0], vy0 = s_vb[1], vx1 = s_vb[2], vy1 = s_vb[3];
            const unsigned VW = (unsigned)vx1 - (unsigned)vx0, VH = (unsigned)vy1 - (unsigned)vy0;
            const bool i32 = VW < (1u << 30) && VH < (1u << 30) && (VW + 1ULL) * (VH + 1ULL) <= (1ULL << 30);
            const bool fy = i32 && VH < (1u << 24);   // the straddle subtraction in FP32 (exact)
            for (int i = tid; i < nt; i += LG_THREADS) {
                const int2 ri = s_v[i], rj = s_v[i + 1];
                if (i32) {
                    int4 r4 = int32_record(ri, rj);
                    if (fy) r4.w = __float_as_int(__int2float_rn(rj.y - vy0));
                    reinterpret_cast<int4 *>(s_rec)[i] = r4;
                    continue;
                }
                const long long ady = llabs((long long)rj.y - ri.y), adx = llabs((long long)rj.x - ri.x);
                // M_x |d_y| + M_y |d_x|, rounded up
                const float S = __fadd_ru(__fmul_ru(fMx, __ll2float_ru(ady)), __fmul_ru(fMy, __ll2float_ru(adx)));
                float4 rec;
                if (!wide) {
                    const int dx = rj.x - ri.x, dy = rj.y - ri.y;
                    const float fdx = __int2float_rn(dx), fdy = __int2float_rn(dy);
                    const float X = __int2float_rn(ri.x - ox), Y = __int2float_rn(ri.y - oy);
                    const float c = __fmaf_rn(X, fdy, -__fmul_rn(Y, fdx));
                    // s_e = 2^-k with 2^k >= S (exact scaling: a power of two)
                    const unsigned eb = (__float_as_uint(S) >> 23) & 0xffu;
                    const float se = S > 0.f ? __uint_as_float((253u - eb) << 23) : 1.f;
                    rec = dy > 0 ? make_float4(-c * se, fdy * se, -fdx * se, __int_as_float(rj.y))
                                 : make_float4(c * se, -fdy * se, fdx * se, __int_as_float(rj.y));
                } else {
                    rec = wide_record(ri, rj, ox, oy);
                    rec.w = __fmul_ru(PM_BOUND_K, S);   // the edge's own bound 13u (M_x |d_y| + M_y |d_x|)
                }
                s_rec[i] = rec;
            }
            __syncthreads();
            if (fy)
                tile_parity_i32<PPT, VERIFY, true>(reinterpret_cast<const int4 *>(s_rec), s_v, nt, pt, ok, vx0, vy0, vx1,
                                                   vy1, par, st_err, st_ver);
            else if (i32)
                tile_parity_i32<PPT, VERIFY, false>(reinterpret_cast<const int4 *>(s_rec), s_v, nt, pt, ok, vx0, vy0, vx1,
                                                    vy1, par, st_err, st_ver);
            else if (!wide)
                tile_parity_scaled<PPT, VERIFY>(reinterpret_cast<const int4 *>(s_rec), s_v, nt, pt, ok, ox, oy, par,
                                                st_fbp, st_err, st_ver);
            else
                tile_parity_multi<PPT, VERIFY>(s_rec, s_v, nt, pt, ok, ox, oy, par, st_fbp, st_err, st_ver);
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
    // a degraded CTA keeps its shared memory until the late copy has landed (bounded wait)
    if (degraded && tid == 0) mbar_wait(&s_bar, fail_phase, 1 << 22);
    if (a.stats) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st_cand += __shfl_down_sync(FULL, st_cand, o);
            st_fbp += __shfl_down_sync(FULL, st_fbp, o);
            if (VERIFY) st_err += __shfl_down_sync(FULL, st_err, o);
            if (VERIFY) st_ver += __shfl_down_sync(FULL, st_ver, o);
        }
        if (lane == 0) {
            if (st_cand) atomicAdd(a.stats + ST_CANDIDATES, st_cand);
            if (st_fbp) atomicAdd(a.stats + ST_FALLBACK_POINTS, st_fbp);
            if (VERIFY && st_err) atomicAdd(a.stats + ST_FILTER_ERRORS, st_err);
            if (VERIFY && st_ver) atomicAdd(a.stats + ST_VERIFIED, st_ver);
            if (tid == 0 && degraded) atomicAdd(a.stats + ST_WAIT_TIMEOUTS, 1ULL);
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

// Per-device launch set-up of the kernels (dynamic shared-memory limit, resident CTAs), done on
// the first launch on each device; calls from several host threads serialise on this lock.
static std::mutex g_setup_mu;

template <typename K>
static int ensure_smem(K kernel, size_t smem, size_t *configured)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (dev >= 0 && dev < 64 && configured[dev] < smem) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        configured[dev] = smem;
    }
    return 0;
}

template <bool DENSE, bool VERIFY, int R>
static int launch_warp_r(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int ctas_per_sm,
                         cudaStream_t stream)
{
    static size_t configured[64] = {0};
    static int blocks_per_sm[64] = {0};
    const size_t smem = sizeof(WarpSmem<R>) * (WP_THREADS / 32);
    int e = ensure_smem(k_pip_warp<DENSE, VERIFY, R>, smem, configured);
    if (e) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    int bps = 1;
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (blocks_per_sm[dev] == 0) {
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pip_warp<DENSE, VERIFY, R>, WP_THREADS, smem) !=
                cudaSuccess)
                nb = 1;
            blocks_per_sm[dev] = std::max(nb, 1);
        }
        bps = blocks_per_sm[dev];
    }
    if (ctas_per_sm > 0) bps = std::min(bps, ctas_per_sm);
    const long long nchunk = ((long long)a.n_polys + 31) / 32;
    const long long need = (nchunk + WP_THREADS / 32 - 1) / (WP_THREADS / 32);
    const int grid = (int)std::max(1LL, std::min((long long)n_sm * bps, need));
    k_pip_warp<DENSE, VERIFY, R><<<grid, WP_THREADS, smem, stream>>>(a, ll, lcap);
    note_launch();
    return (int)cudaGetLastError();
}

template <bool DENSE, bool VERIFY>
static int launch_warp_d(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int slice, int ctas_per_sm,
                         cudaStream_t stream)
{
    return slice == 128 ? launch_warp_r<DENSE, VERIFY, 4>(a, ll, lcap, n_sm, ctas_per_sm, stream)
                        : launch_warp_r<DENSE, VERIFY, 8>(a, ll, lcap, n_sm, ctas_per_sm, stream);
}

template <int PPT, bool VERIFY>
static int launch_large_ppt(const ClassifyArgs &a, long long total_bits, LargeList *ll, int lcap, int T, int grid,
                            cudaStream_t stream)
{
    static size_t configured[64] = {0};
    const size_t smem = filtered_smem_bytes(T);
    int e = ensure_smem(k_pip_large<PPT, VERIFY>, smem, configured);
    if (e) return e;
    // launched with programmatic stream serialization: its launch overlaps the end of the
    // small-polygon kernel, and pdl_wait at its start waits for that kernel's completion
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(LG_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, k_pip_large<PPT, VERIFY>, a, total_bits, ll, lcap, T);
    note_launch();
    return le != cudaSuccess ? (int)le : (int)cudaGetLastError();
}

template <bool VERIFY>
static int launch_filtered_v(const ClassifyArgs &a, long long total_bits, const Tuning &t, int n_sm, LargeList *ll,
                             int lcap, cudaStream_t stream)
{
    if (!a.cand_offsets && a.n_polys > 0 && a.words_per_poly > 0) {
        // dense output zeroed up front (one memset node), so that no warp of k_pip_warp has to
        // clear a large polygon's words on its own
        const cudaError_t m = cudaMemsetAsync(a.out_bits, 0, (size_t)a.n_polys * (size_t)a.words_per_poly * 4, stream);
        if (m != cudaSuccess) return (int)m;
    }
    int e;
    if (t.small_kernel == 1)
        e = launch_small_cmp(a, ll, lcap, n_sm, t.small_slice, t.small_ctas, VERIFY, stream);
    else if (t.small_kernel == 2)
        e = launch_small_tpp(a, ll, lcap, n_sm, t.small_slice / 16, t.small_ctas, VERIFY, stream);
    else
        e = a.cand_offsets ? launch_warp_d<false, VERIFY>(a, ll, lcap, n_sm, t.small_slice, t.small_ctas, stream)
                           : launch_warp_d<true, VERIFY>(a, ll, lcap, n_sm, t.small_slice, t.small_ctas, stream);
    if (e) return e;
    const int grid = n_sm * t.ctas_per_sm;
    switch (t.pts_per_thread) {
        case 1: return launch_large_ppt<1, VERIFY>(a, total_bits, ll, lcap, t.edge_tile, grid, stream);
        case 4: return launch_large_ppt<4, VERIFY>(a, total_bits, ll, lcap, t.edge_tile, grid, stream);
        default: return launch_large_ppt<2, VERIFY>(a, total_bits, ll, lcap, t.edge_tile, grid, stream);
    }
}

int launch_filtered(const ClassifyArgs &a, long long total_bits, const Tuning &t, int n_sm, LargeList *ll, int lcap,
                    cudaStream_t stream)
{
    return t.verify ? launch_filtered_v<true>(a, total_bits, t, n_sm, ll, lcap, stream)
                    : launch_filtered_v<false>(a, total_bits, t, n_sm, ll, lcap, stream);
}

}  // namespace pipdev
