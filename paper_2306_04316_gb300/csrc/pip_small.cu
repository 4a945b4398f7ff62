// Small-polygon kernel of pip_classify that compacts in-box candidates and prefetches the next
// slice (k_pip_cmp).
//
// Method section, steps 2-7 with Constraint 1: for a candidate point p and the edge R_i -> R_j of
// its polygon, the crossing counts when the straddle test (y_i > p_y) != (y_j > p_y) holds and
// sign(d_y) det > 0, det = (x_i - p_x) d_y - (y_i - p_y) d_x; the parity of the count is the inside
// bit.  The per-edge records and the three exact/filtered arithmetic modes are those of
// pip_edge.cuh (int32 for boxes with width x height below 2^30, int64 below 2^31, FP32 with an
// exact recheck above).
//
// Work decomposition.  Every warp works on its own: it takes chunks of 32 consecutive polygons
// (lane = polygon; offsets in registers, the next chunk's loaded one chunk ahead; polygons too
// large for a warp go on the large-polygon list as in k_pip_warp) and cuts each chunk's
// candidates into slices: polygon sets of consecutive small polygons with at most 256 vertices in
// all, and windows of at most CS consecutive candidates of one set.  For each slice:
//   1. the slice after it is found and its candidate ids are loaded into registers;
//   2. when the slice's polygons differ from the previous slice's, their edge records (lane per
//      edge), boxes, arithmetic modes and frames (lane per polygon) are built from the vertices
//      in shared memory, which then receive the next set's vertices (cp.async) as soon as no
//      exact recheck can need them (a set is normally a whole chunk, so several slices share it);
//   3. pass 1, a lane per candidate slot: the owning polygon (a byte per slot, filled by the
//      polygons' lanes), the closed-box test, and compaction of the in-box candidates to the
//      front of the slice's point buffer.  A point outside its polygon's closed box is outside the
//      polygon, so only in-box candidates are walked (on building footprints with points
//      uniform in a 1.5x box, 44 % of them);
//   4. the next slice's points are gathered into the other point buffer (cp.async);
//   5. pass 2, a lane per compacted candidate (two per lane in int32 sets): the lanes walk their
//      polygons' edge records in lockstep, a lane whose polygon is shorter repeating its last record (a repeated edge never
//      straddles, so it adds nothing), and store their parities as per-slot bytes;
//   6. ballots of the per-slot bytes give the slice's output words; the first and last word may
//      be shared with a neighbouring slice or polygon and take a masked AND/OR pair.
// Everything a slice reads from global memory was requested one slice earlier, so a warp never
// waits for memory in steady state; no barrier spans more than one warp.
#include <algorithm>
#include <climits>
#include <mutex>
#include <type_traits>

#include "pip_device.cuh"
#include "pip_edge.cuh"
#include "pip_launch.h"

namespace pipdev {

constexpr int SC_THREADS = 128;   // 4 independent warps per CTA

template <int CS>
struct __align__(16) CmpSmem {
    int4 rec[WP_V];                 // edge records of the slice's polygons
    int2 v[WP_V];                   // their vertices; then the next slice's
    int2 pt[2][CS];                 // candidate points: this slice (compacted in place), the next
    int4 box[32];                   // per chunk polygon: closed bounding box
    int4 fr[32];                    // ox, oy, bound (float bits), e0 | e1 << 9 | mode << 18
    unsigned cm[CS];                // compacted candidate: slot | chunk lane << 8
    unsigned vstart[WP_V / 32 + 1]; // bit i: vertex i starts a polygon of the slice, or i == nv
    unsigned char own[CS];          // slot -> chunk lane of the polygon that owns it
    unsigned char par[CS];          // parity per slot (0 for slots outside their box)
    unsigned char vp[WP_V];         // vertex -> chunk lane (slices with int64 / FP32 polygons)
};

template <int CS>
constexpr size_t cmp_smem_bytes()
{
    return sizeof(CmpSmem<CS>) * (SC_THREADS / 32);
}

// A chunk of 32 consecutive polygons as its lanes see it (lane j = polygon 32 ch + j).
template <typename CI>
struct Chunk {
    int ch;          // chunk index (>= nchunk: none)
    int np;          // polygons in the chunk
    int pb, pe;      // this lane's polygon: vertex range
    CI cb, ce;       // candidate range
    int cum;         // vertices of the chunk's polygons up to and including this lane's
    bool small;      // classified here (else large, or past the chunk's end)
};

// A slice: candidates [c0, c1) of a polygon set, the chunk's polygons j0 .. q-1 (consecutive, all
// small, at most WP_V vertices in all: vertices [vb, ve)), whose candidates end at cend.
// Consecutive slices of one set share its edge records.
template <typename CI>
struct Slice {
    CI c0, c1, cend;
    int j0, q, vb, ve;
    int ch;          // chunk index (< 0: none)
};

// The first slice of the first polygon set of chunk C with candidates at c or later: the set
// starts at the first small polygon with such candidates and takes the polygons after it while
// they are small and their vertices fit in WP_V (every lane gets the same value).
template <typename CI, int CS>
__device__ __forceinline__ Slice<CI> find_set(const Chunk<CI> &C, CI c, int lane)
{
    Slice<CI> s;
    s.c0 = s.c1 = s.cend = 0;
    s.j0 = s.q = s.vb = s.ve = 0;
    s.ch = -1;
    const unsigned cmk = __ballot_sync(FULL, C.small && C.ce > C.cb && C.ce > c);
    if (!cmk) return s;
    const int j0 = __ffs(cmk) - 1;
    s.c0 = max(c, __shfl_sync(FULL, C.cb, j0));
    const int before = __shfl_sync(FULL, C.cum, j0) - (__shfl_sync(FULL, C.pe, j0) - __shfl_sync(FULL, C.pb, j0));
    const unsigned stop = __ballot_sync(FULL, lane >= j0 && (!C.small || C.cum - before > WP_V));
    s.q = stop ? __ffs(stop) - 1 : 32;   // > j0: a small polygon has at most WP_V vertices
    s.cend = __shfl_sync(FULL, C.ce, s.q - 1);
    s.c1 = min(s.c0 + (CI)CS, s.cend);
    s.j0 = j0;
    s.vb = __shfl_sync(FULL, C.pb, j0);
    s.ve = __shfl_sync(FULL, C.pe, s.q - 1);
    s.ch = C.ch;
    return s;
}

template <bool DENSE, bool VERIFY, int CS>
__global__ void __launch_bounds__(SC_THREADS, 4) k_pip_cmp(ClassifyArgs a, LargeList *ll, int lcap)
{
    using CI = typename std::conditional<DENSE, long long, int>::type;
    constexpr int NR = CS / 32;                       // slot rounds of a slice
    extern __shared__ __align__(16) unsigned char dsm[];
    CmpSmem<CS> &S = reinterpret_cast<CmpSmem<CS> *>(dsm)[threadIdx.x >> 5];
    pdl_trigger();   // the large-polygon kernel may launch now; it waits for this grid to finish
    const unsigned rec_base = (unsigned)__cvta_generic_to_shared(S.rec);
    const int lane = threadIdx.x & 31;
    const unsigned lemask = 0xffffffffu >> (31 - lane);   // lanes 0..lane
    const unsigned ltmask = lemask >> 1;                  // lanes below this one
    const int P = a.n_polys;
    const CI W32 = (CI)(a.words_per_poly * 32);
    const long long NPTS = a.n_points;
    const int nchunk = (P + 31) >> 5;
    const int gw = blockIdx.x * (SC_THREADS / 32) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (SC_THREADS / 32);
    unsigned st_cand = 0, st_rej = 0, st_fbp = 0, st_err = 0, st_ver = 0;
    if (!DENSE && gw == 0 && lane == 0 && P > 0) {
        // bits past the last candidate in the final word are 0
        const long long C = __ldg(a.cand_offsets + P);
        if (C & 31) masked_store(a.out_bits + (C >> 5), ~((1u << (C & 31)) - 1u), 0u);
    }

    // ---- chunks: raw offsets of the next chunk loaded one chunk ahead
    int f_ch = gw, f_pb = 0, f_pe = 0;
    CI f_cb = 0, f_ce = 0;
    auto fetch = [&](int ch) {
        f_ch = ch;
        const int kk = (ch << 5) + lane;
        if (ch < nchunk && kk < P) {
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
    // the prefetched chunk as lanes see it (no side effects)
    auto derive = [&]() {
        Chunk<CI> C;
        C.ch = f_ch;
        C.np = f_ch < nchunk ? min(32, P - (f_ch << 5)) : 0;
        const bool has = lane < C.np;
        C.pb = has ? f_pb : 0;
        C.pe = has ? f_pe : 0;
        C.cb = has ? f_cb : 0;
        C.ce = has ? f_ce : 0;
        const long long nlen = DENSE ? min(NPTS, (long long)W32) : (long long)(C.ce - C.cb);
        C.small = has && !is_large_polygon(C.pe - C.pb, nlen);
        int cum = C.small ? C.pe - C.pb : 0;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, cum, o);
            if (lane >= o) cum += t;
        }
        C.cum = cum;
        return C;
    };
    // a chunk becomes current: its large polygons go on the list and their bits are cleared
    auto activate = [&](const Chunk<CI> &C) {
        const bool has = lane < C.np;
        const long long nlen = DENSE ? min(NPTS, (long long)W32) : (long long)(C.ce - C.cb);
        const bool lg = has && !C.small;
        const unsigned lgm = __ballot_sync(FULL, lg);
        if (lg && C.ce > C.cb && NPTS > 0) {
            const int idx = atomicAdd(&ll->count, 1);
            if (idx < lcap) {
                large_entries(ll)[idx] = (C.ch << 5) + lane;
                large_taken(ll, lcap)[idx] = 0;
            } else {
                atomicExch(&ll->overflow, 1);
            }
        }
        (void)nlen;
        // large polygons' bits are 0 here; k_pip_large XORs their parities in afterwards (a dense
        // output is zeroed before this kernel)
        if (!DENSE)
            for (unsigned m = lgm; m; m &= m - 1) {
                const int l = __ffs(m) - 1;
                zero_bits(a.out_bits, (long long)__shfl_sync(FULL, C.cb, l), (long long)__shfl_sync(FULL, C.ce, l),
                          lane);
            }
        fetch(C.ch + nw);
    };

    // ---- loads of a slice: vertices (cp.async to S.v), ids (registers), points (cp.async, once
    //      the ids have arrived)
    CI nid[NR];
    auto load_ids = [&](const Slice<CI> &s) {
        if (DENSE) return;
        #pragma unroll
        for (int r = 0; r < NR; ++r) {
            const CI c = s.c0 + 32 * r + lane;
            nid[r] = c < s.c1 ? (CI)__ldg(a.cand_ids + c) : (CI)-1;
        }
    };
    auto gather = [&](const Slice<CI> &s, int2 *dst) -> unsigned {
        unsigned vm = 0;
        CI dbase = 0;
        if (DENSE) dbase = s.c0 % W32;
        #pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int slot = 32 * r + lane;
            CI pid;
            if (DENSE) {
                CI t = dbase + slot;   // (c0 + slot) mod W32: a slice may span several polygons
                while (t >= W32) t -= W32;
                pid = s.c0 + slot < s.c1 ? t : (CI)-1;
            } else {
                pid = nid[r];
            }
            if (pid >= 0 && (long long)pid < NPTS) {
                cp_async8(&dst[slot], a.points + pid);
                vm |= 1u << r;
            }
        }
        return vm;
    };
    auto load_verts = [&](const Slice<CI> &s) {
        for (int i = lane; i < s.ve - s.vb; i += 32) cp_async8(&S.v[i], a.verts + s.vb + i);
    };

    // ---- the first slice
    fetch(gw);
    Chunk<CI> C = derive();
    activate(C);
    Slice<CI> D = find_set<CI, CS>(C, (CI)0, lane);
    while (D.ch < 0 && f_ch < nchunk) {
        C = derive();
        activate(C);
        D = find_set<CI, CS>(C, (CI)0, lane);
    }
    int cur = 0;
    unsigned validm = 0;
    if (D.ch >= 0) {
        load_verts(D);
        load_ids(D);
        validm = gather(D, S.pt[0]);
        cp_async_commit();
    }
    int set_ch = -1, set_j0 = -1, set_q = -1;   // polygons whose records S.rec holds
    bool set_all32 = true;
    // every slice holds at least one candidate and every chunk is stepped over once, so a warp
    // takes at most (candidates + chunks) turns of this loop; the guard ends it should that ever
    // fail (counted with the timed-out waits, never expected)
    const long long max_turns = (DENSE ? (long long)P * (long long)W32
                                       : (P > 0 ? (long long)__ldg(a.cand_offsets + P) - __ldg(a.cand_offsets) : 0)) +
                                nchunk + 2;
    long long turns = 0;
    bool guard_tripped = false;

    while (D.ch >= 0) {
        if (++turns > max_turns) {
            guard_tripped = true;
            break;
        }
        cp_async_wait_all();   // this slice's points (and vertices, when new) were requested one slice ago
        __syncwarp();
        // ---- the slice after this one (in this set, the chunk's next set, or the next chunk's
        //      first), and its candidate ids
        Slice<CI> Dn = D;
        if (D.c1 < D.cend) {
            Dn.c0 = D.c1;
            Dn.c1 = min(D.c1 + (CI)CS, D.cend);
        } else {
            Dn = find_set<CI, CS>(C, D.c1, lane);
            if (Dn.ch < 0 && f_ch < nchunk) {
                const Chunk<CI> N = derive();
                Dn = find_set<CI, CS>(N, (CI)0, lane);
            }
        }
        const bool dn_new_set = Dn.ch >= 0 && !(Dn.ch == D.ch && Dn.j0 == D.j0 && Dn.q == D.q);
        if (Dn.ch >= 0) load_ids(Dn);
        const bool new_set = !(D.ch == set_ch && D.j0 == set_j0 && D.q == set_q);
        const int nv = D.ve - D.vb;
        const bool mine = lane >= D.j0 && lane < D.q;   // this lane's polygon is in the slice
        if (new_set) {
            set_ch = D.ch; set_j0 = D.j0; set_q = D.q;
            // ---- vertex i starts a polygon (or i == nv)
            if (lane <= WP_V / 32) S.vstart[lane] = 0;
            __syncwarp();
            if (mine && C.pe > C.pb) atomicOr(&S.vstart[(C.pb - D.vb) >> 5], 1u << ((C.pb - D.vb) & 31));
            if (lane == 0) atomicOr(&S.vstart[nv >> 5], 1u << (nv & 31));
            __syncwarp();
            // ---- int32 records of the edges that do not close their polygon (lane per edge)
            for (int i = lane; i + 1 < nv; i += 32)
                if (!((S.vstart[(i + 1) >> 5] >> ((i + 1) & 31)) & 1u)) S.rec[i] = int32_record(S.v[i], S.v[i + 1]);
            __syncwarp();
            // ---- per polygon (lane per polygon): box, arithmetic mode, closing edge
            int mode = MODE_INT32;
            int4 fr4 = make_int4(0, 0, 0, 0), box4 = make_int4(INT_MAX, INT_MAX, INT_MIN, INT_MIN);
            const int e0 = C.pb - D.vb, e1 = C.pe - D.vb;
            int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
            if (D.q - D.j0 <= 16) {
                // two lanes per polygon, alternate vertices; the polygon's lane collects the box
                const int jj = D.j0 + (lane >> 1);
                const int a0 = __shfl_sync(FULL, e0, jj & 31), a1 = __shfl_sync(FULL, e1, jj & 31);
                if (jj < D.q)
                    for (int i = a0 + (lane & 1); i < a1; i += 2) {
                        const int2 v = S.v[i];
                        x0 = min(x0, v.x); y0 = min(y0, v.y); x1 = max(x1, v.x); y1 = max(y1, v.y);
                    }
                x0 = min(x0, __shfl_xor_sync(FULL, x0, 1)); y0 = min(y0, __shfl_xor_sync(FULL, y0, 1));
                x1 = max(x1, __shfl_xor_sync(FULL, x1, 1)); y1 = max(y1, __shfl_xor_sync(FULL, y1, 1));
                const int src = (2 * (lane - D.j0)) & 31;
                x0 = __shfl_sync(FULL, x0, src); y0 = __shfl_sync(FULL, y0, src);
                x1 = __shfl_sync(FULL, x1, src); y1 = __shfl_sync(FULL, y1, src);
            } else if (mine) {
                #pragma unroll 2
                for (int i = e0; i < e1; ++i) {
                    const int2 v = S.v[i];
                    x0 = min(x0, v.x); y0 = min(y0, v.y); x1 = max(x1, v.x); y1 = max(y1, v.y);
                }
            }
            if (mine) {
                const unsigned W = (unsigned)x1 - (unsigned)x0, H = (unsigned)y1 - (unsigned)y0;
                const unsigned Mx = W - (W >> 1), My = H - (H >> 1);
                int bound = 0;
                if (e1 > e0 && !(W < (1u << 30) && H < (1u << 30) && (unsigned long long)W * H < (1ULL << 30))) {
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
            // a slice with any polygon outside the int32 test puts its int32 polygons on the int64
            // test too, so that a round walks at most two kinds of loop
            set_all32 = __all_sync(FULL, mode == MODE_INT32);
            if (!set_all32 && mode == MODE_INT32) mode = MODE_INT64;
            if (mine) {
                S.fr[lane] = make_int4(fr4.x, fr4.y, fr4.z, fr4.w | (mode << 18));
                S.box[lane] = box4;
                if (mode == MODE_INT32 && e1 > e0) S.rec[e1 - 1] = int32_record(S.v[e1 - 1], S.v[e0]);
                if (!set_all32)
                    for (int i = e0; i < e1; ++i) S.vp[i] = (unsigned char)lane;
            }
            __syncwarp();
            if (!set_all32) {
                // int64 / FP32 / wide records, lane per edge, in each polygon's frame
                for (int i = lane; i < nv; i += 32) {
                    const int4 f = S.fr[S.vp[i]];
                    const int pe0 = f.w & 0x1ff, pe1 = (f.w >> 9) & 0x1ff, md = f.w >> 18;
                    const int2 ri = S.v[i], rj = S.v[i + 1 == pe1 ? pe0 : i + 1];
                    if (md == MODE_INT64) {
                        const int dx = rj.x - ri.x, dy = rj.y - ri.y;
                        S.rec[i] = make_int4(ri.x - f.x, dy > 0 ? dy : -dy, dy > 0 ? -dx : dx, rj.y - f.y);
                    } else if (md == MODE_FP32) {
                        const float4 r4 = fp32_record(ri, rj, f.x, f.y);
                        S.rec[i] = make_int4(__float_as_int(r4.x), __float_as_int(r4.y), __float_as_int(r4.z),
                                             __float_as_int(r4.w));
                    } else {
                        const float4 r4 = wide_record(ri, rj, f.x, f.y);
                        S.rec[i] = make_int4(__float_as_int(r4.x), __float_as_int(r4.y), __float_as_int(r4.z),
                                             __float_as_int(r4.w));
                    }
                }
            }
            __syncwarp();
        }
        // the vertex buffer is free once the records exist, unless an exact recheck (FP32 records)
        // or the verification mode may still read it during the walk
        const bool verts_free_early = set_all32 && !VERIFY;
        if (dn_new_set && verts_free_early) load_verts(Dn);

        // ---- pass 1: owner, box test, compaction of the in-box candidates
        const int nc = (int)(D.c1 - D.c0);
        if (mine && C.ce > D.c0 && C.cb < D.c1) {
            // this polygon's slots [s, e) of the slice: owner bytes, four at a time where aligned
            int sl = (int)(max(C.cb, D.c0) - D.c0);
            const int se = (int)(min(C.ce, D.c1) - D.c0);
            const unsigned fill = (unsigned)lane * 0x01010101u;
            for (; sl < se && (sl & 3); ++sl) S.own[sl] = (unsigned char)lane;
            for (; sl + 4 <= se; sl += 4) *reinterpret_cast<unsigned *>(&S.own[sl]) = fill;
            for (; sl < se; ++sl) S.own[sl] = (unsigned char)lane;
        }
        for (int i = lane; i < CS / 4; i += 32) reinterpret_cast<unsigned *>(S.par)[i] = 0u;
        __syncwarp();
        int2 *const pts = S.pt[cur];
        int ncomp = 0;
        #pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (32 * r < nc) {
                const int slot = 32 * r + lane;
                const int own = S.own[slot] & 31;   // slots past the slice hold stale owners: not valid
                const int2 p = pts[slot];
                const int4 b = S.box[own];
                const bool in = ((validm >> r) & 1u) && p.x >= b.x && p.x <= b.z && p.y >= b.y && p.y <= b.w;
                const unsigned im = __ballot_sync(FULL, in);
                if (in) {
                    const int pos = ncomp + __popc(im & ltmask);
                    pts[pos] = p;
                    S.cm[pos] = (unsigned)slot | ((unsigned)own << 8);
                }
                ncomp += __popc(im);
            }
        }
        st_cand += __popc(validm);
        if (lane == 0) st_rej += (unsigned)ncomp;   // in-box candidates; rejects = candidates - these
        __syncwarp();
        // ---- the next slice's points, into the other buffer (its ids have had pass 1 to arrive)
        unsigned validm_n = 0;
        if (Dn.ch >= 0) validm_n = gather(Dn, S.pt[cur ^ 1]);

        // ---- pass 2: the compacted candidates walk their polygons' records in lockstep.  Int32
        //      sets: each lane takes two candidates (positions r0 + lane and r0 + 32 + lane), two
        //      independent chains over one loop, so a round covers 64 candidates
        if (set_all32) {
            for (int r0 = 0; r0 < ncomp; r0 += 64) {
                const int pa = r0 + lane, pb2 = r0 + 32 + lane;
                const bool aa = pa < ncomp, ab = pb2 < ncomp;
                const unsigned ca = aa ? S.cm[pa] : 0u, cb2 = ab ? S.cm[pb2] : 0u;
                const int2 qa = pts[aa ? pa : 0], qb = pts[ab ? pb2 : 0];
                const int fa = S.fr[(ca >> 8) & 31u].w, fb = S.fr[(cb2 >> 8) & 31u].w;   // e0 | e1 << 9 | ...
                const int a0 = aa ? (fa & 0x1ff) : 0, a1 = aa ? ((fa >> 9) & 0x1ff) : 1;   // inactive: record 0
                const int b0 = ab ? (fb & 0x1ff) : 0, b1 = ab ? ((fb >> 9) & 0x1ff) : 1;
                const int K = __reduce_max_sync(FULL, (unsigned)max(a1 - a0, b1 - b0));
                // nt = -sign(d_y) det exactly; the sign bit of (u_j ^ u_i) is the straddle test,
                // u = p_y - y; a crossing counts when both sign bits are set
                unsigned ada = rec_base + 16u * (unsigned)a0, adb = rec_base + 16u * (unsigned)b0;
                const unsigned ala = rec_base + 16u * (unsigned)(a1 - 1), alb = rec_base + 16u * (unsigned)(b1 - 1);
                const unsigned pxa = (unsigned)qa.x, pya = (unsigned)qa.y, pxb = (unsigned)qb.x, pyb = (unsigned)qb.y;
                unsigned upa = pya - (unsigned)lds128(ala).w, upb = pyb - (unsigned)lds128(alb).w;   // vertex e0
                unsigned acca = 0, accb = 0;
                #pragma unroll 2
                for (int k = 0; k < K; ++k) {
                    const unsigned cura = ada, curb = adb;
                    const int4 ra = lds128(ada), rb = lds128(adb);
                    ada = __viaddmin_u32(ada, 16u, ala);
                    adb = __viaddmin_u32(adb, 16u, alb);
                    const unsigned ua = pya - (unsigned)ra.w, ub = pyb - (unsigned)rb.w;
                    const unsigned nta = (unsigned)ra.x + pxa * (unsigned)ra.y + pya * (unsigned)ra.z;
                    const unsigned ntb = (unsigned)rb.x + pxb * (unsigned)rb.y + pyb * (unsigned)rb.z;
                    if (VERIFY) {   // straddling edges: their exact tests
                        if (aa && (int)(ua ^ upa) < 0) {
                            const int e = (int)((cura - rec_base) >> 4);
                            const int2 ri = S.v[e], rj = S.v[e + 1 == a1 ? a0 : e + 1];
                            st_err += exact_edge_counts(qa.x, qa.y, ri.x, ri.y, rj.x, rj.y) != (int)(nta >> 31);
                            ++st_ver;
                        }
                        if (ab && (int)(ub ^ upb) < 0) {
                            const int e = (int)((curb - rec_base) >> 4);
                            const int2 ri = S.v[e], rj = S.v[e + 1 == b1 ? b0 : e + 1];
                            st_err += exact_edge_counts(qb.x, qb.y, ri.x, ri.y, rj.x, rj.y) != (int)(ntb >> 31);
                            ++st_ver;
                        }
                    }
                    acca ^= (ua ^ upa) & nta;
                    accb ^= (ub ^ upb) & ntb;
                    upa = ua;
                    upb = ub;
                }
                if (aa) S.par[ca & 0xffu] = (unsigned char)(acca >> 31);
                if (ab) S.par[cb2 & 0xffu] = (unsigned char)(accb >> 31);
            }
        }
        for (int r0 = 0; !set_all32 && r0 < ncomp; r0 += 32) {
            const int pos = r0 + lane;
            const bool act = pos < ncomp;
            const unsigned cmv = act ? S.cm[pos] : 0u;
            const int2 p2 = pts[act ? pos : 0];
            const int fw = S.fr[(cmv >> 8) & 31u].w;   // e0 | e1 << 9 | mode << 18
            const int e0 = act ? (fw & 0x1ff) : 0, e1 = act ? ((fw >> 9) & 0x1ff) : 1;   // inactive: record 0 once
            int parity = 0;
            {   // int64 / FP32 sets
                const int4 f = S.fr[(cmv >> 8) & 31u];
                const int mode = f.w >> 18;
                const bool g6 = act && mode == MODE_INT64;
                const int k6 = __reduce_max_sync(FULL, g6 ? (unsigned)(e1 - e0) : 0u);
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
                const bool gf = act && mode >= MODE_FP32;
                const int kf = __reduce_max_sync(FULL, gf ? (unsigned)(e1 - e0) : 0u);
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
            if (act) S.par[cmv & 0xffu] = (unsigned char)parity;
        }
        __syncwarp();
        if (dn_new_set && !verts_free_early) load_verts(Dn);
        cp_async_commit();

        // ---- the slice's words: word k = bits_k << sh | bits_(k-1) >> (32 - sh), of which bits
        //      [sh, sh + nc) of words c0 >> 5 ... belong to the slice
        const int sh = (int)(D.c0 & 31);
        unsigned mybits = 0;
        #pragma unroll
        for (int r = 0; r < NR; ++r) {
            const unsigned bits = __ballot_sync(FULL, S.par[32 * r + lane] != 0);
            if (lane == r) mybits = bits;
        }
        const unsigned prev = __shfl_up_sync(FULL, mybits, 1);
        unsigned myw = mybits << sh;
        if (sh && lane > 0) myw |= prev >> (32 - sh);
        const int nwd = (sh + nc + 31) >> 5;
        if (lane < nwd)
            masked_store(a.out_bits + (D.c0 >> 5) + lane, range_mask(lane == 0 ? sh : 0, min(32, sh + nc - 32 * lane)),
                         myw);
        __syncwarp();   // S.own, S.par, S.cm and this point buffer are rewritten by the next slice

        // ---- on to the next slice
        if (Dn.ch >= 0) {
            if (Dn.ch != D.ch) {
                C = derive();   // the prefetched chunk, in which the next slice was found
                activate(C);
            }
            D = Dn;
            cur ^= 1;
            validm = validm_n;
        } else {
            // no slice was found in this chunk or the next one: step through chunks (activating
            // each) until one has small candidates, then load its first slice without overlap
            D.ch = -1;
            while (D.ch < 0 && f_ch < nchunk) {
                C = derive();
                activate(C);
                D = find_set<CI, CS>(C, (CI)0, lane);
            }
            if (D.ch >= 0) {
                cp_async_wait_all();
                __syncwarp();
                load_verts(D);
                load_ids(D);
                cur ^= 1;
                validm = gather(D, S.pt[cur]);
                cp_async_commit();
                set_ch = -1;
            }
        }
    }
    cp_async_wait_all();
    if (guard_tripped && lane == 0 && a.stats) atomicAdd(a.stats + ST_WAIT_TIMEOUTS, 1ULL);
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
            st_rej = st_cand - st_rej;   // st_rej held the in-box count
            if (VERIFY && st_ver) atomicAdd(a.stats + ST_VERIFIED, (unsigned long long)st_ver);
            if (st_cand) atomicAdd(a.stats + ST_CANDIDATES, (unsigned long long)st_cand);
            if (st_rej) atomicAdd(a.stats + ST_BBOX_REJECTS, (unsigned long long)st_rej);
            if (st_fbp) atomicAdd(a.stats + ST_FALLBACK_POINTS, (unsigned long long)st_fbp);
            if (VERIFY && st_err) atomicAdd(a.stats + ST_FILTER_ERRORS, (unsigned long long)st_err);
        }
    }
}

// =============================================================================================
// launch
// =============================================================================================

static std::mutex g_cmp_mu;

template <bool DENSE, bool VERIFY, int CS>
static int launch_cmp_t(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int ctas_per_sm,
                        cudaStream_t stream)
{
    static size_t configured[64] = {0};
    static int max_bps[64] = {0};
    const size_t smem = cmp_smem_bytes<CS>();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    int bps = 1;
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lock(g_cmp_mu);
        if (configured[dev] < smem) {
            e = cudaFuncSetAttribute(k_pip_cmp<DENSE, VERIFY, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return (int)e;
            configured[dev] = smem;
        }
        if (max_bps[dev] == 0) {
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pip_cmp<DENSE, VERIFY, CS>, SC_THREADS, smem) !=
                cudaSuccess)
                nb = 1;
            max_bps[dev] = std::max(nb, 1);
        }
        bps = max_bps[dev];
    }
    if (ctas_per_sm > 0) bps = std::min(bps, ctas_per_sm);
    const long long nchunk = ((long long)a.n_polys + 31) / 32;
    const long long need = (nchunk + SC_THREADS / 32 - 1) / (SC_THREADS / 32);
    const int grid = (int)std::max(1LL, std::min((long long)n_sm * bps, need));
    k_pip_cmp<DENSE, VERIFY, CS><<<grid, SC_THREADS, smem, stream>>>(a, ll, lcap);
    note_launch();
    return (int)cudaGetLastError();
}

template <bool DENSE, bool VERIFY>
static int launch_cmp_d(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int slice, int ctas_per_sm,
                        cudaStream_t stream)
{
    return slice == 128 ? launch_cmp_t<DENSE, VERIFY, 128>(a, ll, lcap, n_sm, ctas_per_sm, stream)
                        : launch_cmp_t<DENSE, VERIFY, 256>(a, ll, lcap, n_sm, ctas_per_sm, stream);
}

int launch_small_cmp(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int slice, int ctas_per_sm,
                     bool verify, cudaStream_t stream)
{
    const bool dense = a.cand_offsets == nullptr;
    if (dense)
        return verify ? launch_cmp_d<true, true>(a, ll, lcap, n_sm, slice, ctas_per_sm, stream)
                      : launch_cmp_d<true, false>(a, ll, lcap, n_sm, slice, ctas_per_sm, stream);
    return verify ? launch_cmp_d<false, true>(a, ll, lcap, n_sm, slice, ctas_per_sm, stream)
                  : launch_cmp_d<false, false>(a, ll, lcap, n_sm, slice, ctas_per_sm, stream);
}

}  // namespace pipdev
