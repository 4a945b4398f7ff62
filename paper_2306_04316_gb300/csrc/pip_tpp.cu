// Small-polygon kernel of pip_classify with one thread per polygon and its candidates in
// registers (k_pip_tpp).
//
// Method section, steps 2-7 with Constraint 1: for a candidate point p and the edge R_i -> R_j of
// its polygon, the crossing counts when the straddle test (y_i > p_y) != (y_j > p_y) holds and
// sign(d_y) det > 0, det = (x_i - p_x) d_y - (y_i - p_y) d_x; the parity of the count is the inside
// bit.
//
// Work decomposition.  Every thread takes whole polygons (polygon k = global thread, + all
// threads, ...; a warp's polygons are consecutive).  For its polygon it reads the vertices
// straight from global memory (the L1 keeps them for the second pass), computes the closed box,
// and then classifies the candidates in blocks of NB held in registers: per edge it forms the
// int32 record (c, a, b, y_j) of pip_edge.cuh in registers and applies it to all NB candidates,
// nt = c + p_x a + p_y b = -sign(d_y) det modulo 2^32 and the straddle test as the sign bit of
// (p_y - y_j) ^ (p_y - y_i), carried from edge to edge.  Nothing is staged in shared memory, no
// candidate looks up its owner, and the record of an edge is built once for NB candidates.
//
// Exactness without a box test.  A point is first clamped to [x0 - 1, x1 + 1] x [y0 - 1, y1]
// (x0..x1, y0..y1 the polygon's closed box).  The parity does not change: a point below y0 or at
// or above y1 has no straddling edge before or after; a point left of x0 (right of x1) is left
// (right) of every crossing of its ray before and after, so every (no) straddling edge counts.
// For a clamped point |det| <= (W + 1)|d_y| + (H + 1)|d_x| < 2 (W + 1)(H + 1), so when
// (W + 1)(H + 1) < 2^30 the wrapping 32-bit evaluation gives -sign(d_y) det exactly.  Boxes below
// 2^31 on both sides take the same walk with exact int64 products in the frame of the box's
// corner, and boxes of 2^31 or more the exact 64/128-bit test edge by edge in the same thread:
// correct, but slow, so the autotuner keeps the lockstep kernel for batches with many of those.
//
// Polygons with more than 256 vertices or more than 2^18 (candidate, edge) pairs go on the
// large-polygon list and get bit 0 here, as in the other small-polygon kernels.  Each thread
// writes its block's bits with a masked AND/OR pair per output word (neighbouring polygons share
// words).
#include <algorithm>
#include <climits>
#include <mutex>
#include <type_traits>

#include "pip_device.cuh"
#include "pip_edge.cuh"
#include "pip_launch.h"

namespace pipdev {

constexpr int TP_THREADS = 128;

// Sets bits [c, c + n) of the output to the low n bits of `bits` (n <= 32), the words shared
// with other polygons by a masked AND/OR pair.
__device__ __forceinline__ void put_bits(uint32_t *out, long long c, int n, unsigned bits)
{
    if (n <= 0) return;
    const long long w = c >> 5;
    const int sh = (int)(c & 31);
    const unsigned lowmask = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
    bits &= lowmask;
    masked_store(out + w, lowmask << sh, bits << sh);
    if (sh + n > 32) masked_store(out + w + 1, lowmask >> (32 - sh), bits >> (32 - sh));
}

// A CTA takes groups of TP_G consecutive polygons.  Per group: offsets and large-polygon tests
// (thread per polygon), a counting sort of the polygons with candidates by vertex count (keys
// 0..WP_V) so that the 32 items of a warp walk similar numbers of edges, and a scan that numbers
// the items (polygon, block of NB candidates); threads then take items in that order.  Output
// bits of the group (the candidate range [C0, C1) of its polygons) are gathered in shared memory
// when they fit TP_OB words and written once, plain stores inside and masked ones at the two
// ends; otherwise every item writes its own bits to global memory.
constexpr int TP_G = TP_THREADS;          // polygons of a group
constexpr int TP_KEYS = WP_V + 1;         // sort keys: vertex counts 0..WP_V
constexpr int TP_OB = 1024;               // output words staged per group
constexpr int TP_ITAB = 1024;             // items whose sorted position is tabulated (else a binary search)

template <typename CI>
struct TppSmem {
    unsigned hist[TP_KEYS];               // per key: items (low 24 bits), polygons (high 8 bits)
    CI cb[TP_G];                          // first output bit of each polygon's candidates
    int pb[TP_G];                         // first vertex
    int m[TP_G];                          // vertices
    int n[TP_G];                          // candidates
    int start[TP_G + 1];                  // first item at each sorted position (+ the total)
    unsigned char lp[TP_G];               // polygon (of the group) at each sorted position
    unsigned char ipos[TP_ITAB];          // sorted position of each item, when the group has at most TP_ITAB
    alignas(16) unsigned out[2][TP_OB];   // staged output words, a buffer per group parity (zeroed with 16-byte stores)
    int n_items, n_pos;
    CI c0, c1;                            // candidate range of the group
};

// Exact parity of the candidates c0 .. c0 + nc - 1 of a polygon (vertices v[0..m)) whose box is
// too large for the int32 test: the straddle test and, on straddling edges, the exact side test in
// int64 (int128 beyond 2^31), candidate by candidate.  Rare; out of line so that the int32 walk
// keeps its registers.  Returns the parities as bits 0..nc-1.
template <bool DENSE>
static __device__ __noinline__ unsigned tpp_exact_block(const ClassifyArgs a, const int2 *__restrict__ v, int m,
                                                        long long cbase, int c0, int nc)
{
    unsigned bits = 0;
    for (int j = 0; j < nc; ++j) {
        const long long id = DENSE ? (long long)(c0 + j) : (long long)__ldg(a.cand_ids + cbase + c0 + j);
        if (id < 0 || id >= a.n_points) continue;
        const int2 p = __ldg(a.points + id);
        int par = 0;
        int2 ri = __ldg(v + m - 1);
        for (int e = 0; e < m; ++e) {
            const int2 rj = __ldg(v + e);
            if ((ri.y > p.y) != (rj.y > p.y)) par ^= exact_edge_counts(p.x, p.y, ri.x, ri.y, rj.x, rj.y);
            ri = rj;
        }
        bits |= (unsigned)par << j;
    }
    return bits;
}

template <bool DENSE, bool VERIFY, int NB>
__global__ void __launch_bounds__(TP_THREADS) k_pip_tpp(ClassifyArgs a, LargeList *ll, int lcap)
{
    using CI = typename std::conditional<DENSE, long long, int>::type;
    __shared__ __align__(16) TppSmem<CI> S;
    pdl_trigger();   // the large-polygon kernel may launch now; it waits for this grid to finish
    const int t = threadIdx.x, lane = t & 31;
    const int P = a.n_polys;
    const long long NPTS = a.n_points;
    const CI W32 = (CI)(a.words_per_poly * 32);
    const int ngroups = (P + TP_G - 1) / TP_G;
    unsigned st_cand = 0, st_in = 0, st_err = 0, st_ver = 0, st_fb = 0;
    if (!DENSE && blockIdx.x == 0 && t == 0 && P > 0) {
        // bits past the last candidate in the final word are 0
        const long long C = __ldg(a.cand_offsets + P);
        if (C & 31) masked_store(a.out_bits + (C >> 5), ~((1u << (C & 31)) - 1u), 0u);
    }

    // the histogram is zero at the start of every group: cleared here, and again by each group
    // after its last read (two barriers before the next group's counts)
    for (int i = t; i < TP_KEYS; i += TP_THREADS) S.hist[i] = 0u;
    __syncthreads();
    for (int g = blockIdx.x, it = 0; g < ngroups; g += gridDim.x, ++it) {
        // the group's output words: the buffer the previous group did not use, so that this
        // group's set-up does not wait for the previous group's writes
        unsigned *const outw = S.out[it & 1];
        const int k0 = g * TP_G, np = min(TP_G, P - k0);
        for (int i = t; i < TP_OB / 4; i += TP_THREADS) reinterpret_cast<uint4 *>(outw)[i] = make_uint4(0, 0, 0, 0);
        // ---- polygon k0 + t: offsets, large-polygon test, items, sort key
        int m = 0, n = 0;
        CI cb = 0, ce = 0;
        bool zr = false;                       // bits to zero here (CSR): a large or empty polygon
        bool sorted = false;                   // the polygon has items
        unsigned slot = 0;                     // its place in its key's bucket
        if (t < np) {
            const int k = k0 + t;
            const int pb = __ldg(a.poly_offsets + k);
            m = __ldg(a.poly_offsets + k + 1) - pb;
            if (DENSE) {
                cb = (CI)k * W32;
                ce = cb + W32;
            } else {
                cb = __ldg(a.cand_offsets + k);
                ce = __ldg(a.cand_offsets + k + 1);
            }
            const long long nlen = DENSE ? min(NPTS, (long long)W32) : (long long)(ce - cb);
            const bool lg = is_large_polygon(m, nlen);
            if (lg && ce > cb && NPTS > 0) {
                const int idx = atomicAdd(&ll->count, 1);
                if (idx < lcap) {
                    large_entries(ll)[idx] = k;
                    large_taken(ll, lcap)[idx] = 0;
                } else {
                    atomicExch(&ll->overflow, 1);
                }
            }
            zr = !DENSE && (lg || m <= 0) && ce > cb;
            if (!lg && nlen > 0) {
                n = (int)nlen;                 // below 2^18 when m > 0
                if (m > 0) {
                    const unsigned nb = (unsigned)((n + NB - 1) / NB);
                    slot = atomicAdd(&S.hist[m], (1u << 24) | nb);   // below 2^22 items, 128 polygons a group
                    sorted = true;
                } else {
                    st_cand += (unsigned)n;    // an empty polygon: every candidate outside, bit 0
                }
            }
            S.pb[t] = pb;
            S.m[t] = m;
            S.n[t] = n;
            S.cb[t] = cb;
            if (t == 0) S.c0 = cb;
            if (t == np - 1) S.c1 = ce;
        }
        __syncthreads();
        // ---- exclusive scan of the histogram (warp 0; 9 keys per lane); the two packed fields
        //      never carry into each other
        if (t < 32) {
            constexpr int KPL = (TP_KEYS + 31) / 32;
            unsigned loc[KPL], s = 0;
            #pragma unroll
            for (int i = 0; i < KPL; ++i) {
                const int key = KPL * lane + i;
                loc[i] = key < TP_KEYS ? S.hist[key] : 0u;
                s += loc[i];
            }
            unsigned incl = s;
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            unsigned run = incl - s;
            #pragma unroll
            for (int i = 0; i < KPL; ++i) {
                const int key = KPL * lane + i;
                if (key < TP_KEYS) S.hist[key] = run;
                run += loc[i];
            }
            if (lane == 31) {
                S.n_items = (int)(incl & 0xffffffu);
                S.n_pos = (int)(incl >> 24);
            }
        }
        __syncthreads();
        const CI gc0 = S.c0, gc1 = S.c1;
        const long long gw0 = (long long)gc0 >> 5;
        const long long gnw = gc1 > gc0 ? (((long long)gc1 + 31) >> 5) - gw0 : 0;
        const bool staged = gnw <= TP_OB;
        if (sorted) {
            const unsigned base = S.hist[m] + slot;
            const int pos = (int)(base >> 24), first = (int)(base & 0xffffffu);
            S.lp[pos] = (unsigned char)t;
            S.start[pos] = first;
            if (S.n_items <= TP_ITAB)   // each item's position, so that an item needs no search
                for (int q = first, qe = first + (n + NB - 1) / NB; q < qe; ++q) S.ipos[q] = (unsigned char)pos;
        }
        if (t == 0) S.start[S.n_pos] = S.n_items;
        if (!staged)   // large and empty polygons' bits to 0 (k_pip_large XORs its parities in later)
            for (unsigned zm = __ballot_sync(FULL, zr); zm; zm &= zm - 1) {
                const int l = __ffs(zm) - 1;
                zero_bits(a.out_bits, (long long)__shfl_sync(FULL, cb, l), (long long)__shfl_sync(FULL, ce, l), lane);
            }
        __syncthreads();
        for (int i = t; i < TP_KEYS; i += TP_THREADS) S.hist[i] = 0u;   // read for the last time above
        // ---- items in sorted order: item i is block (i - start[pos]) of the polygon at sorted
        //      position pos, start[pos] <= i < start[pos + 1]
        const int n_items = S.n_items, n_pos = S.n_pos;
        for (int i = t; i < n_items; i += TP_THREADS) {
            int lo = 0;
            if (n_items <= TP_ITAB) {
                lo = S.ipos[i];
            } else {
                int hi = n_pos;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (S.start[mid] <= i) lo = mid; else hi = mid;
                }
            }
            const int l = S.lp[lo];
            const int c0 = (i - S.start[lo]) * NB;
            const int mv = S.m[l];
            const int nc = min(NB, S.n[l] - c0);
            const CI cbv = S.cb[l];
            const int2 *__restrict__ V = a.verts + S.pb[l];
            // candidate ids (issued first), then the polygon's closed box
            int id[NB];
            #pragma unroll
            for (int j = 0; j < NB; ++j) {
                id[j] = -1;
                if (j < nc) id[j] = DENSE ? c0 + j : __ldg(a.cand_ids + cbv + c0 + j);
            }
            int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
            #pragma unroll 4
            for (int e = 0; e < mv; ++e) {
                const int2 q = __ldg(V + e);
                x0 = min(x0, q.x); y0 = min(y0, q.y); x1 = max(x1, q.x); y1 = max(y1, q.y);
            }
            unsigned valid = 0, inm = 0;
            int px[NB], py[NB];
            #pragma unroll
            for (int j = 0; j < NB; ++j) {
                px[j] = x1;   // outside candidates: a point at the top of the box never straddles
                py[j] = y1;
                if (id[j] >= 0 && (long long)id[j] < NPTS) {
                    const int2 p = __ldg(a.points + id[j]);
                    px[j] = p.x;
                    py[j] = p.y;
                    valid |= 1u << j;
                    inm |= (unsigned)(p.x >= x0 && p.x <= x1 && p.y >= y0 && p.y <= y1) << j;
                }
            }
            asm volatile("" : "+r"(inm));   // the box test here: the raw points need not outlive the clamp
            st_cand += __popc(valid);
            st_in += __popc(inm);
            const unsigned W = (unsigned)x1 - (unsigned)x0, H = (unsigned)y1 - (unsigned)y0;
            unsigned bits = 0;
            if (W < (1u << 30) && H < (1u << 30) && (W + 1ULL) * (H + 1ULL) <= (1ULL << 30)) {
                // clamped to [x0 - 1, x1] x [y0 - 1, y1] (same parity); then |det| < 2^31
                int ox[NB], oy[NB];
                #pragma unroll
                for (int j = 0; j < NB; ++j) {
                    ox[j] = px[j];
                    oy[j] = py[j];
                    px[j] = min(px[j] < x0 ? x0 - 1 : px[j], x1);
                    py[j] = min(py[j] < y0 ? y0 - 1 : py[j], y1);
                }
                int2 ri = __ldg(V + mv - 1);
                // NB = 16: p_y - y_i recomputed per edge instead of carried (16 registers fewer)
                constexpr bool CARRY = NB <= 8;
                unsigned u[CARRY ? NB : 1], acc[NB];
                #pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (CARRY) u[j] = (unsigned)py[j] - (unsigned)ri.y;
                    acc[j] = 0;
                }
                // edge ri -> rj: nt = c + p_x a + p_y b = -sign(d_y) det (exact), u = p_y - y; the
                // crossing counts when the sign bits of u_i ^ u_j (straddle) and nt are both set
                #pragma unroll CARRY ? 2 : 1
                for (int e = 0; e < mv; ++e) {
                    const int2 rj = __ldg(V + e);
                    const int4 r = int32_record(ri, rj);
                    #pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        const unsigned uj = (unsigned)py[j] - (unsigned)rj.y;
                        const unsigned ui = CARRY ? u[CARRY ? j : 0] : (unsigned)py[j] - (unsigned)ri.y;
                        const unsigned nt = (unsigned)r.x + (unsigned)px[j] * (unsigned)r.y + (unsigned)py[j] * (unsigned)r.z;
                        if (VERIFY && ((valid >> j) & 1u) && (int)(ui ^ uj) < 0) {
                            st_err += exact_edge_counts(ox[j], oy[j], ri.x, ri.y, rj.x, rj.y) != (int)(nt >> 31);
                            ++st_ver;
                        }
                        acc[j] ^= (ui ^ uj) & nt;
                        if (CARRY) u[CARRY ? j : 0] = uj;
                    }
                    ri = rj;
                }
                #pragma unroll
                for (int j = 0; j < NB; ++j) bits |= (acc[j] >> 31) << j;
            } else if (W < 0x7fffffffu && H < 0x7fffffffu) {
                // boxes below 2^31: the same clamp, then the exact test in int64 in the frame of the
                // box's corner (x0, y0): every clamped difference fits in 32 bits, so
                // nt = (P_x - X_i)|d_y| + (P_y - Y_i)(-s d_x) = -sign(d_y) det takes two 32 x 32 -> 64
                // multiply-adds; the straddle test is the sign bit of (P_y - Y_i) ^ (P_y - Y_j)
                int fx[NB], fy[NB];
                #pragma unroll
                for (int j = 0; j < NB; ++j) {
                    fx[j] = (int)((unsigned)min(px[j] < x0 ? x0 - 1 : px[j], x1) - (unsigned)x0);
                    fy[j] = (int)((unsigned)min(py[j] < y0 ? y0 - 1 : py[j], y1) - (unsigned)y0);
                }
                int2 ri = __ldg(V + mv - 1);
                int ri_x = (int)((unsigned)ri.x - (unsigned)x0), ri_y = (int)((unsigned)ri.y - (unsigned)y0);
                int u[NB];
                unsigned acc[NB];
                #pragma unroll
                for (int j = 0; j < NB; ++j) {
                    u[j] = fy[j] - ri_y;
                    acc[j] = 0;
                }
                for (int e = 0; e < mv; ++e) {
                    const int2 rj = __ldg(V + e);
                    const int rj_x = (int)((unsigned)rj.x - (unsigned)x0), rj_y = (int)((unsigned)rj.y - (unsigned)y0);
                    const int dx = rj_x - ri_x, dy = rj_y - ri_y;   // |d_x| <= W, |d_y| <= H: no overflow
                    const int ady = dy > 0 ? dy : -dy, nsdx = dy > 0 ? -dx : dx;
                    #pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        const int uj = fy[j] - rj_y;
                        const long long nt = (long long)(fx[j] - ri_x) * ady + (long long)u[j] * nsdx;
                        if (VERIFY && ((valid >> j) & 1u) && (u[j] ^ uj) < 0) {
                            st_err += exact_edge_counts(px[j], py[j], ri.x, ri.y, rj.x, rj.y) != (int)(nt < 0);
                            ++st_ver;
                        }
                        acc[j] ^= (unsigned)(u[j] ^ uj) & (unsigned)((unsigned long long)nt >> 32);
                        u[j] = uj;
                    }
                    ri = rj;
                    ri_x = rj_x;
                    ri_y = rj_y;
                }
                #pragma unroll
                for (int j = 0; j < NB; ++j) bits |= (acc[j] >> 31) << j;
            } else if (NB > 8) {
                // (16-candidate blocks keep their registers for the int32 walk)
                bits = tpp_exact_block<DENSE>(a, V, mv, (long long)cbv, c0, nc);
            } else {
                // boxes of 2^31 or more on a side: the FP32 filter in the frame of the box's centre
                // (records from int64 differences) with the forward-error bound 13u (M_x H + M_y W)
                // of pip_edge.cuh, valid for points in the closed box; a point outside it has
                // parity 0 (masked below), and a candidate whose sign came within the bound on a
                // straddling edge is decided exactly
                const unsigned Mx = W - (W >> 1), My = H - (H >> 1);
                const int ox = x0 + (int)(W >> 1), oy = y0 + (int)(H >> 1);
                const float B = __fmul_ru(PM_BOUND_K, __fadd_ru(__fmul_ru(__uint2float_ru(Mx), __uint2float_ru(H)),
                                                                __fmul_ru(__uint2float_ru(My), __uint2float_ru(W))));
                float fx[NB], fy[NB];
                #pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const bool in = (inm >> j) & 1u;
                    fx[j] = in ? __ll2float_rn((long long)px[j] - ox) : 0.f;
                    fy[j] = in ? __ll2float_rn((long long)py[j] - oy) : 0.f;
                }
                int2 ri = __ldg(V + mv - 1);
                unsigned sp = 0, par = 0, unc = 0;   // per candidate: y_i > p_y, parity, uncertain
                #pragma unroll
                for (int j = 0; j < NB; ++j) sp |= (unsigned)(ri.y > py[j]) << j;
                for (int e = 0; e < mv; ++e) {
                    const int2 rj = __ldg(V + e);
                    const float3 r = fp32_record_ll(ri, rj, ox, oy);
                    unsigned sn = 0;
                    #pragma unroll
                    for (int j = 0; j < NB; ++j) sn |= (unsigned)(rj.y > py[j]) << j;
                    const unsigned st = sn ^ sp;   // straddling edges
                    sp = sn;
                    unsigned pos = 0, near = 0;
                    #pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        // tt = det (d_y > 0) or -det (d_y < 0): a straddling edge counts when tt > 0
                        const float tt = __fmaf_rn(fy[j], r.z, __fmaf_rn(-fx[j], r.y, r.x));
                        pos |= (unsigned)(tt > 0.f) << j;
                        near |= (unsigned)(fabsf(tt) <= B) << j;
                        if (VERIFY && ((inm & st) >> j & 1u) && !(fabsf(tt) <= B)) {
                            st_err += exact_edge_counts(px[j], py[j], ri.x, ri.y, rj.x, rj.y) != (int)(tt > 0.f);
                            ++st_ver;
                        }
                    }
                    par ^= pos & st;
                    unc |= near & st;
                    ri = rj;
                }
                bits = par & inm;
                unc &= inm;
                st_fb += __popc(unc);
                for (unsigned q = unc; q; q &= q - 1) {
                    const int j = __ffs(q) - 1;
                    bits = (bits & ~(1u << j)) | (tpp_exact_block<DENSE>(a, V, mv, (long long)cbv, c0 + j, 1) << j);
                }
            }
            bits &= valid;
            // ---- the item's bits
            const long long pos0 = (long long)cbv + c0;
            if (staged) {
                const long long rel = pos0 - (gw0 << 5);
                const long long wi = rel >> 5;
                const int sh = (int)(rel & 31);
                if (wi >= 0 && wi < gnw) atomicOr(&outw[wi], bits << sh);
                if (sh + nc > 32 && wi + 1 >= 0 && wi + 1 < gnw) atomicOr(&outw[wi + 1], bits >> (32 - sh));
            } else {
                put_bits(a.out_bits, pos0, nc, bits);
            }
        }
        __syncthreads();
        // ---- the group's staged words: plain stores inside [C0, C1), masked at the ends
        if (staged)
            for (long long w = t; w < gnw; w += TP_THREADS) {
                const long long b0 = (gw0 + w) << 5;
                const int lo = (int)max(0LL, (long long)gc0 - b0), hi = (int)min(32LL, (long long)gc1 - b0);
                masked_store(a.out_bits + gw0 + w, range_mask(lo, hi), outw[w]);
            }
        // no barrier here: the next group's set-up writes only the other output buffer and
        // shared data that this group last read before its items barrier
    }
    if (a.stats) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st_cand += __shfl_down_sync(FULL, st_cand, o);
            st_in += __shfl_down_sync(FULL, st_in, o);
            st_fb += __shfl_down_sync(FULL, st_fb, o);
            if (VERIFY) st_err += __shfl_down_sync(FULL, st_err, o);
            if (VERIFY) st_ver += __shfl_down_sync(FULL, st_ver, o);
        }
        if (lane == 0) {
            const unsigned st_rej = st_cand - st_in;
            if (VERIFY && st_ver) atomicAdd(a.stats + ST_VERIFIED, (unsigned long long)st_ver);
            if (st_cand) atomicAdd(a.stats + ST_CANDIDATES, (unsigned long long)st_cand);
            if (st_rej) atomicAdd(a.stats + ST_BBOX_REJECTS, (unsigned long long)st_rej);
            if (st_fb) atomicAdd(a.stats + ST_FALLBACK_POINTS, (unsigned long long)st_fb);
            if (VERIFY && st_err) atomicAdd(a.stats + ST_FILTER_ERRORS, (unsigned long long)st_err);
        }
    }
}

// =============================================================================================
// launch
// =============================================================================================

static std::mutex g_tpp_mu;

template <bool DENSE, bool VERIFY, int NB>
static int launch_tpp_t(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int ctas_per_sm,
                        cudaStream_t stream)
{
    static int max_bps[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    int bps = 1;
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lock(g_tpp_mu);
        if (max_bps[dev] == 0) {
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pip_tpp<DENSE, VERIFY, NB>, TP_THREADS, 0) !=
                cudaSuccess)
                nb = 1;
            max_bps[dev] = std::max(nb, 1);
        }
        bps = max_bps[dev];
    }
    if (ctas_per_sm > 0) bps = std::min(bps, ctas_per_sm);
    const long long ngroups = ((long long)a.n_polys + TP_G - 1) / TP_G;
    const int grid = (int)std::max(1LL, std::min((long long)n_sm * bps, ngroups));
    k_pip_tpp<DENSE, VERIFY, NB><<<grid, TP_THREADS, 0, stream>>>(a, ll, lcap);
    note_launch();
    return (int)cudaGetLastError();
}

template <bool DENSE, bool VERIFY>
static int launch_tpp_d(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int block, int ctas_per_sm,
                        cudaStream_t stream)
{
    return block == 8 ? launch_tpp_t<DENSE, VERIFY, 8>(a, ll, lcap, n_sm, ctas_per_sm, stream)
                      : launch_tpp_t<DENSE, VERIFY, 16>(a, ll, lcap, n_sm, ctas_per_sm, stream);
}

int launch_small_tpp(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int block, int ctas_per_sm,
                     bool verify, cudaStream_t stream)
{
    const bool dense = a.cand_offsets == nullptr;
    if (dense)
        return verify ? launch_tpp_d<true, true>(a, ll, lcap, n_sm, block, ctas_per_sm, stream)
                      : launch_tpp_d<true, false>(a, ll, lcap, n_sm, block, ctas_per_sm, stream);
    return verify ? launch_tpp_d<false, true>(a, ll, lcap, n_sm, block, ctas_per_sm, stream)
                  : launch_tpp_d<false, false>(a, ll, lcap, n_sm, block, ctas_per_sm, stream);
}

}  // namespace pipdev
