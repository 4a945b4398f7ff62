// FP32-filtered persistent kernel with an exact integer recheck.
//
// Method section, steps 2-7 with Constraint 1.  For the edge R_i -> R_j of a polygon and a
// candidate point p, the crossing counts when the straddle test (y_i > p_y) != (y_j > p_y)
// holds (int32, exact) and sign(d_y) * det > 0, where det = (x_i - p_x) d_y - (y_i - p_y) d_x
// is the paper's side test (p - R_i) . n up to the sign fixed by orienting n so that
// n_x >= 0.  Parity of the count = inside bit.
//
// Local frame and FP32 evaluation.  Every polygon (or, for polygons too large for one
// shared-memory pass, every tile of edges together with the tile's candidate points) gets
// an integer origin o at the centre of a box that holds all vertices and points used with
// it; M_x, M_y bound |x - o_x|, |y - o_y| over that box.  Per edge the staging pass stores
//     c' = s (X_i d_y - Y_i d_x)   (X = x - o_x, Y = y - o_y, s = sign(d_y); int64 exact,
//                                   rounded once to FP32; double for frames >= 2^30)
//     a = |d_y|,  b = s d_x        (rounded to FP32)
//     B = 8.5 * 2^-24 (M_x |d_y| + M_y |d_x|)   (FP32, every operation rounded upward)
// and per (point, edge) pair the kernel evaluates t = fma(P_y, b, fma(-P_x, a, c')) with
// P = p - o rounded to FP32, so that t approximates s * det.  Forward error: with
// S = M_x |d_y| + M_y |d_x| and u = 2^-24, rounding c' costs <= (u + 2^-51) S, rounding
// P_x, P_y, a, b costs <= (2u + u^2) S in the two products, and the two fused operations
// cost <= u (2 + 4u) S and <= u (3 + 8u) S; in total < 8.01 u S <= B.  Hence |t| > B
// implies sign(t) = sign(s det) and det != 0, and only pairs with a straddle and |t| <= B
// need the exact 64/128-bit recheck, which the kernel runs in place.  Points outside
// their polygon's closed bounding box are outside the polygon (the count of straddling
// edges is even and all crossings lie on one side of p), so they skip the edge loop.
//
// Work decomposition.  Candidates are cut into chunks of 256 * PPT consecutive candidates
// (whole output words).  A persistent CTA takes chunks in a strided order; a warp finds the
// polygon owning the chunk's first candidate with 32-way probes of cand_offsets; the CTA
// stages the offsets of the next 256 polygons, then the vertices of as many whole polygons
// as fit in a tile of T edges, computes each polygon's frame (bounding box by shared-memory
// atomics) and edge records, and every thread walks its candidates' polygons' edges from
// shared memory.  A polygon with more than T edges streams through shared memory in tiles,
// each tile framed by the union of its vertices and the chunk's candidate points; parities
// of the tiles combine by XOR.  Each warp packs its 32 parities with a ballot and writes
// whole words (a chunk owns its words, so no atomics are needed).
#include <algorithm>

#include "pip_device.cuh"
#include "pip_launch.h"

namespace pipdev {

constexpr int FT_THREADS = 256;
constexpr int FT_WIN = 256;                              // polygons per offsets window
constexpr float FT_BOUND_K = 5.066394805908203125e-07f;  // 8.5 * 2^-24 (exact in FP32)

size_t filtered_smem_bytes(int T)
{
    // records float4[T], vertices int2[T + 1], next-y int[T], vertex owner ushort[T]
    size_t b = (size_t)T * 16 + (size_t)(T + 1) * 8 + (size_t)T * 4 + (size_t)T * 2;
    return (b + 15) & ~(size_t)15;
}

struct Frame {
    int ox, oy;
    float mx, my;   // upper bounds of |x - ox|, |y - oy| over the frame's box
    int wide;       // M >= 2^30: form c' in double
};

__device__ __forceinline__ Frame make_frame(int xmin, int ymin, int xmax, int ymax)
{
    Frame f;
    long long ox = (long long)xmin + (((long long)xmax - xmin) >> 1);
    long long oy = (long long)ymin + (((long long)ymax - ymin) >> 1);
    long long Mx = max((long long)xmax - ox, ox - xmin);
    long long My = max((long long)ymax - oy, oy - ymin);
    f.ox = (int)ox;
    f.oy = (int)oy;
    f.mx = __ll2float_ru(Mx);
    f.my = __ll2float_ru(My);
    f.wide = (Mx >= (1LL << 30)) | (My >= (1LL << 30));
    return f;
}

// Edge record of R_i -> R_j in frame f: (c', |d_y|, s d_x, B).  Horizontal edges never
// straddle, so their record is never used for a decision.
__device__ __forceinline__ float4 make_record(int2 ri, int2 rj, int ox, int oy, float mx, float my,
                                              int wide)
{
    const long long dx = (long long)rj.x - ri.x, dy = (long long)rj.y - ri.y;
    if (dy == 0) return make_float4(0.f, 0.f, 0.f, 0.f);
    const long long X = (long long)ri.x - ox, Y = (long long)ri.y - oy;
    float c;
    if (!wide) {
        c = __ll2float_rn(X * dy - Y * dx);              // |X dy|, |Y dx| < 2^61: exact int64
    } else {
        c = __double2float_rn(__dmul_rn((double)X, (double)dy) - __dmul_rn((double)Y, (double)dx));
    }
    const long long ady = dy > 0 ? dy : -dy;
    const long long adx = dx >= 0 ? dx : -dx;
    const float B = __fmul_ru(FT_BOUND_K, __fadd_ru(__fmul_ru(mx, __ll2float_ru(ady)),
                                                    __fmul_ru(my, __ll2float_ru(adx))));
    return make_float4(dy > 0 ? c : -c, __ll2float_rn(ady), __ll2float_rn(dy > 0 ? dx : -dx), B);
}

// Parity over edges [e0, e1) of the staged tile.  Edge e runs from s_v[e] to s_v[nx(e)],
// nx(e) = e + 1, or e0 for the last edge when `wrap` (a whole polygon in the tile).
__device__ __forceinline__ int tile_parity(const float4 *__restrict__ s_rec, const int *__restrict__ s_yn,
                                           const int2 *__restrict__ s_v, int e0, int e1, bool wrap,
                                           int2 p, int ox, int oy, unsigned long long &n_fb_pts,
                                           unsigned long long &n_fb_edges)
{
    const float Px = __ll2float_rn((long long)p.x - ox);
    const float Py = __ll2float_rn((long long)p.y - oy);
    bool sp = s_v[e0].y > p.y;
    int parity = 0, unc = 0;
    for (int e = e0; e < e1; ++e) {
        const float4 q = s_rec[e];
        const bool s = s_yn[e] > p.y;
        const bool st = s != sp;
        sp = s;
        float t = __fmaf_rn(-Px, q.y, q.x);
        t = __fmaf_rn(Py, q.z, t);
        parity ^= (int)(st & (t > 0.f));
        unc += (int)(st & (fabsf(t) <= q.w));
    }
    if (unc) {
        // some sign was within the error bound: redo this candidate exactly
        ++n_fb_pts;
        n_fb_edges += (unsigned long long)unc;
        parity = 0;
        for (int e = e0; e < e1; ++e) {
            const int nx = (wrap && e + 1 == e1) ? e0 : e + 1;
            const int2 ri = s_v[e], rj = s_v[nx];
            if ((ri.y > p.y) != (rj.y > p.y)) parity ^= exact_edge_counts(p.x, p.y, ri.x, ri.y, rj.x, rj.y);
        }
    }
    return parity;
}

template <int PPT>
__global__ void __launch_bounds__(FT_THREADS) k_pip_filtered(ClassifyArgs a, long long total_bits, int T)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *s_rec = reinterpret_cast<float4 *>(dsm);
    int2 *s_v = reinterpret_cast<int2 *>(s_rec + T);
    int *s_yn = reinterpret_cast<int *>(s_v + T + 1);
    unsigned short *s_vp = reinterpret_cast<unsigned short *>(s_yn + T);

    __shared__ long long s_co[FT_WIN + 1];
    __shared__ int s_po[FT_WIN + 1];
    __shared__ int s_bb[FT_WIN][4];
    __shared__ Frame s_fr[FT_WIN];
    __shared__ int s_pb[4], s_tb[4];
    __shared__ Frame s_tf;
    __shared__ int s_k0;

    constexpr int CH = FT_THREADS * PPT;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool dense = a.cand_offsets == nullptr;
    const int P = a.n_polys;
    const long long C = dense ? total_bits : (P > 0 ? (long long)__ldg(a.cand_offsets + P) : 0);
    const long long nchunks = (C + CH - 1) / CH;
    const long long W32 = a.words_per_poly * 32;
    const int end_v = P > 0 ? __ldg(a.poly_offsets + P) : 0;
    unsigned long long st_cand = 0, st_rej = 0, st_fbp = 0, st_fbe = 0;

    for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const long long c0 = ch * CH, c1 = min(c0 + CH, C);
        long long cc[PPT];
        int2 pt[PPT];
        int jj[PPT], par[PPT];
        #pragma unroll
        for (int r = 0; r < PPT; ++r) {
            cc[r] = c0 + tid + r * FT_THREADS;
            par[r] = 0;
            pt[r] = make_int2(0, 0);
            if (!dense && cc[r] < c1) pt[r] = __ldg(a.points + __ldg(a.cand_ids + cc[r]));
        }
        if (wid == 0) {
            int k0 = dense ? (int)(c0 / W32) : warp_owner_search(a.cand_offsets, P, c0, lane);
            if (lane == 0) s_k0 = k0 < 0 ? 0 : k0;
        }
        __syncthreads();
        int kw = s_k0;
        while (true) {
            for (int j = tid; j <= FT_WIN; j += FT_THREADS) {
                const long long k = (long long)kw + j;
                if (k <= P) {
                    s_co[j] = dense ? k * W32 : (long long)__ldg(a.cand_offsets + k);
                    s_po[j] = __ldg(a.poly_offsets + k);
                } else {
                    s_co[j] = LLONG_MAX;
                    s_po[j] = end_v;
                }
            }
            __syncthreads();
            const long long win_end = s_co[FT_WIN];
            #pragma unroll
            for (int r = 0; r < PPT; ++r) {
                jj[r] = -1;
                if (cc[r] < c1 && cc[r] >= s_co[0] && cc[r] < win_end) {
                    const int j = upper_bound_dev(s_co, FT_WIN + 1, cc[r]) - 1;
                    jj[r] = j;
                    if (dense) {
                        const long long pid = cc[r] - ((long long)kw + j) * W32;
                        if (pid < a.n_points) pt[r] = __ldg(a.points + pid); else jj[r] = -1;
                    }
                    if (jj[r] >= 0) ++st_cand;
                }
            }
            const int nw = min(FT_WIN, upper_bound_dev(s_co, FT_WIN + 1, c1 - 1));
            int jb = 0;
            while (jb < nw) {
                const int base = s_po[jb];
                // largest je in [jb, nw] with s_po[je] - base <= T
                int lo = jb, hi = nw;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if ((long long)s_po[mid] - base <= T) lo = mid; else hi = mid - 1;
                }
                const int je = lo;
                if (je > jb) {
                    // ---- small polygons [jb, je): whole polygons in one tile ----
                    const int nv = s_po[je] - base;
                    for (int i = tid; i < nv; i += FT_THREADS) {
                        s_v[i] = __ldg(a.verts + base + i);
                        s_vp[i] = (unsigned short)(jb + upper_bound_dev(s_po + jb, je - jb + 1, base + i) - 1);
                    }
                    for (int j = jb + tid; j < je; j += FT_THREADS) {
                        s_bb[j][0] = INT_MAX; s_bb[j][1] = INT_MAX;
                        s_bb[j][2] = INT_MIN; s_bb[j][3] = INT_MIN;
                    }
                    __syncthreads();
                    for (int i = tid; i < nv; i += FT_THREADS) {
                        const int j = s_vp[i];
                        const int2 v = s_v[i];
                        atomicMin(&s_bb[j][0], v.x); atomicMin(&s_bb[j][1], v.y);
                        atomicMax(&s_bb[j][2], v.x); atomicMax(&s_bb[j][3], v.y);
                    }
                    __syncthreads();
                    for (int j = jb + tid; j < je; j += FT_THREADS)
                        if (s_po[j + 1] > s_po[j]) s_fr[j] = make_frame(s_bb[j][0], s_bb[j][1], s_bb[j][2], s_bb[j][3]);
                    __syncthreads();
                    for (int i = tid; i < nv; i += FT_THREADS) {
                        const int j = s_vp[i];
                        const int nx = (i + 1 == s_po[j + 1] - base) ? s_po[j] - base : i + 1;
                        const Frame f = s_fr[j];
                        const int2 rj = s_v[nx];
                        s_rec[i] = make_record(s_v[i], rj, f.ox, f.oy, f.mx, f.my, f.wide);
                        s_yn[i] = rj.y;
                    }
                    __syncthreads();
                    #pragma unroll
                    for (int r = 0; r < PPT; ++r) {
                        const int j = jj[r];
                        if (j >= jb && j < je) {
                            const int e0 = s_po[j] - base, e1 = s_po[j + 1] - base;
                            const int2 p = pt[r];
                            if (e1 == e0 || p.x < s_bb[j][0] || p.x > s_bb[j][2] || p.y < s_bb[j][1] ||
                                p.y > s_bb[j][3]) {
                                ++st_rej;
                                par[r] = 0;
                            } else {
                                const Frame f = s_fr[j];
                                par[r] = tile_parity(s_rec, s_yn, s_v, e0, e1, true, p, f.ox, f.oy, st_fbp, st_fbe);
                            }
                        }
                    }
                    __syncthreads();
                    jb = je;
                } else {
                    // ---- one polygon with more than T edges: stream its edges in tiles ----
                    const int m = s_po[jb + 1] - base;
                    if (tid == 0) { s_pb[0] = INT_MAX; s_pb[1] = INT_MAX; s_pb[2] = INT_MIN; s_pb[3] = INT_MIN; }
                    __syncthreads();
                    #pragma unroll
                    for (int r = 0; r < PPT; ++r)
                        if (jj[r] == jb) {
                            atomicMin(&s_pb[0], pt[r].x); atomicMin(&s_pb[1], pt[r].y);
                            atomicMax(&s_pb[2], pt[r].x); atomicMax(&s_pb[3], pt[r].y);
                        }
                    __syncthreads();
                    const bool any = s_pb[0] <= s_pb[2];
                    for (int e0 = 0; any && e0 < m; e0 += T) {
                        const int nt = min(T, m - e0);
                        if (tid == 0) {
                            s_tb[0] = s_pb[0]; s_tb[1] = s_pb[1]; s_tb[2] = s_pb[2]; s_tb[3] = s_pb[3];
                        }
                        for (int i = tid; i <= nt; i += FT_THREADS) {
                            int g = e0 + i;
                            if (g >= m) g -= m;
                            s_v[i] = __ldg(a.verts + base + g);
                        }
                        __syncthreads();
                        for (int i = tid; i <= nt; i += FT_THREADS) {
                            const int2 v = s_v[i];
                            atomicMin(&s_tb[0], v.x); atomicMin(&s_tb[1], v.y);
                            atomicMax(&s_tb[2], v.x); atomicMax(&s_tb[3], v.y);
                        }
                        __syncthreads();
                        if (tid == 0) s_tf = make_frame(s_tb[0], s_tb[1], s_tb[2], s_tb[3]);
                        __syncthreads();
                        const Frame f = s_tf;
                        for (int i = tid; i < nt; i += FT_THREADS) {
                            const int2 rj = s_v[i + 1];
                            s_rec[i] = make_record(s_v[i], rj, f.ox, f.oy, f.mx, f.my, f.wide);
                            s_yn[i] = rj.y;
                        }
                        __syncthreads();
                        #pragma unroll
                        for (int r = 0; r < PPT; ++r)
                            if (jj[r] == jb)
                                par[r] ^= tile_parity(s_rec, s_yn, s_v, 0, nt, false, pt[r], f.ox, f.oy, st_fbp, st_fbe);
                        __syncthreads();
                    }
                    jb += 1;
                }
            }
            if (nw < FT_WIN || win_end >= c1) break;
            kw += FT_WIN;
            __syncthreads();
        }
        #pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const unsigned w = __ballot_sync(FULL, par[r]);
            const long long word = (c0 + r * FT_THREADS + wid * 32) >> 5;
            if (lane == 0 && (word << 5) < C) a.out_bits[word] = w;
        }
        __syncthreads();
    }
    if (a.stats) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st_cand += __shfl_down_sync(FULL, st_cand, o);
            st_rej += __shfl_down_sync(FULL, st_rej, o);
            st_fbp += __shfl_down_sync(FULL, st_fbp, o);
            st_fbe += __shfl_down_sync(FULL, st_fbe, o);
        }
        if (lane == 0) {
            if (st_cand) atomicAdd(a.stats + ST_CANDIDATES, st_cand);
            if (st_rej) atomicAdd(a.stats + ST_BBOX_REJECTS, st_rej);
            if (st_fbp) atomicAdd(a.stats + ST_FALLBACK_POINTS, st_fbp);
            if (st_fbe) atomicAdd(a.stats + ST_FALLBACK_EDGES, st_fbe);
        }
    }
}

template <int PPT>
static int launch_ppt(const ClassifyArgs &a, long long total_bits, int T, int grid, cudaStream_t stream)
{
    const size_t smem = filtered_smem_bytes(T);
    static size_t configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && configured[dev] < smem) {
        cudaError_t e = cudaFuncSetAttribute(k_pip_filtered<PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return (int)e;
        configured[dev] = smem;
    }
    k_pip_filtered<PPT><<<grid, FT_THREADS, smem, stream>>>(a, total_bits, T);
    return (int)cudaGetLastError();
}

int launch_filtered(const ClassifyArgs &a, long long total_bits, const Tuning &t, int n_sm, cudaStream_t stream)
{
    long long grid = (long long)n_sm * t.ctas_per_sm;
    if (a.cand_offsets == nullptr) {
        const long long ch = (long long)FT_THREADS * t.pts_per_thread;
        grid = std::min(grid, (total_bits + ch - 1) / ch);
    }
    if (grid < 1) grid = 1;
    switch (t.pts_per_thread) {
        case 1: return launch_ppt<1>(a, total_bits, t.edge_tile, (int)grid, stream);
        case 2: return launch_ppt<2>(a, total_bits, t.edge_tile, (int)grid, stream);
        default: return launch_ppt<4>(a, total_bits, t.edge_tile, (int)grid, stream);
    }
}

}  // namespace pipdev
