// Plain exact kernel: every (candidate point, edge) pair in integer arithmetic.
//
// Method section, steps 2-7 with Constraint 1, formulated directly: one warp per output
// word (32 consecutive candidates), one lane per candidate; each lane walks its polygon's
// edges straight from global memory (read-only cache), tests the straddle in int32 and the
// side of the edge with int64 products (128-bit when a difference reaches 2^31), and the
// warp packs the 32 parities with a ballot.  No staging, no local frame, no filter: this
// is the baseline formulation the FP32-filtered kernel is measured against.
//
// The same kernel also evaluates the paper's printed algorithms literally (RULE 1, 2; see
// pip_classify_paper): an edge is a candidate when f_i f_{i+1} <= 0, and it counts when
// (p - r_i) . n <= 0 (Algorithm 1, exact integers) or when the float64 crossing abscissa
// x_i + ((p_y - y_i) / d_y) d_x exceeds p_x (Algorithm 2, each of its three operations rounded
// once, as IEEE float64 does; 0/0 gives NaN, which never counts).
#include "pip_device.cuh"
#include "pip_launch.h"

namespace pipdev {

// Algorithm 1's decision for a candidate edge: (p - r_i) . n <= 0, n = (d_y, -d_x) with
// n_x >= 0.  int64 products when every difference is below 2^31, else 128-bit.
__device__ __forceinline__ int alg1_counts(int px, int py, int xi, int yi, int xj, int yj)
{
    long long nx = (long long)yj - yi, ny = (long long)xi - xj;
    if (nx < 0) { nx = -nx; ny = -ny; }
    const long long ax = (long long)px - xi, ay = (long long)py - yi;
    if (fits31(ax) & fits31(ay) & fits31(nx) & fits31(ny)) return ax * nx + ay * ny <= 0;
    return (__int128)ax * nx + (__int128)ay * ny <= 0;
}

// Algorithm 2's decision for a candidate edge, in float64 with one rounding per operation.
__device__ __forceinline__ int alg2_counts(int px, int py, int xi, int yi, int xj, int yj)
{
    const double dx = (double)((long long)xj - xi), dy = (double)((long long)yj - yi);
    const double l = __ddiv_rn((double)((long long)py - yi), dy);
    const double xn = __dadd_rn((double)xi, __dmul_rn(l, dx));
    return xn > (double)px;
}

template <int RULE>
__global__ void __launch_bounds__(256) k_pip_exact(ClassifyArgs a, long long total_bits)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const bool dense = a.cand_offsets == nullptr;
    const long long C = dense ? total_bits
                              : (a.n_polys > 0 ? (long long)__ldg(a.cand_offsets + a.n_polys) : 0);
    const long long n_words = (C + 31) >> 5;
    const long long W32 = a.words_per_poly * 32;
    unsigned long long n_done = 0;

    for (long long w = warp; w < n_words; w += nwarps) {
        const long long c0 = w << 5, c = c0 + lane;
        int k = -1;
        long long pid = -1;
        if (dense) {
            k = (int)(c0 / W32);
            pid = c - (long long)k * W32;
            if (pid >= a.n_points) k = -1;
        } else {
            int k0 = warp_owner_search(a.cand_offsets, a.n_polys, c0, lane);
            if (k0 >= 0) {
                // ends of the next 32 polygons, then each lane finds its own owner
                long long kk = (long long)k0 + 1 + lane;
                long long end = kk <= a.n_polys ? (long long)__ldg(a.cand_offsets + kk) : LLONG_MAX;
                // first l with end_l > c; [lo, hi) shrinks 32 -> 16 -> 8 -> 4 -> 2 -> 1 -> 0,
                // so six rounds (every lane joins each shuffle)
                int lo = 0, hi = 32;
                #pragma unroll
                for (int s = 0; s < 6; ++s) {
                    const int mid = (lo + hi) >> 1;
                    const long long e = __shfl_sync(FULL, end, mid & 31);
                    if (lo < hi) {
                        if (e <= c) lo = mid + 1; else hi = mid;
                    }
                }
                if (lo < 32) {
                    k = k0 + lo;
                } else {   // more than 32 polygons (empty ones) inside this word
                    int l2 = k0 + 32, h2 = a.n_polys;
                    while (l2 < h2) {
                        int mid = (l2 + h2) >> 1;
                        if ((long long)__ldg(a.cand_offsets + mid + 1) <= c) l2 = mid + 1; else h2 = mid;
                    }
                    k = l2;
                }
            } else if (a.n_polys > 0 && c >= (long long)__ldg(a.cand_offsets)) {
                // cand_offsets[0] > c0 (not a valid CSR): plain per-lane search
                int l2 = 0, h2 = a.n_polys - 1;
                while (l2 < h2) {
                    int mid = (l2 + h2 + 1) >> 1;
                    if ((long long)__ldg(a.cand_offsets + mid) <= c) l2 = mid; else h2 = mid - 1;
                }
                k = l2;
            }
            if (c >= C) k = -1;
            if (k >= 0) {
                pid = __ldg(a.cand_ids + c);
                if (pid < 0 || pid >= a.n_points) k = -1;   // an id outside the points: no candidate
            }
        }
        int inside = 0;
        if (k >= 0) {
            const int2 p = __ldg(a.points + pid);
            const int v0 = __ldg(a.poly_offsets + k), v1 = __ldg(a.poly_offsets + k + 1);
            const int m = v1 - v0;
            if (m > 0 && RULE == 0) {
                int2 r_i = __ldg(a.verts + v1 - 1);   // closing edge first: R_{m-1} -> R_0
                bool s_i = r_i.y > p.y;
                for (int i = 0; i < m; ++i) {
                    const int2 r_j = __ldg(a.verts + v0 + i);
                    const bool s_j = r_j.y > p.y;
                    if (s_i != s_j) inside ^= exact_edge_counts(p.x, p.y, r_i.x, r_i.y, r_j.x, r_j.y);
                    r_i = r_j;
                    s_i = s_j;
                }
            } else if (m > 0) {
                int2 r_i = __ldg(a.verts + v1 - 1);
                int g_i = (r_i.y > p.y) - (r_i.y < p.y);   // sign of f_i
                for (int i = 0; i < m; ++i) {
                    const int2 r_j = __ldg(a.verts + v0 + i);
                    const int g_j = (r_j.y > p.y) - (r_j.y < p.y);
                    if (g_i * g_j <= 0)                      // f_i f_{i+1} <= 0
                        inside ^= RULE == 1 ? alg1_counts(p.x, p.y, r_i.x, r_i.y, r_j.x, r_j.y)
                                            : alg2_counts(p.x, p.y, r_i.x, r_i.y, r_j.x, r_j.y);
                    r_i = r_j;
                    g_i = g_j;
                }
            }
            ++n_done;
        }
        const unsigned word = __ballot_sync(FULL, inside);
        if (lane == 0) a.out_bits[w] = word;
    }
    if (a.stats) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_done += __shfl_down_sync(FULL, n_done, o);
        if (lane == 0 && n_done) atomicAdd(a.stats + ST_EXACT_CANDIDATES, n_done);
    }
}

int launch_exact(const ClassifyArgs &a, long long total_bits, int grid, cudaStream_t stream, int rule)
{
    if (rule == 1) k_pip_exact<1><<<grid, 256, 0, stream>>>(a, total_bits);
    else if (rule == 2) k_pip_exact<2><<<grid, 256, 0, stream>>>(a, total_bits);
    else k_pip_exact<0><<<grid, 256, 0, stream>>>(a, total_bits);
    note_launch();
    return (int)cudaGetLastError();
}

}  // namespace pipdev
