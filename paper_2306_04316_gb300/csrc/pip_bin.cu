// Uniform-grid binning: builds the candidate CSR of a spatial join on the device.
//
// Not part of the paper's method (the paper tests every point against one polygon); this is
// the pre-pass that feeds the batched classify kernel.  Candidates of polygon k are all points
// inside k's CLOSED bounding box -- a necessary condition for being inside k, so no inside
// point is ever dropped.  Steps, all on the device, no host synchronisation:
//   1. polygon bounding boxes (one warp per polygon), the points' bounding box, and the mean
//      polygon extent;
//   2. grid parameters (one thread): cell = requested size, or the mean polygon extent,
//      doubled until the grid has at most 2^24 cells;
//   3. cell id of every point, cell histogram, exclusive scan -> cell start offsets;
//   4. stable LSD radix sort of (cell id, point id) in three passes of 8 bits (so
//      ids ascend within a cell; each pass orders a tile in shared memory first so that its
//      writes are coalesced), then a gather of the points into cell order;
//   5. per polygon (one warp): walk the rows of cells its box covers -- each row is one
//      contiguous range of the sorted points -- and count (pip_bin_count) or write
//      (pip_bin_fill) the points inside the closed box, in that order.
// The count pass writes per-polygon counts into cand_offsets and scans them in place.
#include <algorithm>

#include "pip_device.cuh"
#include "pip_launch.h"

namespace pipdev {

constexpr int BIN_MAX_CELLS_LOG2 = 24;
constexpr long long BIN_MAX_CELLS = 1LL << BIN_MAX_CELLS_LOG2;
constexpr int RADIX_THREADS = 256;
constexpr int RADIX_ITEMS = 16;
constexpr int RADIX_TILE = RADIX_THREADS * RADIX_ITEMS;
constexpr int SCAN_TILE = 1024;     // elements per scan block (256 threads x 4)

struct BinHeader {
    int px0, py0, px1, py1;          // points' bounding box
    long long cell;                  // cell edge in units
    long long gx0, gy0;              // grid origin
    int gnx, gny;                    // grid size in cells
    unsigned long long ext_sum;      // sum over polygons of max(width, height)
    unsigned long long n_nonempty;   // polygons with >= 1 vertex
    long long total;                 // candidates (int64)
    int requested_cell;
    int pad;
};

// Workspace layout (offsets in bytes, each 256-aligned).
struct BinLayout {
    size_t header, poly_bb, keys_a, keys_b, vals_a, vals_b, spts, cell_start, hist, scan_tmp, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

long long scan_tmp_elems(long long n)
{
    long long t = 0;
    while (n > SCAN_TILE) {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        t += n;
    }
    return t + 1;
}

static BinLayout bin_layout(long long N, int P)
{
    BinLayout L;
    const long long nblk = std::max<long long>(1, (N + RADIX_TILE - 1) / RADIX_TILE);
    const long long scan_max = std::max<long long>({BIN_MAX_CELLS + 1, 256 * nblk, (long long)P + 1});
    size_t o = 0;
    L.header = o; o += align256(sizeof(BinHeader));
    L.poly_bb = o; o += align256((size_t)std::max(P, 1) * 16);
    L.keys_a = o; o += align256((size_t)std::max<long long>(N, 1) * 4);
    L.keys_b = o; o += align256((size_t)std::max<long long>(N, 1) * 4);
    L.vals_a = o; o += align256((size_t)std::max<long long>(N, 1) * 4);
    L.vals_b = o; o += align256((size_t)std::max<long long>(N, 1) * 4);
    L.spts = o; o += align256((size_t)std::max<long long>(N, 1) * 8);
    L.cell_start = o; o += align256((size_t)(BIN_MAX_CELLS + 1) * 4);
    L.hist = o; o += align256((size_t)256 * nblk * 4);
    L.scan_tmp = o; o += align256((size_t)scan_tmp_elems(scan_max) * 4);
    L.total = o;
    return L;
}

size_t bin_workspace_bytes(long long n_points, int n_polys) { return bin_layout(n_points, n_polys).total; }

// ------------------------------------------------------------------------------------------
// exclusive scan of uint32 (in place, multi-level)
// ------------------------------------------------------------------------------------------
__global__ void k_scan_block(unsigned *d, long long n, unsigned *block_sums)
{
    __shared__ unsigned s_w[8];
    const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * 4;
    unsigned v[4], sum = 0;
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[i] = base + i < n ? d[base + i] : 0u;
        sum += v[i];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned incl = sum;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        unsigned x = lane < 8 ? s_w[lane] : 0u, xi = x;
        #pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            unsigned t = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < 8) s_w[lane] = xi - x;   // exclusive warp offsets
        if (lane == 7 && block_sums) block_sums[blockIdx.x] = xi;
    }
    __syncthreads();
    unsigned run = s_w[w] + incl - sum;
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (base + i < n) d[base + i] = run;
        run += v[i];
    }
}

__global__ void k_scan_add(unsigned *d, long long n, const unsigned *block_sums)
{
    const unsigned add = block_sums[blockIdx.x];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x)
        if (base + i < n) d[base + i] += add;
}

int scan_exclusive(unsigned *d, long long n, unsigned *tmp, cudaStream_t s)
{
    const long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb <= 1) {
        k_scan_block<<<1, 256, 0, s>>>(d, n, nullptr);
        note_launch();
        return (int)cudaGetLastError();
    }
    k_scan_block<<<(unsigned)nb, 256, 0, s>>>(d, n, tmp);
    note_launch();
    int e = scan_exclusive(tmp, nb, tmp + nb, s);
    if (e) return e;
    k_scan_add<<<(unsigned)nb, 256, 0, s>>>(d, n, tmp);
    note_launch();
    return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// bounding boxes and grid
// ------------------------------------------------------------------------------------------
__global__ void k_bin_init(BinHeader *h, int requested_cell, long long *d_total)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        h->px0 = INT_MAX; h->py0 = INT_MAX; h->px1 = INT_MIN; h->py1 = INT_MIN;
        h->ext_sum = 0; h->n_nonempty = 0; h->total = 0;
        h->requested_cell = requested_cell;
        if (d_total) *d_total = 0;
    }
}

__global__ void k_poly_bbox(const int32_t *__restrict__ po, const int2 *__restrict__ verts, int P, int4 *bb,
                            BinHeader *h)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long ext = 0, nne = 0;
    for (long long k = warp; k < P; k += nw) {
        const int v0 = __ldg(po + k), v1 = __ldg(po + k + 1);
        int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
        for (int i = v0 + lane; i < v1; i += 32) {
            const int2 v = __ldg(verts + i);
            x0 = min(x0, v.x); y0 = min(y0, v.y); x1 = max(x1, v.x); y1 = max(y1, v.y);
        }
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x0 = min(x0, __shfl_xor_sync(FULL, x0, o));
            y0 = min(y0, __shfl_xor_sync(FULL, y0, o));
            x1 = max(x1, __shfl_xor_sync(FULL, x1, o));
            y1 = max(y1, __shfl_xor_sync(FULL, y1, o));
        }
        if (lane == 0) {
            bb[k] = make_int4(x0, y0, x1, y1);
            if (v1 > v0) {
                ext += (unsigned long long)max((long long)x1 - x0, (long long)y1 - y0);
                ++nne;
            }
        }
    }
    if (lane == 0 && nne) {
        atomicAdd(&h->ext_sum, ext);
        atomicAdd(&h->n_nonempty, nne);
    }
}

__global__ void k_points_bbox(const int2 *__restrict__ pts, long long N, BinHeader *h)
{
    int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int2 p = __ldg(pts + i);
        x0 = min(x0, p.x); y0 = min(y0, p.y); x1 = max(x1, p.x); y1 = max(y1, p.y);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = min(x0, __shfl_xor_sync(FULL, x0, o));
        y0 = min(y0, __shfl_xor_sync(FULL, y0, o));
        x1 = max(x1, __shfl_xor_sync(FULL, x1, o));
        y1 = max(y1, __shfl_xor_sync(FULL, y1, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&h->px0, x0); atomicMin(&h->py0, y0); atomicMax(&h->px1, x1); atomicMax(&h->py1, y1);
    }
}

__global__ void k_grid_params(BinHeader *h)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long w = 1, hgt = 1;
    if (h->px0 <= h->px1) {
        w = (long long)h->px1 - h->px0 + 1;
        hgt = (long long)h->py1 - h->py0 + 1;
        h->gx0 = h->px0;
        h->gy0 = h->py0;
    } else {
        h->gx0 = 0;
        h->gy0 = 0;
    }
    long long cell = h->requested_cell;
    if (cell <= 0) cell = h->n_nonempty ? (long long)(h->ext_sum / h->n_nonempty) : 1;
    if (cell < 1) cell = 1;
    long long nx = (w + cell - 1) / cell, ny = (hgt + cell - 1) / cell;
    while (nx * ny > BIN_MAX_CELLS) {
        cell *= 2;
        nx = (w + cell - 1) / cell;
        ny = (hgt + cell - 1) / cell;
    }
    h->cell = cell;
    h->gnx = (int)nx;
    h->gny = (int)ny;
}

__device__ __forceinline__ long long cell_coord(long long v, long long g0, long long cell, int n)
{
    long long c = v < g0 ? 0 : (v - g0) / cell;
    return c >= n ? n - 1 : c;
}

__global__ void k_point_keys(const int2 *__restrict__ pts, long long N, const BinHeader *__restrict__ h,
                             unsigned *keys, int *vals, unsigned *cell_count)
{
    const long long cell = h->cell, gx0 = h->gx0, gy0 = h->gy0;
    const int nx = h->gnx, ny = h->gny;
    // every point lies in [g0, g0 + 2^32): 32-bit offsets and, for cells below 2^32, a 32-bit
    // division instead of a 64-bit one
    const bool narrow = cell <= 0xffffffffLL;
    const unsigned ucell = (unsigned)cell;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int2 p = __ldg(pts + i);
        unsigned id;
        if (narrow) {
            const unsigned cx = min((unsigned)((long long)p.x - gx0) / ucell, (unsigned)(nx - 1));
            const unsigned cy = min((unsigned)((long long)p.y - gy0) / ucell, (unsigned)(ny - 1));
            id = cy * (unsigned)nx + cx;
        } else {
            id = (unsigned)(cell_coord(p.y, gy0, cell, ny) * nx + cell_coord(p.x, gx0, cell, nx));
        }
        keys[i] = id;
        vals[i] = (int)i;
        atomicAdd(cell_count + id, 1u);
    }
}

// ------------------------------------------------------------------------------------------
// stable LSD radix sort pass (digit of `bits` bits at `shift`)
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(RADIX_THREADS) k_radix_hist(const unsigned *__restrict__ keys, long long N,
                                                             int shift, int nblk, unsigned *hist)
{
    __shared__ unsigned cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RADIX_TILE;
    #pragma unroll 4
    for (int r = 0; r < RADIX_ITEMS; ++r) {
        const long long i = base + r * RADIX_THREADS + threadIdx.x;
        if (i < N) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(RADIX_THREADS) k_radix_scatter(const unsigned *__restrict__ kin,
                                                                const int *__restrict__ vin, unsigned *kout,
                                                                int *vout, long long N, int shift, int nblk,
                                                                const unsigned *__restrict__ hist)
{
    // The tile's keys are ranked stably within their digit (tile order = input order), placed
    // in digit order in shared memory, then written out so that consecutive threads write
    // consecutive positions of one digit's run (coalesced), at the run's global start.
    __shared__ unsigned s_base[256];    // global start of digit d's keys from this tile
    __shared__ unsigned s_run[256];     // keys of digit d ranked so far (then: tile count)
    __shared__ unsigned s_lstart[256];  // tile-local start of digit d
    __shared__ unsigned s_wc[RADIX_THREADS / 32][256];
    __shared__ unsigned s_key[RADIX_TILE];
    __shared__ int s_val[RADIX_TILE];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    s_base[tid] = hist[(long long)tid * nblk + blockIdx.x];
    s_run[tid] = 0;
    #pragma unroll
    for (int q = 0; q < RADIX_THREADS / 32; ++q) s_wc[q][tid] = 0;
    const long long base = (long long)blockIdx.x * RADIX_TILE;
    const int nt = (int)min((long long)RADIX_TILE, N - base);
    unsigned key[RADIX_ITEMS];
    int val[RADIX_ITEMS];
    unsigned packed[RADIX_ITEMS];   // digit << 16 | rank within the digit
    #pragma unroll
    for (int r = 0; r < RADIX_ITEMS; ++r) {
        const int i = r * RADIX_THREADS + tid;
        key[r] = i < nt ? kin[base + i] : 0u;
        val[r] = i < nt ? vin[base + i] : 0;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    #pragma unroll
    for (int r = 0; r < RADIX_ITEMS; ++r) {
        const bool valid = r * RADIX_THREADS + tid < nt;
        const unsigned d = valid ? ((key[r] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(FULL, d);
        const unsigned rank = __popc(peers & lt);
        if (valid && (peers & lt) == 0) s_wc[w][d] = __popc(peers);
        __syncthreads();
        unsigned off = 0;
        if (valid) {
            off = s_run[d] + rank;
            for (int q = 0; q < w; ++q) off += s_wc[q][d];
        }
        packed[r] = (d << 16) | off;
        __syncthreads();
        unsigned add = 0;
        #pragma unroll
        for (int q = 0; q < RADIX_THREADS / 32; ++q) { add += s_wc[q][tid]; s_wc[q][tid] = 0; }
        s_run[tid] += add;
        __syncthreads();
    }
    // tile-local digit starts: exclusive scan of s_run over the 256 digits
    {
        const unsigned c = s_run[tid];
        unsigned incl = c;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_wc[0][w] = incl;
        __syncthreads();
        if (w == 0) {
            const unsigned x = lane < RADIX_THREADS / 32 ? s_wc[0][lane] : 0u;
            unsigned xi = x;
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(FULL, xi, o);
                if (lane >= o) xi += t;
            }
            if (lane < RADIX_THREADS / 32) s_wc[1][lane] = xi - x;
        }
        __syncthreads();
        s_lstart[tid] = s_wc[1][w] + incl - c;
        __syncthreads();
    }
    #pragma unroll
    for (int r = 0; r < RADIX_ITEMS; ++r) {
        if (r * RADIX_THREADS + tid < nt) {
            const unsigned d = packed[r] >> 16;
            const unsigned pos = s_lstart[d] + (packed[r] & 0xffffu);
            s_key[pos] = key[r];
            s_val[pos] = val[r];
        }
    }
    __syncthreads();
    for (int i = tid; i < nt; i += RADIX_THREADS) {
        const unsigned k = s_key[i];
        const unsigned d = (k >> shift) & 255u;
        const unsigned g = s_base[d] + (unsigned)i - s_lstart[d];
        kout[g] = k;
        vout[g] = s_val[i];
    }
}

__global__ void k_gather_sorted(const int2 *__restrict__ pts, const int *__restrict__ ids, long long N, int2 *spts)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        spts[i] = __ldg(pts + __ldg(ids + i));
}

// ------------------------------------------------------------------------------------------
// per-polygon candidate count / fill (one warp per polygon)
// ------------------------------------------------------------------------------------------
template <bool FILL>
__global__ void k_poly_candidates(const int4 *__restrict__ bb, const int32_t *__restrict__ po, int P,
                                  const BinHeader *__restrict__ h, const unsigned *__restrict__ cell_start,
                                  const int2 *__restrict__ spts, const int *__restrict__ sids,
                                  unsigned *counts, const int32_t *__restrict__ cand_offsets,
                                  int32_t *cand_ids, long long capacity, long long *d_total)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long cell = h->cell, gx0 = h->gx0, gy0 = h->gy0;
    const int nx = h->gnx, ny = h->gny;
    const bool have_pts = h->px0 <= h->px1;
    unsigned long long tot = 0;
    if (!FILL && warp == 0 && lane == 0) counts[P] = 0;
    for (long long k = warp; k < P; k += nwarp) {
        const int4 b = bb[k];
        long long n = 0;
        long long pos = FILL ? (long long)cand_offsets[k] : 0;
        const bool nonempty = __ldg(po + k + 1) > __ldg(po + k);
        if (nonempty && have_pts && b.z >= h->px0 && b.x <= h->px1 && b.w >= h->py0 && b.y <= h->py1) {
            const long long cx0 = cell_coord(b.x, gx0, cell, nx), cx1 = cell_coord(b.z, gx0, cell, nx);
            const long long cy0 = cell_coord(b.y, gy0, cell, ny), cy1 = cell_coord(b.w, gy0, cell, ny);
            for (long long cy = cy0; cy <= cy1; ++cy) {
                const long long r0 = cell_start[cy * nx + cx0], r1 = cell_start[cy * nx + cx1 + 1];
                // 128 points per step, four loads per lane in flight, tested in order
                for (long long i0 = r0; i0 < r1; i0 += 128) {
                    int2 pp[4];
                    #pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long i = i0 + 32 * u + lane;
                        pp[u] = i < r1 ? spts[i] : make_int2(0, 0);
                    }
                    #pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long i = i0 + 32 * u + lane;
                        const bool in = i < r1 && pp[u].x >= b.x && pp[u].x <= b.z && pp[u].y >= b.y && pp[u].y <= b.w;
                        const unsigned m = __ballot_sync(FULL, in);
                        if (FILL && in) {
                            const long long dst = pos + n + __popc(m & ((1u << lane) - 1u));
                            if (dst < capacity) cand_ids[dst] = sids[i];
                        }
                        n += __popc(m);
                    }
                }
            }
        }
        if (!FILL && lane == 0) {
            counts[k] = (unsigned)n;
            tot += (unsigned long long)n;
        }
    }
    if (!FILL && lane == 0 && tot) atomicAdd(reinterpret_cast<unsigned long long *>(d_total), tot);
}

__global__ void k_bin_finish(BinHeader *h, const long long *d_total, const int32_t *cand_offsets, int P,
                             long long capacity, int32_t *d_overflow)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (d_total) h->total = *d_total;
        if (d_overflow) *d_overflow = h->total > capacity ? 1 : 0;
    }
}

// ------------------------------------------------------------------------------------------
// host launch sequences
// ------------------------------------------------------------------------------------------
int launch_bin_count(const int2 *points, long long N, const int32_t *po, const int2 *verts, int P, int cell_size,
                     void *ws, size_t ws_bytes, int32_t *cand_offsets, long long *d_total, int n_sm,
                     cudaStream_t s)
{
    const BinLayout L = bin_layout(N, P);
    if (ws_bytes < L.total) return (int)cudaErrorInvalidValue;
    char *w = static_cast<char *>(ws);
    BinHeader *h = reinterpret_cast<BinHeader *>(w + L.header);
    int4 *bb = reinterpret_cast<int4 *>(w + L.poly_bb);
    unsigned *ka = reinterpret_cast<unsigned *>(w + L.keys_a), *kb = reinterpret_cast<unsigned *>(w + L.keys_b);
    int *va = reinterpret_cast<int *>(w + L.vals_a), *vb = reinterpret_cast<int *>(w + L.vals_b);
    int2 *spts = reinterpret_cast<int2 *>(w + L.spts);
    unsigned *cstart = reinterpret_cast<unsigned *>(w + L.cell_start);
    unsigned *hist = reinterpret_cast<unsigned *>(w + L.hist);
    unsigned *tmp = reinterpret_cast<unsigned *>(w + L.scan_tmp);
    const int grid = n_sm * 8;
    int e;

    k_bin_init<<<1, 32, 0, s>>>(h, cell_size, d_total);
    if (P > 0) k_poly_bbox<<<grid, 256, 0, s>>>(po, verts, P, bb, h);
    if (N > 0) k_points_bbox<<<grid, 256, 0, s>>>(points, N, h);
    k_grid_params<<<1, 32, 0, s>>>(h);
    note_launch(2 + (P > 0) + (N > 0));
    if ((e = (int)cudaMemsetAsync(cstart, 0, (size_t)(BIN_MAX_CELLS + 1) * 4, s))) return e;
    if (N > 0) {
        k_point_keys<<<grid, 256, 0, s>>>(points, N, h, ka, va, cstart);
        note_launch();
        if ((e = scan_exclusive(cstart, BIN_MAX_CELLS + 1, tmp, s))) return e;
        const int nblk = (int)((N + RADIX_TILE - 1) / RADIX_TILE);
        const int shifts[3] = {0, 8, 16};
        for (int pass = 0; pass < 3; ++pass) {
            k_radix_hist<<<nblk, RADIX_THREADS, 0, s>>>(ka, N, shifts[pass], nblk, hist);
            note_launch();
            if ((e = scan_exclusive(hist, 256LL * nblk, tmp, s))) return e;
            k_radix_scatter<<<nblk, RADIX_THREADS, 0, s>>>(ka, va, kb, vb, N, shifts[pass], nblk, hist);
            note_launch();
            std::swap(ka, kb);
            std::swap(va, vb);
        }
        // after three passes the sorted ids are in the buffer that started as vals_b
        k_gather_sorted<<<grid, 256, 0, s>>>(points, va, N, spts);
        note_launch();
    }
    if (P > 0) {
        k_poly_candidates<false><<<grid, 256, 0, s>>>(bb, po, P, h, cstart, spts, va,
                                                      reinterpret_cast<unsigned *>(cand_offsets), nullptr,
                                                      nullptr, 0, d_total);
        note_launch();
        if ((e = scan_exclusive(reinterpret_cast<unsigned *>(cand_offsets), (long long)P + 1, tmp, s))) return e;
    } else {
        if ((e = (int)cudaMemsetAsync(cand_offsets, 0, 4, s))) return e;
    }
    k_bin_finish<<<1, 32, 0, s>>>(h, d_total, cand_offsets, P, 0, nullptr);
    note_launch();
    return (int)cudaGetLastError();
}

int launch_bin_fill(const int2 *points, long long N, const int32_t *po, const int2 *verts, int P, void *ws,
                    size_t ws_bytes, const int32_t *cand_offsets, int32_t *cand_ids, long long capacity,
                    int32_t *d_overflow, int n_sm, cudaStream_t s)
{
    const BinLayout L = bin_layout(N, P);
    if (ws_bytes < L.total) return (int)cudaErrorInvalidValue;
    char *w = static_cast<char *>(ws);
    BinHeader *h = reinterpret_cast<BinHeader *>(w + L.header);
    const int4 *bb = reinterpret_cast<const int4 *>(w + L.poly_bb);
    // sorted ids after three passes: vals_b (odd number of swaps)
    const int *sids = reinterpret_cast<const int *>(w + L.vals_b);
    const int2 *spts = reinterpret_cast<const int2 *>(w + L.spts);
    const unsigned *cstart = reinterpret_cast<const unsigned *>(w + L.cell_start);
    const int grid = n_sm * 8;
    if (P > 0 && N > 0) {
        k_poly_candidates<true><<<grid, 256, 0, s>>>(bb, po, P, h, cstart, spts, sids, nullptr, cand_offsets,
                                                     cand_ids, capacity, nullptr);
        note_launch();
    }
    k_bin_finish<<<1, 32, 0, s>>>(h, nullptr, cand_offsets, P, capacity, d_overflow);
    note_launch();
    return (int)cudaGetLastError();
}

}  // namespace pipdev
