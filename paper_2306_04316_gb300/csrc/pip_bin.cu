// Uniform-grid binning: builds the candidate CSR of a spatial join on the device.
//
// Not part of the paper's method (the paper tests every point against one polygon); this is
// the pre-pass that feeds the batched classify kernel.  Candidates of polygon k are all points
// inside k's CLOSED bounding box -- a necessary condition for being inside k, so no inside
// point is ever dropped.  The polygons are binned, not the points, so no pass ever sorts the
// points: steps 1-3 build a polygon index (pip_bin_index, once per polygon set), steps 4-5
// probe it with a batch of points (pip_bin_probe_count / pip_bin_probe_fill; several batches
// may probe one index at once, each with its own probe workspace).  pip_bin_count and
// pip_bin_fill run both on one workspace.  All on the device, no host synchronisation:
//   1. polygon bounding boxes (one warp per polygon); lane l of the warp also counts the cells
//      of edge 2^l that the box covers, for every level l at once;
//   2. the level (one warp, a lane per level): the finest cell edge 2^l at which the
//      (polygon, cell) pairs of the boxes covering at most 64 cells fit the pair list (4 per
//      polygon + 1024), with at most 256 larger boxes -- those go on a short list that every
//      point tests directly;
//   3. the occupied cells in an open-addressing hash table keyed by the cell (cx, cy),
//      cx = (x + 2^31) >> l: insert, count polygons per cell, scan, fill the per-cell lists
//      (each entry a copy of the polygon's box, so that a point reads its cell's slot -- key,
//      first entry and count in 16 bytes -- and then one contiguous run of boxes);
//   4. per point (one thread): its cell's polygons and the short list, each box tested; the
//      count pass counts per polygon with atomics, scans the counts into cand_offsets and
//      records the (polygon, point) pairs in the probe workspace; the fill pass places each
//      recorded id by an atomic cursor (probing the points again only if more pairs were found
//      than the workspace records: N / 2 + 1024);
//   5. every polygon's id list sorted ascending (bitonic: one lane per polygon in its registers
//      up to 16 ids; longer lists queued for one warp each, in its registers up to 32 or its
//      shared memory up to 1024, or for one CTA each, in shared memory up to 8192, else in place
//      in global memory), so that the CSR is the same on every run.
#include <algorithm>

#include "pip_device.cuh"
#include "pip_launch.h"

namespace pipdev {

constexpr int BIN_CELL_CAP = 64;       // boxes covering more cells than this go on the short list
constexpr int BIN_BIG_CAP = 256;       // most polygons on the short list
constexpr int BIN_PACK_LEVEL = 16;     // cell edges up to 2^16: list boxes stored in 8 bytes, relative to the cell
constexpr unsigned long long BIN_EMPTY = ~0ull;   // an empty hash slot (cx < 2^31 for level >= 1)
constexpr int SCAN_TILE = 1024;        // elements per scan block (256 threads x 4)
constexpr int SORT_LANE = 16;          // ids a lane sorts in its registers
constexpr int SORT_WARP_REG = 4;       // ids a lane holds when a warp sorts a list in registers (128 a warp)
constexpr int SORT_WARP_SMEM = 512;    // ids a warp sorts in its own shared memory
constexpr int SORT_CTA_SMEM = 8192;    // ids a CTA sorts in shared memory

constexpr unsigned INDEX_MAGIC = 0x50495849u;   // a polygon index whose build has completed

// The polygon index: built once per polygon set, read-only while batches of points probe it.
struct IndexHeader {
    unsigned long long cells[32];    // cells[l]: (polygon, cell) pairs of the boxes with <= BIN_CELL_CAP cells
    unsigned long long big[32];      // big[l]: boxes with more cells than that, at cell edge 2^l
    int level;                       // chosen cell edge 2^level
    int n_big;                       // polygons on the short list
    int requested_level;             // 0: automatic
    int n_polys;                     // polygons indexed
    unsigned magic;                  // INDEX_MAGIC once the build has completed
    int pad[3];
};

// State of one batch's probe passes.
struct ProbeHeader {
    long long total;                 // candidates (int64)
    unsigned long long n_pairs;      // (polygon, point) pairs the count pass recorded
    int n_long;                      // id lists queued for the CTA-wide sort
    int n_medium;                    // id lists queued for the warp-wide sort
};

// Layouts (offsets in bytes, each 256-aligned).  The index is sized by the polygon count only.
struct IndexLayout {
    size_t header, poly_bb, ent, cnt, off, list_bb, list_id, big, scan_tmp, total;
    long long H, lcap;               // hash slots (a power of two), pair-list capacity
    int hbits;
};
struct ProbeLayout {
    size_t header, cursor, medium_list, long_list, pairs, scan_tmp, total;
    long long pcap;                  // (polygon, point) pairs the count pass can record
};

// A slot of the cell table: the cell's key, then (first list entry, polygons) once built.
struct __align__(16) CellEntry {
    unsigned long long key;
    int start, count;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static long long pair_capacity(int P) { return 4LL * P + 1024; }

long long scan_tmp_elems(long long n)
{
    long long t = 0;
    while (n > SCAN_TILE) {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        t += n;
    }
    return t + 1;
}

static IndexLayout index_layout(int P)
{
    IndexLayout L;
    L.lcap = pair_capacity(P);
    L.hbits = 1;
    while ((1LL << L.hbits) < 4 * L.lcap) ++L.hbits;   // at most a quarter full
    L.H = 1LL << L.hbits;
    size_t o = 0;
    L.header = o; o += align256(sizeof(IndexHeader));
    L.poly_bb = o; o += align256((size_t)std::max(P, 1) * 16);
    L.ent = o; o += align256((size_t)L.H * sizeof(CellEntry));
    L.cnt = o; o += align256((size_t)L.H * 4);
    L.off = o; o += align256((size_t)L.H * 4);
    L.list_bb = o; o += align256((size_t)L.lcap * 16);
    L.list_id = o; o += align256((size_t)L.lcap * 4);
    L.big = o; o += align256((size_t)BIN_BIG_CAP * 4);
    L.scan_tmp = o; o += align256((size_t)scan_tmp_elems(L.H) * 4);
    L.total = o;
    return L;
}

static ProbeLayout probe_layout(long long N, int P)
{
    ProbeLayout L;
    L.pcap = N / 2 + 1024;
    size_t o = 0;
    L.header = o; o += align256(sizeof(ProbeHeader));
    L.cursor = o; o += align256((size_t)std::max(P, 1) * 4);
    L.medium_list = o; o += align256((size_t)std::max(P, 1) * 4);
    L.long_list = o; o += align256((size_t)std::max(P, 1) * 4);
    L.pairs = o; o += align256((size_t)L.pcap * 8);
    L.scan_tmp = o; o += align256((size_t)scan_tmp_elems((long long)P + 1) * 4);
    L.total = o;
    return L;
}

size_t bin_index_bytes(int n_polys) { return index_layout(n_polys).total; }
size_t bin_probe_bytes(long long n_points, int n_polys) { return probe_layout(n_points, n_polys).total; }
// pip_bin_count / pip_bin_fill: the index, then one probe workspace
size_t bin_workspace_bytes(long long n_points, int n_polys)
{
    return bin_index_bytes(n_polys) + bin_probe_bytes(n_points, n_polys);
}

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
// polygon boxes and the level
// ------------------------------------------------------------------------------------------
__global__ void k_index_init(IndexHeader *h, int requested_level, int P)
{
    const int t = threadIdx.x;
    if (blockIdx.x == 0 && t < 32) {
        h->cells[t] = 0;
        h->big[t] = 0;
        if (t == 0) {
            h->level = 31;
            h->n_big = 0;
            h->requested_level = requested_level;
            h->n_polys = P;
            h->magic = 0;
        }
    }
}

__global__ void k_index_finish(IndexHeader *h)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) h->magic = INDEX_MAGIC;
}

__global__ void k_probe_init(ProbeHeader *q, long long *d_total)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        q->total = 0;
        q->n_pairs = 0;
        q->n_long = 0;
        q->n_medium = 0;
        if (d_total) *d_total = 0;
    }
}

// the index was built, for this many polygons
__device__ __forceinline__ bool index_ok(const IndexHeader *h, int P)
{
    return h->magic == INDEX_MAGIC && h->n_polys == P;
}

// cell coordinate of x at level l: (x + 2^31) >> l
__device__ __forceinline__ unsigned cell_of(int x, int l) { return ((unsigned)x ^ 0x80000000u) >> l; }

__device__ __forceinline__ unsigned long long cell_key(unsigned cx, unsigned cy)
{
    return ((unsigned long long)cy << 32) | cx;
}

// A list box clipped to its cell (cx, cy) of edge 2^l <= 2^BIN_PACK_LEVEL, in coordinates relative
// to the cell's corner: (x0 | x1 << 16, y0 | y1 << 16).  A point of that cell lies in the box
// exactly when its own relative coordinates lie in the clipped one, so the probe's closed-box
// test is unchanged while each list entry it reads takes 8 bytes instead of 16.
__device__ __forceinline__ uint2 pack_box(int4 b, unsigned cx, unsigned cy, int l)
{
    const unsigned ox = cx << l, oy = cy << l, top = (1u << l) - 1u;
    const unsigned bx0 = (unsigned)b.x ^ 0x80000000u, bx1 = (unsigned)b.z ^ 0x80000000u;
    const unsigned by0 = (unsigned)b.y ^ 0x80000000u, by1 = (unsigned)b.w ^ 0x80000000u;
    // the box covers the cell: bx0 <= ox + top and bx1 >= ox (likewise in y)
    const unsigned x0 = bx0 > ox ? bx0 - ox : 0u, x1 = min(bx1 - ox, top);
    const unsigned y0 = by0 > oy ? by0 - oy : 0u, y1 = min(by1 - oy, top);
    return make_uint2(x0 | (x1 << 16), y0 | (y1 << 16));
}

__device__ __forceinline__ unsigned long long hash_slot(unsigned long long key, int hbits)
{
    return (key * 0x9E3779B97F4A7C15ull) >> (64 - hbits);
}

__global__ void k_poly_bbox(const int32_t *__restrict__ po, const int2 *__restrict__ verts, int P, int4 *bb,
                            IndexHeader *h)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    __shared__ unsigned long long s_cells[32], s_big[32];
    if (threadIdx.x < 32) {
        s_cells[threadIdx.x] = 0;
        s_big[threadIdx.x] = 0;
    }
    __syncthreads();
    unsigned long long my_cells = 0, my_big = 0;   // lane l: level l
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
        if (lane == 0) bb[k] = make_int4(x0, y0, x1, y1);
        if (v1 > v0 && lane >= 1) {
            const unsigned long long n = (unsigned long long)(cell_of(x1, lane) - cell_of(x0, lane) + 1) *
                                         (cell_of(y1, lane) - cell_of(y0, lane) + 1);
            if (n <= BIN_CELL_CAP) my_cells += n; else ++my_big;
        }
    }
    if (lane >= 1) {
        if (my_cells) atomicAdd(&s_cells[lane], my_cells);
        if (my_big) atomicAdd(&s_big[lane], my_big);
    }
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x < 32) {
        if (s_cells[threadIdx.x]) atomicAdd(&h->cells[threadIdx.x], s_cells[threadIdx.x]);
        if (s_big[threadIdx.x]) atomicAdd(&h->big[threadIdx.x], s_big[threadIdx.x]);
    }
}

// The finest level at or above the requested one whose pairs fit the list and whose larger boxes
// fit the short list.  Level 31 always qualifies: every box covers at most 2 x 2 cells.
__global__ void k_bin_level(IndexHeader *h, long long lcap)
{
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int l = threadIdx.x;
    const bool ok = l == 31 || (l >= max(1, h->requested_level) && h->cells[l] <= (unsigned long long)lcap &&
                                h->big[l] <= (unsigned long long)BIN_BIG_CAP);
    const unsigned m = __ballot_sync(FULL, ok);
    if (l == 0) h->level = __ffs(m) - 1;
}

// ------------------------------------------------------------------------------------------
// the cell table
// ------------------------------------------------------------------------------------------
// INSERT: claim every covered cell's slot and count the polygon there; else find the slot and
// append the polygon to the cell's list.  Boxes with too many cells go on the short list.
template <bool INSERT>
__global__ void k_cells(const int4 *__restrict__ bb, const int32_t *__restrict__ po, int P, IndexHeader *h,
                        CellEntry *ent, unsigned *cnt, unsigned *off, int4 *list_bb, int *list_id, int *big,
                        int hbits)
{
    const int l = h->level;
    const unsigned long long hmask = (1ull << hbits) - 1;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += (long long)gridDim.x * blockDim.x) {
        if (__ldg(po + k + 1) <= __ldg(po + k)) continue;   // no vertices, no box
        const int4 b = bb[k];
        const unsigned cx0 = cell_of(b.x, l), cx1 = cell_of(b.z, l), cy0 = cell_of(b.y, l), cy1 = cell_of(b.w, l);
        if ((unsigned long long)(cx1 - cx0 + 1) * (cy1 - cy0 + 1) > BIN_CELL_CAP) {
            if (INSERT) {
                const int i = atomicAdd(&h->n_big, 1);
                if (i < BIN_BIG_CAP) big[i] = (int)k;
            }
            continue;
        }
        for (unsigned cy = cy0; cy <= cy1; ++cy)
            for (unsigned cx = cx0; cx <= cx1; ++cx) {
                const unsigned long long key = cell_key(cx, cy);
                unsigned long long s = hash_slot(key, hbits);
                // the table is at most a quarter full, so a free or matching slot is always found
                for (unsigned long long it = 0; it <= hmask; ++it, s = (s + 1) & hmask) {
                    if (INSERT) {
                        const unsigned long long prev = atomicCAS(&ent[s].key, BIN_EMPTY, key);
                        if (prev == BIN_EMPTY || prev == key) {
                            atomicAdd(cnt + s, 1u);
                            break;
                        }
                    } else if (ent[s].key == key) {
                        const unsigned j = atomicAdd(off + s, 1u);
                        if (l <= BIN_PACK_LEVEL) reinterpret_cast<uint2 *>(list_bb)[j] = pack_box(b, cx, cy, l);
                        else list_bb[j] = b;
                        list_id[j] = (int)k;
                        break;
                    }
                }
            }
    }
}

// (first list entry, count) of every occupied slot, after the fill advanced off[] to the list ends
__global__ void k_cells_pack(const unsigned *cnt, const unsigned *off, CellEntry *ent, long long H)
{
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < H; s += (long long)gridDim.x * blockDim.x) {
        const unsigned c = cnt[s];
        if (c) {
            ent[s].start = (int)(off[s] - c);
            ent[s].count = (int)c;
        }
    }
}

// ------------------------------------------------------------------------------------------
// per point: the polygons of its cell and the short list
// ------------------------------------------------------------------------------------------
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_STAGE = 1024;      // pairs a CTA stages in shared memory per pass over 256 points

// The polygons whose closed box holds point i: those of its cell and those of the short list.
template <typename Emit>
__device__ __forceinline__ void probe_point(int2 p, long long i, int l, unsigned long long hmask, int hbits,
                                            const CellEntry *__restrict__ ent, const int4 *__restrict__ list_bb,
                                            const int *__restrict__ list_id, const int *__restrict__ big, int nbig,
                                            const int4 *__restrict__ bb, Emit emit)
{
    const unsigned long long key = cell_key(cell_of(p.x, l), cell_of(p.y, l));
    unsigned long long s = hash_slot(key, hbits);
    for (unsigned long long it = 0; it <= hmask; ++it, s = (s + 1) & hmask) {
        const int4 e = __ldg(reinterpret_cast<const int4 *>(ent + s));   // key, start, count
        const unsigned long long kk = ((unsigned long long)(unsigned)e.y << 32) | (unsigned)e.x;
        if (kk == key) {
            if (l <= BIN_PACK_LEVEL) {   // boxes clipped to the cell, relative to its corner
                const unsigned lm = (1u << l) - 1u;
                const unsigned rx = ((unsigned)p.x ^ 0x80000000u) & lm, ry = ((unsigned)p.y ^ 0x80000000u) & lm;
                const uint2 *__restrict__ lb = reinterpret_cast<const uint2 *>(list_bb);
                const int je = e.z + e.w;
                // four boxes' loads in flight at a time (the loop would otherwise wait for each
                // box before loading the next); a box past the run is empty (x0 > x1)
                for (int j = e.z; j < je; j += 4) {
                    uint2 b[4];
                    #pragma unroll
                    for (int u = 0; u < 4; ++u) b[u] = j + u < je ? __ldg(lb + j + u) : make_uint2(1u, 1u);
                    #pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (rx >= (b[u].x & 0xffffu) && rx <= (b[u].x >> 16) && ry >= (b[u].y & 0xffffu) &&
                            ry <= (b[u].y >> 16))
                            emit(__ldg(list_id + j + u), i);
                }
            } else {
                for (int j = e.z; j < e.z + e.w; ++j) {
                    const int4 b = __ldg(list_bb + j);
                    if (p.x >= b.x && p.x <= b.z && p.y >= b.y && p.y <= b.w) emit(__ldg(list_id + j), i);
                }
            }
            break;
        }
        if (kk == BIN_EMPTY) break;
    }
    for (int j = 0; j < nbig; ++j) {
        const int k = __ldg(big + j);
        const int4 b = __ldg(bb + k);
        if (p.x >= b.x && p.x <= b.z && p.y >= b.y && p.y <= b.w) emit(k, i);
    }
}

// Count pass: per polygon counts (atomics), the total, and every (polygon, point) pair recorded
// for the fill pass -- staged per warp in shared memory and appended with one atomic per flush,
// in any order (the fill's sort fixes the order); pairs past the capacity are dropped and the
// fill pass then probes the points again.  Warps run on their own: no CTA barrier.
__global__ void __launch_bounds__(PROBE_THREADS, 8) k_probe_count(
    const int2 *__restrict__ pts, long long N, const IndexHeader *__restrict__ h, int P, ProbeHeader *q,
    const CellEntry *__restrict__ ent, const int4 *__restrict__ list_bb, const int *__restrict__ list_id,
    const int *__restrict__ big, const int4 *__restrict__ bb, int hbits, unsigned *counts, int2 *pairs,
    long long pcap, long long *d_total)
{
    if (!index_ok(h, P)) return;
    constexpr int WS = PROBE_STAGE / (PROBE_THREADS / 32);   // a warp's stage
    __shared__ int2 s_pair[PROBE_STAGE];
    __shared__ int s_n[PROBE_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int2 *stage = s_pair + w * WS;
    const int l = h->level;
    const int nbig = min(h->n_big, BIN_BIG_CAP);
    const unsigned long long hmask = (1ull << hbits) - 1;
    unsigned long long tot = 0;
    auto emit = [&](int k, long long i) {
        atomicAdd(counts + k, 1u);
        ++tot;
        const int j = atomicAdd(&s_n[w], 1);
        if (j < WS) {
            stage[j] = make_int2(k, (int)i);
        } else {   // the stage is full: straight to the global list
            const unsigned long long g = atomicAdd(&q->n_pairs, 1ull);
            if (g < (unsigned long long)pcap) pairs[g] = make_int2(k, (int)i);
        }
    };
    auto flush = [&]() {
        __syncwarp();
        const int n = min(s_n[w], WS);
        unsigned long long b = 0;
        if (lane == 0 && n) b = atomicAdd(&q->n_pairs, (unsigned long long)n);
        b = __shfl_sync(FULL, b, 0);
        for (int j = lane; j < n; j += 32)
            if (b + j < (unsigned long long)pcap) pairs[b + j] = stage[j];
        __syncwarp();
        if (lane == 0) s_n[w] = 0;
        __syncwarp();
    };
    if (lane == 0) s_n[w] = 0;
    __syncwarp();
    const long long gw = ((long long)blockIdx.x * PROBE_THREADS + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * PROBE_THREADS) >> 5;
    for (long long base = gw * 32; base < N; base += nw * 32) {
        const long long i = base + lane;
        if (i < N) probe_point(__ldg(pts + i), i, l, hmask, hbits, ent, list_bb, list_id, big, nbig, bb, emit);
        __syncwarp();
        if (s_n[w] >= WS / 2) flush();
    }
    flush();
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(FULL, tot, o);
    if (lane == 0 && tot) atomicAdd(reinterpret_cast<unsigned long long *>(d_total), tot);
}

// Fill pass: every id placed at its polygon's offset plus an atomic cursor -- from the pairs the
// count pass recorded, or, when they did not all fit, by probing the points again.
__global__ void __launch_bounds__(PROBE_THREADS, 8) k_probe_fill(
    const int2 *__restrict__ pts, long long N, const IndexHeader *__restrict__ h, int P,
    const ProbeHeader *__restrict__ q, const CellEntry *__restrict__ ent, const int4 *__restrict__ list_bb,
    const int *__restrict__ list_id, const int *__restrict__ big, const int4 *__restrict__ bb, int hbits,
    const int2 *__restrict__ pairs, long long pcap, const int32_t *__restrict__ cand_offsets, unsigned *cursor,
    int32_t *cand_ids, long long capacity)
{
    if (!index_ok(h, P)) return;
    auto place = [&](int k, long long i) {
        const long long pos = (long long)__ldg(cand_offsets + k) + atomicAdd(cursor + k, 1u);
        if (pos < capacity) cand_ids[pos] = (int32_t)i;
    };
    const unsigned long long np = q->n_pairs;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    if (np <= (unsigned long long)pcap) {
        for (long long j = t0; j < (long long)np; j += nt) {
            const int2 q = __ldg(pairs + j);
            place(q.x, q.y);
        }
    } else {
        const int l = h->level;
        const int nbig = min(h->n_big, BIN_BIG_CAP);
        const unsigned long long hmask = (1ull << hbits) - 1;
        for (long long i = t0; i < N; i += nt)
            probe_point(__ldg(pts + i), i, l, hmask, hbits, ent, list_bb, list_id, big, nbig, bb, place);
    }
}

// ------------------------------------------------------------------------------------------
// per polygon: its ids sorted ascending
// ------------------------------------------------------------------------------------------
// 32 K values, value r * 32 + lane in register v[r] of the lane, sorted ascending across the warp
// in the same layout.  Bitonic network whose comparators all put the smaller value at the lower
// position: each stage of block size kk starts by comparing position p with its mirror
// p ^ (kk - 1), then p with p ^ j for j = kk / 4 .. 1.  A partner in another lane comes by a
// shuffle; one in another register of the same lane (j >= 32) is compared in place.
template <int K>
__device__ __forceinline__ void warp_sort_regs(int (&v)[K], int lane)
{
    #pragma unroll
    for (int kk = 2; kk <= 32 * K; kk <<= 1) {
        if (kk <= 32) {
            #pragma unroll
            for (int r = 0; r < K; ++r) {
                const int o = __shfl_xor_sync(FULL, v[r], kk - 1);
                v[r] = (lane & (kk >> 1)) ? max(v[r], o) : min(v[r], o);
            }
        } else {
            // mirror of (r, lane) is (r ^ (kk / 32 - 1), lane ^ 31); the lower one of the pair is
            // the one whose register has bit kk / 64 clear
            int o[K];
            #pragma unroll
            for (int r = 0; r < K; ++r) o[r] = __shfl_xor_sync(FULL, v[r ^ (kk / 32 - 1)], 31);
            #pragma unroll
            for (int r = 0; r < K; ++r) v[r] = (r & (kk / 64)) ? max(v[r], o[r]) : min(v[r], o[r]);
        }
        #pragma unroll
        for (int j = kk >> 2; j > 0; j >>= 1) {
            if (j >= 32) {
                #pragma unroll
                for (int r = 0; r < K; ++r)
                    if (!(r & (j / 32))) {
                        const int x = v[r], y = v[r | (j / 32)];
                        v[r] = min(x, y);
                        v[r | (j / 32)] = max(x, y);
                    }
            } else {
                #pragma unroll
                for (int r = 0; r < K; ++r) {
                    const int o = __shfl_xor_sync(FULL, v[r], j);
                    v[r] = (lane & j) ? max(v[r], o) : min(v[r], o);
                }
            }
        }
    }
}

// A list of n <= 32 K ids at ids[a ..) sorted by one warp in registers.
template <int K>
__device__ __forceinline__ void warp_sort_list(int32_t *ids, long long a, long long n, int lane)
{
    int v[K];
    #pragma unroll
    for (int r = 0; r < K; ++r) v[r] = r * 32 + lane < n ? ids[a + r * 32 + lane] : INT_MAX;
    warp_sort_regs<K>(v, lane);
    #pragma unroll
    for (int r = 0; r < K; ++r)
        if (r * 32 + lane < n) ids[a + r * 32 + lane] = v[r];
}

// V[0..n) sorted ascending by threads t0, t0 + nt, ... of a group that `sync` synchronises: the
// same network over the next power of two, positions n and beyond counting as +infinity (a
// comparator never moves one of them below n, so they are never touched).
// Idx: int for the shared-memory sorts, long long for lists in global memory (up to 2^31 ids).
template <typename Idx, typename Sync>
__device__ void bitonic_sort(int *V, Idx n, int t0, int nt, Sync sync)
{
    Idx P2 = 1;
    while (P2 < n) P2 <<= 1;
    for (Idx kk = 2; kk <= P2; kk <<= 1) {
        for (Idx j = kk >> 1; j > 0; j >>= 1) {
            const int lj = __ffsll((long long)j) - 1;
            for (Idx t = t0; t < (P2 >> 1); t += nt) {
                const Idx blk = t >> lj, r = t & (j - 1);
                const Idx i = (blk << (lj + 1)) + r;
                const Idx q = j == (kk >> 1) ? (blk << (lj + 1)) + kk - 1 - r : i + j;
                if (q < n) {
                    const int x = V[i], y = V[q];
                    if (x > y) {
                        V[i] = y;
                        V[q] = x;
                    }
                }
            }
            sync();
        }
    }
}

// One lane per polygon: lists of up to SORT_LANE ids sorted in the lane's registers; longer ones
// queued, up to SORT_WARP_SMEM ids for k_seg_sort_medium (a warp each), beyond for
// k_seg_sort_long (a CTA each).
__global__ void __launch_bounds__(256) k_seg_sort(const int32_t *__restrict__ cand_offsets, int P, int32_t *ids,
                                                  long long capacity, ProbeHeader *h, int *medium_list,
                                                  int *long_list)
{
    const int lane = threadIdx.x & 31;
    for (long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x - lane; k0 < P;
         k0 += (long long)gridDim.x * blockDim.x) {
        const long long k = k0 + lane;   // k0: the warp's first polygon
        long long a = 0, n = 0;
        if (k < P) {
            a = min((long long)cand_offsets[k], capacity);
            n = min((long long)cand_offsets[k + 1], capacity) - a;
        }
        if (n > 1 && n <= SORT_LANE) {
            int v[SORT_LANE];
            #pragma unroll
            for (int i = 0; i < SORT_LANE; ++i) v[i] = i < n ? ids[a + i] : INT_MAX;
            #pragma unroll
            for (int kk = 2; kk <= SORT_LANE; kk <<= 1) {
                #pragma unroll
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    #pragma unroll
                    for (int i = 0; i < SORT_LANE; ++i) {
                        const int q = j == (kk >> 1) ? (i ^ (kk - 1)) : (i ^ j);
                        if (q > i) {
                            const int x = min(v[i], v[q]), y = max(v[i], v[q]);
                            v[i] = x;
                            v[q] = y;
                        }
                    }
                }
            }
            #pragma unroll
            for (int i = 0; i < SORT_LANE; ++i)
                if (i < n) ids[a + i] = v[i];
        }
        // queue the longer lists, one atomic per warp and queue
        const bool med = n > SORT_LANE && n <= SORT_WARP_SMEM, lng = n > SORT_WARP_SMEM;
        const unsigned mm = __ballot_sync(FULL, med), ml = __ballot_sync(FULL, lng);
        int bm = 0, bl = 0;
        if (lane == 0) {
            if (mm) bm = atomicAdd(&h->n_medium, __popc(mm));
            if (ml) bl = atomicAdd(&h->n_long, __popc(ml));
        }
        bm = __shfl_sync(FULL, bm, 0);
        bl = __shfl_sync(FULL, bl, 0);
        const unsigned below = (1u << lane) - 1u;
        if (med) medium_list[bm + __popc(mm & below)] = (int)k;
        if (lng) long_list[bl + __popc(ml & below)] = (int)k;
    }
}

// The queued lists of up to SORT_WARP_SMEM ids, one warp each: in registers up to
// 32 SORT_WARP_REG ids, else in the warp's shared memory.
__global__ void __launch_bounds__(256) k_seg_sort_medium(const int32_t *__restrict__ cand_offsets, int32_t *ids,
                                                         long long capacity, const ProbeHeader *h,
                                                         const int *medium_list)
{
    __shared__ int s_v[8 * SORT_WARP_SMEM];
    const int lane = threadIdx.x & 31;
    int *wv = s_v + (threadIdx.x >> 5) * SORT_WARP_SMEM;
    const int nm = h->n_medium;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = gw; t < nm; t += nw) {
        const int k = medium_list[t];
        const long long a = min((long long)cand_offsets[k], capacity);
        const long long n = min((long long)cand_offsets[k + 1], capacity) - a;
        if (n <= 32) {
            warp_sort_list<1>(ids, a, n, lane);
        } else if (n <= 64) {
            warp_sort_list<2>(ids, a, n, lane);
        } else if (n <= 32 * SORT_WARP_REG) {
            warp_sort_list<SORT_WARP_REG>(ids, a, n, lane);
        } else {
            for (int i = lane; i < n; i += 32) wv[i] = ids[a + i];
            __syncwarp();
            bitonic_sort<int>(wv, (int)n, lane, 32, [] { __syncwarp(); });
            for (int i = lane; i < n; i += 32) ids[a + i] = wv[i];
            __syncwarp();
        }
    }
}

// The queued longer lists, one CTA per polygon: in shared memory up to SORT_CTA_SMEM ids, else in
// place in global memory.
__global__ void __launch_bounds__(256) k_seg_sort_long(const int32_t *__restrict__ cand_offsets, int32_t *ids,
                                                       long long capacity, const ProbeHeader *h,
                                                       const int *long_list)
{
    __shared__ int s_v[SORT_CTA_SMEM];
    const int tid = threadIdx.x;
    const int nl = h->n_long;
    for (int t = blockIdx.x; t < nl; t += gridDim.x) {
        const int k = long_list[t];
        const long long a = min((long long)cand_offsets[k], capacity);
        const long long n = min((long long)cand_offsets[k + 1], capacity) - a;
        if (n <= SORT_CTA_SMEM) {
            for (int i = tid; i < n; i += 256) s_v[i] = ids[a + i];
            __syncthreads();
            bitonic_sort<int>(s_v, (int)n, tid, 256, [] { __syncthreads(); });
            for (int i = tid; i < n; i += 256) ids[a + i] = s_v[i];
        } else {
            bitonic_sort<long long>(ids + a, n, tid, 256, [] { __syncthreads(); });
        }
        __syncthreads();
    }
}

__global__ void k_bin_finish(ProbeHeader *h, const long long *d_total, long long capacity, int32_t *d_overflow)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (d_total) h->total = *d_total;
        if (d_overflow) *d_overflow = h->total > capacity ? 1 : 0;
    }
}

// ------------------------------------------------------------------------------------------
// host launch sequences
// ------------------------------------------------------------------------------------------
int launch_bin_index(const int32_t *po, const int2 *verts, int P, int cell_size, void *index, size_t index_bytes,
                     int n_sm, cudaStream_t s)
{
    const IndexLayout L = index_layout(P);
    if (index_bytes < L.total) return (int)cudaErrorInvalidValue;
    char *w = static_cast<char *>(index);
    IndexHeader *h = reinterpret_cast<IndexHeader *>(w + L.header);
    int4 *bb = reinterpret_cast<int4 *>(w + L.poly_bb);
    CellEntry *ent = reinterpret_cast<CellEntry *>(w + L.ent);
    unsigned *cnt = reinterpret_cast<unsigned *>(w + L.cnt);
    unsigned *off = reinterpret_cast<unsigned *>(w + L.off);
    int4 *list_bb = reinterpret_cast<int4 *>(w + L.list_bb);
    int *list_id = reinterpret_cast<int *>(w + L.list_id);
    int *big = reinterpret_cast<int *>(w + L.big);
    unsigned *tmp = reinterpret_cast<unsigned *>(w + L.scan_tmp);
    const int grid = n_sm * 8;
    int requested = 0;   // cell edge rounded up to a power of two
    if (cell_size > 0) {
        requested = 1;
        while (requested < 31 && (1LL << requested) < cell_size) ++requested;
    }
    int e;
    k_index_init<<<1, 32, 0, s>>>(h, requested, P);
    note_launch();
    if (P > 0) {
        k_poly_bbox<<<grid, 256, 0, s>>>(po, verts, P, bb, h);
        k_bin_level<<<1, 32, 0, s>>>(h, L.lcap);
        note_launch(2);
        if ((e = (int)cudaMemsetAsync(ent, 0xff, (size_t)L.H * sizeof(CellEntry), s))) return e;
        if ((e = (int)cudaMemsetAsync(cnt, 0, (size_t)L.H * 4, s))) return e;
        k_cells<true><<<grid, 256, 0, s>>>(bb, po, P, h, ent, cnt, off, list_bb, list_id, big, L.hbits);
        note_launch();
        if ((e = (int)cudaMemcpyAsync(off, cnt, (size_t)L.H * 4, cudaMemcpyDeviceToDevice, s))) return e;
        if ((e = scan_exclusive(off, L.H, tmp, s))) return e;
        k_cells<false><<<grid, 256, 0, s>>>(bb, po, P, h, ent, cnt, off, list_bb, list_id, big, L.hbits);
        k_cells_pack<<<grid, 256, 0, s>>>(cnt, off, ent, L.H);
        note_launch(2);
    }
    k_index_finish<<<1, 32, 0, s>>>(h);
    note_launch();
    return (int)cudaGetLastError();
}

int launch_bin_probe_count(const int2 *points, long long N, const void *index, size_t index_bytes, int P,
                           void *probe, size_t probe_bytes, int32_t *cand_offsets, long long *d_total, int n_sm,
                           cudaStream_t s)
{
    const IndexLayout L = index_layout(P);
    const ProbeLayout Q = probe_layout(N, P);
    if (index_bytes < L.total || probe_bytes < Q.total) return (int)cudaErrorInvalidValue;
    const char *w = static_cast<const char *>(index);
    char *pw = static_cast<char *>(probe);
    const IndexHeader *h = reinterpret_cast<const IndexHeader *>(w + L.header);
    ProbeHeader *q = reinterpret_cast<ProbeHeader *>(pw + Q.header);
    int e;
    k_probe_init<<<1, 32, 0, s>>>(q, d_total);
    note_launch();
    if ((e = (int)cudaMemsetAsync(cand_offsets, 0, ((size_t)P + 1) * 4, s))) return e;
    if (P > 0) {
        if (N > 0) {
            k_probe_count<<<n_sm * 8, PROBE_THREADS, 0, s>>>(
                points, N, h, P, q, reinterpret_cast<const CellEntry *>(w + L.ent),
                reinterpret_cast<const int4 *>(w + L.list_bb), reinterpret_cast<const int *>(w + L.list_id),
                reinterpret_cast<const int *>(w + L.big), reinterpret_cast<const int4 *>(w + L.poly_bb), L.hbits,
                reinterpret_cast<unsigned *>(cand_offsets), reinterpret_cast<int2 *>(pw + Q.pairs), Q.pcap, d_total);
            note_launch();
        }
        if ((e = scan_exclusive(reinterpret_cast<unsigned *>(cand_offsets), (long long)P + 1,
                                reinterpret_cast<unsigned *>(pw + Q.scan_tmp), s)))
            return e;
    }
    k_bin_finish<<<1, 32, 0, s>>>(q, d_total, 0, nullptr);
    note_launch();
    return (int)cudaGetLastError();
}

int launch_bin_probe_fill(const int2 *points, long long N, const void *index, size_t index_bytes, int P,
                          void *probe, size_t probe_bytes, const int32_t *cand_offsets, int32_t *cand_ids,
                          long long capacity, int32_t *d_overflow, int n_sm, cudaStream_t s)
{
    const IndexLayout L = index_layout(P);
    const ProbeLayout Q = probe_layout(N, P);
    if (index_bytes < L.total || probe_bytes < Q.total) return (int)cudaErrorInvalidValue;
    const char *w = static_cast<const char *>(index);
    char *pw = static_cast<char *>(probe);
    const IndexHeader *h = reinterpret_cast<const IndexHeader *>(w + L.header);
    ProbeHeader *q = reinterpret_cast<ProbeHeader *>(pw + Q.header);
    unsigned *cursor = reinterpret_cast<unsigned *>(pw + Q.cursor);
    int *medium_list = reinterpret_cast<int *>(pw + Q.medium_list);
    int *long_list = reinterpret_cast<int *>(pw + Q.long_list);
    const int grid = n_sm * 8;
    int e;
    if (P > 0 && N > 0) {
        if ((e = (int)cudaMemsetAsync(cursor, 0, (size_t)P * 4, s))) return e;
        if ((e = (int)cudaMemsetAsync(&q->n_long, 0, 2 * sizeof(int), s))) return e;   // n_long, n_medium
        k_probe_fill<<<grid, PROBE_THREADS, 0, s>>>(
            points, N, h, P, q, reinterpret_cast<const CellEntry *>(w + L.ent),
            reinterpret_cast<const int4 *>(w + L.list_bb), reinterpret_cast<const int *>(w + L.list_id),
            reinterpret_cast<const int *>(w + L.big), reinterpret_cast<const int4 *>(w + L.poly_bb), L.hbits,
            reinterpret_cast<const int2 *>(pw + Q.pairs), Q.pcap, cand_offsets, cursor, cand_ids, capacity);
        k_seg_sort<<<grid, 256, 0, s>>>(cand_offsets, P, cand_ids, capacity, q, medium_list, long_list);
        k_seg_sort_medium<<<grid, 256, 0, s>>>(cand_offsets, cand_ids, capacity, q, medium_list);
        k_seg_sort_long<<<n_sm * 4, 256, 0, s>>>(cand_offsets, cand_ids, capacity, q, long_list);
        note_launch(4);
    }
    k_bin_finish<<<1, 32, 0, s>>>(q, nullptr, capacity, d_overflow);
    note_launch();
    return (int)cudaGetLastError();
}

int launch_bin_count(const int2 *points, long long N, const int32_t *po, const int2 *verts, int P, int cell_size,
                     void *ws, size_t ws_bytes, int32_t *cand_offsets, long long *d_total, int n_sm,
                     cudaStream_t s)
{
    const size_t ib = bin_index_bytes(P), pb = bin_probe_bytes(N, P);
    if (ws_bytes < ib + pb) return (int)cudaErrorInvalidValue;
    int e = launch_bin_index(po, verts, P, cell_size, ws, ib, n_sm, s);
    if (e) return e;
    return launch_bin_probe_count(points, N, ws, ib, P, static_cast<char *>(ws) + ib, pb, cand_offsets, d_total,
                                  n_sm, s);
}

int launch_bin_fill(const int2 *points, long long N, const int32_t *po, const int2 *verts, int P, void *ws,
                    size_t ws_bytes, const int32_t *cand_offsets, int32_t *cand_ids, long long capacity,
                    int32_t *d_overflow, int n_sm, cudaStream_t s)
{
    (void)verts;
    (void)po;
    const size_t ib = bin_index_bytes(P), pb = bin_probe_bytes(N, P);
    if (ws_bytes < ib + pb) return (int)cudaErrorInvalidValue;
    return launch_bin_probe_fill(points, N, ws, ib, P, static_cast<char *>(ws) + ib, pb, cand_offsets, cand_ids,
                                 capacity, d_overflow, n_sm, s);
}

}  // namespace pipdev
