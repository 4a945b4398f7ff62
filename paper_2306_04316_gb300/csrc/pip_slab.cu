// y-slab edge index of large polygons (pip_slab_build; used by pip_classify_slab).
//
// Not part of the paper's method, which tests every edge of the polygon for every point
// (Method section, steps 2-7).  An edge R_i -> R_j can only straddle the ray of a point whose
// p_y lies in [min(y_i, y_j), max(y_i, y_j)) (half-open straddle test), so a point needs only
// the edges whose y-range meets its own y.  Each polygon with more than 256 vertices gets S
// slabs of equal height h covering its y-range from y0 (S about m / edges_per_slab, but h no
// lower than the polygon's mean edge height); every
// edge is listed in each slab its y-range meets, or, when it meets more than SLAB_TALL slabs,
// once in the polygon's tall list (slab S).  A point in slab s tests the edges of slab s and
// the tall list: exactly the set of edges that can straddle its ray, so the parity -- and the
// bit -- is the method's.  The number of pair tests drops from m to about the number of
// boundary crossings of a horizontal line plus edges_per_slab.
//
// Build, all on the device (one warp per polygon; the entry order within a slab is that of the
// atomics and does not matter, the parity being an XOR):
//   1. y-range and slab geometry per polygon; slab counts scanned into slab offsets;
//   2. per edge, the slabs it meets (or the tall list): per-slab counts and the total;
//   3. counts scanned into entry offsets; if the total fits the buffer, the entries are
//      written through per-slab cursors and the index is marked valid.
#include <algorithm>

#include "pip_device.cuh"
#include "pip_launch.h"

namespace pipdev {

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SlabLayout {
    size_t geom, slab, entry, cursor, scan, entries, total;
    long long n_slabs;
};

SlabLayout slab_layout(int P, long long V, int E, long long capacity)
{
    SlabLayout L;
    // slabs of a polygon: at most m / E + 1, plus its tall list
    L.n_slabs = V / std::max(E, 1) + 2LL * P + 1;
    const long long scan_n = std::max<long long>(L.n_slabs + 1, (long long)P + 1);
    size_t o = align256(sizeof(SlabHeader));
    L.geom = o; o += align256((size_t)std::max(P, 1) * 16);
    L.slab = o; o += align256(((size_t)P + 1) * 4);
    L.entry = o; o += align256(((size_t)L.n_slabs + 1) * 4);
    L.cursor = o; o += align256((size_t)L.n_slabs * 4);
    L.scan = o; o += align256((size_t)scan_tmp_elems(scan_n) * 4);
    L.entries = o; o += (size_t)std::max<long long>(capacity, 1) * 16;
    L.total = o;
    return L;
}

__global__ void k_slab_init(SlabHeader *h, int P, int E, long long n_slabs, long long capacity, SlabLayout L)
{
    h->valid = 0;
    h->n_polys = P;
    h->edges_per_slab = E;
    h->pad0 = 0;
    h->n_slabs = n_slabs;
    h->n_entries = 0;
    h->capacity = capacity;
    h->off_geom = (long long)L.geom;
    h->off_slab = (long long)L.slab;
    h->off_entry = (long long)L.entry;
    h->off_cursor = (long long)L.cursor;
    h->off_scan = (long long)L.scan;
    h->off_entries = (long long)L.entries;
}

// Warp per polygon: y-range, slab count S and height h; slab[k] = S + 1 (tall list) or 0.
__global__ void k_slab_geom(const int32_t *__restrict__ po, const int2 *__restrict__ verts, int P, int E,
                            int4 *geom, unsigned *slab)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = warp; k < P; k += nw) {
        const int v0 = __ldg(po + k), v1 = __ldg(po + k + 1), m = v1 - v0;
        int y0 = INT_MAX, y1 = INT_MIN;
        unsigned long long sum_dy = 0;
        for (int i = v0 + lane; i < v1; i += 32) {
            const int y = __ldg(verts + i).y, yn = __ldg(verts + (i + 1 < v1 ? i + 1 : v0)).y;
            y0 = min(y0, y);
            y1 = max(y1, y);
            sum_dy += (unsigned long long)llabs((long long)yn - y);
        }
        y0 = __reduce_min_sync(FULL, y0);
        y1 = __reduce_max_sync(FULL, y1);
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum_dy += __shfl_xor_sync(FULL, sum_dy, o);
        if (lane == 0) {
            int S = 0;
            unsigned long long hh = 1;
            if (m >= SLAB_MIN_M) {
                const long long range = (long long)y1 - y0 + 1;   // 1 .. 2^32
                // about m / E slabs, but none lower than the mean edge height, so that a typical
                // edge meets one or two slabs and few are tall
                const long long mean_dy = std::max<long long>(1, (long long)(sum_dy / (unsigned long long)m));
                S = (int)std::min<long long>({std::max(m / std::max(E, 1), 1), (range + mean_dy - 1) / mean_dy,
                                              1LL << 22});
                S = std::max(S, 1);
                hh = (unsigned long long)((range + S - 1) / S);
                if (hh > 0xffffffffULL) {                          // S = 1 over the full int32 range
                    hh = 0xffffffffULL;
                    S = (int)((range + (long long)hh - 1) / (long long)hh);
                }
            }
            geom[k] = make_int4(y0, (int)(unsigned)hh, S, 0);
            slab[k] = S > 0 ? (unsigned)S + 1u : 0u;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) slab[P] = 0;
}

// Slabs met by the edge (a -> b) of a polygon with geometry g: [s_lo, s_hi], or the tall list.
__device__ __forceinline__ bool edge_slabs(int2 a, int2 b, int4 g, unsigned &s_lo, unsigned &s_hi)
{
    const int ymin = min(a.y, b.y), ymax = max(a.y, b.y);
    if (ymax == ymin) return false;                           // never straddles
    const unsigned h = (unsigned)g.y;
    s_lo = ((unsigned)ymin - (unsigned)g.x) / h;
    s_hi = ((unsigned)(ymax - 1) - (unsigned)g.x) / h;
    return true;
}

// Warp per slabbed polygon, lane per edge.  FILL = false: per-slab counts and the total;
// FILL = true: the entries, through per-slab cursors.
template <bool FILL>
__global__ void k_slab_edges(const int32_t *__restrict__ po, const int2 *__restrict__ verts, int P,
                             SlabHeader *h, const int4 *__restrict__ geom, const unsigned *__restrict__ slab,
                             unsigned *entry, unsigned *cursor, int4 *entries)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    if (FILL && (h->n_entries > h->capacity || h->n_entries >= (1LL << 31))) return;
    unsigned long long total = 0;
    for (long long k = warp; k < P; k += nw) {
        const int4 g = geom[k];
        if (g.z == 0) continue;
        const int v0 = __ldg(po + k), v1 = __ldg(po + k + 1);
        const unsigned base = slab[k];
        for (int i = v0 + lane; i < v1; i += 32) {
            const int2 a = __ldg(verts + i), b = __ldg(verts + (i + 1 < v1 ? i + 1 : v0));
            unsigned s_lo, s_hi;
            if (!edge_slabs(a, b, g, s_lo, s_hi)) continue;
            const bool tall = s_hi - s_lo >= (unsigned)SLAB_TALL;
            if (tall) { s_lo = (unsigned)g.z; s_hi = (unsigned)g.z; }
            for (unsigned s = s_lo; s <= s_hi; ++s) {
                if (FILL) {
                    const unsigned pos = entry[base + s] + atomicAdd(cursor + base + s, 1u);
                    entries[pos] = make_int4(a.x, a.y, b.x, b.y);
                } else {
                    atomicAdd(entry + base + s, 1u);
                }
            }
            total += s_hi - s_lo + 1;
        }
    }
    if (!FILL) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_down_sync(FULL, total, o);
        if (lane == 0 && total) atomicAdd(reinterpret_cast<unsigned long long *>(&h->n_entries), total);
    }
}

__global__ void k_slab_finish(SlabHeader *h)
{
    h->valid = (h->n_entries <= h->capacity && h->n_entries < (1LL << 31)) ? 1 : 0;
}

}  // namespace

size_t slab_index_bytes(int n_polys, long long n_verts, int edges_per_slab, long long capacity)
{
    return slab_layout(n_polys, n_verts, edges_per_slab, capacity).total;
}

int launch_slab_build(const int32_t *po, const int2 *verts, int P, long long V, int E, void *index,
                      size_t index_bytes, long long *d_entries, int n_sm, cudaStream_t s)
{
    // the capacity is what the buffer holds beyond the fixed sections
    const SlabLayout L0 = slab_layout(P, V, E, 0);
    if (index_bytes < L0.entries) return (int)cudaErrorInvalidValue;
    const long long capacity = (long long)((index_bytes - L0.entries) / 16);
    const SlabLayout L = slab_layout(P, V, E, capacity);
    char *w = static_cast<char *>(index);
    SlabHeader *h = reinterpret_cast<SlabHeader *>(w);
    int4 *geom = reinterpret_cast<int4 *>(w + L.geom);
    unsigned *slab = reinterpret_cast<unsigned *>(w + L.slab);
    unsigned *entry = reinterpret_cast<unsigned *>(w + L.entry);
    unsigned *cursor = reinterpret_cast<unsigned *>(w + L.cursor);
    unsigned *scan = reinterpret_cast<unsigned *>(w + L.scan);
    int4 *entries = reinterpret_cast<int4 *>(w + L.entries);
    const int grid = n_sm * 8;
    int e;
    k_slab_init<<<1, 1, 0, s>>>(h, P, E, L.n_slabs, capacity, L);
    note_launch();
    if ((e = (int)cudaMemsetAsync(entry, 0, ((size_t)L.n_slabs + 1) * 4, s))) return e;
    if ((e = (int)cudaMemsetAsync(cursor, 0, (size_t)L.n_slabs * 4, s))) return e;
    if (P > 0) {
        k_slab_geom<<<grid, 256, 0, s>>>(po, verts, P, E, geom, slab);
        note_launch();
        if ((e = scan_exclusive(slab, (long long)P + 1, scan, s))) return e;
        k_slab_edges<false><<<grid, 256, 0, s>>>(po, verts, P, h, geom, slab, entry, cursor, entries);
        note_launch();
        if ((e = scan_exclusive(entry, L.n_slabs + 1, scan, s))) return e;
        k_slab_edges<true><<<grid, 256, 0, s>>>(po, verts, P, h, geom, slab, entry, cursor, entries);
        note_launch();
    }
    k_slab_finish<<<1, 1, 0, s>>>(h);
    note_launch();
    if (d_entries) {
        if ((e = (int)cudaMemcpyAsync(d_entries, &h->n_entries, sizeof(long long), cudaMemcpyDeviceToDevice, s)))
            return e;
    }
    return (int)cudaGetLastError();
}

}  // namespace pipdev
