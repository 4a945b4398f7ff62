// Device helpers shared by the CUDA kernels of libpip (sm_103a).
//
// Method section, seven-step algorithm with Constraint 1: for a query point p and the
// edge R_i -> R_j (j = i + 1, cyclic) the ray d = (1, 0) from p crosses the edge when
// f(R_i) = y_i - p_y and f(R_j) = y_j - p_y lie on opposite sides of the ray, and the
// crossing lies to the right of p when the side test (p - R_i) . n, with the edge normal
// n = (d_y, -d_x) oriented so that n_x >= 0, is negative.  With det = (x_i - p_x) d_y -
// (y_i - p_y) d_x this is sign(d_y) * det > 0.  Half-open reading: a vertex with
// y = p_y lies below the ray, and a crossing exactly at p does not count.
#pragma once

#include <cstdint>
#include <climits>
#include <cuda_runtime.h>

namespace pipdev {

constexpr unsigned FULL = 0xffffffffu;

// Device-side statistics counters (indices into the workspace array).
enum StatIdx {
    ST_CANDIDATES = 0,
    ST_BBOX_REJECTS = 1,
    ST_FALLBACK_POINTS = 2,
    ST_EXACT_CANDIDATES = 4,
    ST_FILTER_ERRORS = 5,     // verification mode: fast-path decisions that the exact test contradicts
    ST_VERIFIED = 6,          // verification mode: fast-path decisions checked
    ST_WAIT_TIMEOUTS = 7,     // bounded waits (or loop guards) in a kernel that gave up (never expected)
    ST_COUNT = 8
};

// Device-side list of polygons too large for a warp tile, filled by the batched kernel
// and consumed by the large-polygon kernel.  Header followed by `cap` entries and `cap`
// per-entry work counters.  The large-polygon kernel's last CTA resets the header, so the
// list is empty between calls.
struct LargeList {
    int count;     // entries appended
    int cursor;    // first entry whose work items are not all taken
    int done;      // CTAs of the large-polygon kernel that have finished
    int overflow;  // an append found the list full
    int pad[4];
};

__device__ __forceinline__ int *large_entries(LargeList *l) { return reinterpret_cast<int *>(l + 1); }
__device__ __forceinline__ int *large_taken(LargeList *l, int cap) { return reinterpret_cast<int *>(l + 1) + cap; }

// One-dimensional bulk copy global -> shared through the tensor memory accelerator, completed on
// an mbarrier (dst, src and bytes multiples of 16), and the barrier operations it needs.
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *smem_dst, const void *gmem_src, unsigned bytes,
                                              unsigned long long *bar)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(d), "l"(gmem_src), "r"(bytes), "r"(b) : "memory");
}
// Waits for the barrier's phase `parity` to complete, giving up after `limit` polls; returns
// whether it completed.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int limit)
{
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    for (int i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(b), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while the kernel before it on the stream is still running; pdl_wait blocks until that
// kernel has completed and its memory operations are visible (a no-op without the attribute),
// and pdl_trigger lets the next kernel start launching early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// 8- and 4-byte asynchronous global -> shared copies (LDGSTS) and their group fences.
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// y-slab edge index of the large polygons (see pip_slab.cu).  The index is one caller-owned
// device buffer: this header, then per polygon (y0, h, S, 0) (S slabs of height h from y0; S = 0
// for polygons without slabs), the first slab of each polygon, the first entry of each slab, a
// scratch array of per-slab cursors and scan space, and the entries: one (x_i, y_i, x_j, y_j) per
// (edge, slab) whose y-range [min y, max y) meets the slab.  Slab S of a polygon holds its tall
// edges (those meeting more than SLAB_TALL slabs), which every point of the polygon tests.
constexpr int SLAB_MIN_M = 257;     // polygons with more vertices get slabs
constexpr int SLAB_TALL = 8;
struct SlabHeader {
    int valid;                      // 1 when the build completed and every entry fitted
    int n_polys;
    int edges_per_slab;
    int pad0;
    long long n_slabs;              // slab bound used by the layout (tall lists included)
    long long n_entries;            // entries the polygons need
    long long capacity;             // entries the buffer holds
    long long off_geom, off_slab, off_entry, off_cursor, off_scan, off_entries;
};

struct ClassifyArgs {
    const int2 *points;
    long long n_points;
    const int32_t *poly_offsets;
    const int2 *verts;
    int n_polys;
    const int32_t *cand_offsets;   // nullptr => dense mode
    const int32_t *cand_ids;
    uint32_t *out_bits;
    long long words_per_poly;      // dense mode: W = ceil(n_points / 32)
    unsigned long long *stats;     // device counters (may be nullptr)
    const unsigned char *slab;     // y-slab index of the large polygons (may be nullptr)
};

// |v| < 2^31, so that products of two such values fit in 62 bits.
__device__ __forceinline__ bool fits31(long long v)
{
    return (unsigned long long)(v + 0x7fffffffLL) <= 0xfffffffeULL;
}

// Exact side test of a straddling edge (x_i, y_i) -> (x_j, y_j): 1 when the crossing of
// the ray from (px, py) lies strictly to its right.  int64 products when every difference
// is below 2^31 in magnitude, 128-bit products otherwise (full int32 range).
__device__ __forceinline__ int exact_edge_counts(int px, int py, int xi, int yi, int xj, int yj)
{
    long long ax = (long long)xi - px, ay = (long long)yi - py;
    long long dx = (long long)xj - xi, dy = (long long)yj - yi;
    int sgn;
    if (fits31(ax) & fits31(ay) & fits31(dx) & fits31(dy)) {
        long long det = ax * dy - ay * dx;
        sgn = (det > 0) - (det < 0);
    } else {
        __int128 det = (__int128)ax * dy - (__int128)ay * dx;
        sgn = (det > 0) - (det < 0);
    }
    return dy > 0 ? (sgn > 0) : (sgn < 0);
}

// Largest k in [0, n_polys) with co[k] <= c0, found by a warp with 32-way probes
// (log32(n_polys) rounds of one load per lane).  Returns -1 when co[0] > c0.  Every
// lane of the warp must call it with the same arguments.
__device__ __forceinline__ int warp_owner_search(const int32_t *__restrict__ co, int n_polys,
                                                 long long c0, int lane)
{
    if (n_polys <= 0 || (long long)__ldg(co) > c0) return -1;
    int lo = 0, hi = n_polys;
    while (hi - lo > 1) {
        int step = (hi - lo + 31) >> 5;
        long long probe = (long long)lo + (long long)lane * step;
        bool ok = probe < hi && (long long)__ldg(co + probe) <= c0;
        unsigned mask = __ballot_sync(FULL, ok);
        int j = 31 - __clz(mask);          // bit 0 is set: co[lo] <= c0
        lo = lo + j * step;
        hi = min(lo + step, hi);
    }
    return lo;
}

// First index i in [0, n) with a[i] > v (n if none); a non-decreasing.
template <typename T, typename V>
__device__ __forceinline__ int upper_bound_dev(const T *a, int n, V v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((V)a[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

}  // namespace pipdev
