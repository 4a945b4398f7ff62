/*
 * pip.h -- C ABI of libpip: GB300 (sm_103a) point-in-polygon classification by the
 * vector-geometric ray-casting method (Schwinger et al., "Point in polygon calculation
 * using vector geometric methods with application to geospatial data").
 *
 * The method (Method section, the seven-step algorithm with Constraint 1): cast the ray
 * d = (1, 0) from the query point p; f(r) = (r - p) . (0, 1) = r_y - p_y; an edge
 * R_i -> R_{i+1} is a candidate crossing when f changes sign along it (steps 2-4); it is
 * counted when p lies on the left of the edge, i.e. when (p - R_i) . n has the counting
 * sign for the edge normal n = (d_y, -d_x) oriented so that n_x >= 0 (Constraint 1,
 * Eq. (normal form of a line)); p is inside when the count is odd (step 7).
 *
 * Boundary rule (fixed, half-open; the paper's text is ambiguous at vertices and edges
 * lying on the ray): a vertex with y_i = p_y counts as lying below the ray, and an edge is
 * counted only when the crossing lies strictly to the right of p.  Every point therefore
 * has exactly one answer: that of p + (eps, delta), 0 < delta << eps, under the even-odd
 * rule.  Points on a bottom or left edge are inside, on a top or right edge outside.
 *
 * Data (all int32, fixed point; the intended unit is 1e-7 degree):
 *   points        device, int32 [n_points][2] interleaved (x, y); 8-byte aligned.
 *   poly_offsets  device, int32 [n_polys + 1], non-decreasing: polygon k owns vertices
 *                 verts[poly_offsets[k] .. poly_offsets[k+1]).  Edges are i -> (i+1) mod m,
 *                 so the closing edge is implicit; a repeated closing vertex R_n = R_0 (the
 *                 paper's convention) is allowed and changes nothing.  m < 3 gives all 0.
 *                 Self-intersecting polygons follow the even-odd rule.
 *   verts         device, int32 [V][2] interleaved (x, y); 8-byte aligned.
 *   cand_offsets, cand_ids
 *                 device CSR of candidate points: polygon k's candidates are
 *                 cand_ids[cand_offsets[k] .. cand_offsets[k+1]) (cand_offsets
 *                 non-decreasing and >= 0, ids in [0, n_points)).  Offsets are absolute
 *                 indices into cand_ids and out_bits, so a call may cover a range of a larger
 *                 CSR (pointers to poly_offsets + p0 and cand_offsets + p0 with n_polys = p1 - p0);
 *                 normally cand_offsets[0] = 0.  Both NULL selects DENSE mode: every point
 *                 against every polygon.
 *   out_bits      device, uint32.  CSR mode: ceil(C / 32) words, C = cand_offsets[n_polys];
 *                 bit c (word c >> 5, bit c & 31, LSB first) = "point cand_ids[c] is inside
 *                 the polygon that owns candidate c".  Dense mode: n_polys * W words,
 *                 W = ceil(n_points / 32); bit k*32*W + j = "point j is inside polygon k".
 *                 Every bit of [cand_offsets[0], C) is written and the bits of the final word
 *                 past C are 0; bits below cand_offsets[0] are left as they are (dense mode:
 *                 every word is written).
 *   stream        a cudaStream_t passed as void* (NULL = the legacy default stream).
 *
 * Ownership and errors: the caller owns every buffer.  Calls are asynchronous on `stream`
 * and never synchronise it; they check host-visible arguments only (NULL, sizes,
 * alignment) and return PIP_OK or a negative PIP_ERR_* code without launching anything.
 * The contents of device arrays (monotone offsets, ids in range) are checked only by
 * pip_validate; the classify kernels never read a point through an id outside
 * [0, n_points) (such a candidate gets bit 0).  The library owns a small per-device workspace (work counters and
 * statistics), created on the first call made outside stream capture; a call made during
 * capture before the workspace exists returns PIP_ERR_WORKSPACE.  Calls on different
 * streams that overlap on the GPU share the statistics counters only.
 */
#ifndef PIP_H
#define PIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIP_OK              0
#define PIP_ERR_NULL       -1   /* a required pointer is NULL (or only one CSR array given) */
#define PIP_ERR_SIZE       -2   /* negative size, or a capacity too small */
#define PIP_ERR_ALIGN      -3   /* points / verts not 8-byte aligned, ids not 4-byte aligned */
#define PIP_ERR_TOO_LARGE  -4   /* a count that int32 offsets or ids cannot address */
#define PIP_ERR_WORKSPACE  -5   /* workspace missing or too small during stream capture */
#define PIP_ERR_CUDA       -6   /* a CUDA runtime call failed (see pip_last_cuda_error) */
#define PIP_ERR_INVALID    -7   /* invalid tuning value */

/* Counters accumulated on the device since the last pip_reset_stats. */
typedef struct pip_stats {
    uint64_t candidates;       /* candidates classified by pip_classify */
    uint64_t bbox_rejects;     /* candidates outside their polygon's bounding box */
    uint64_t fallback_points;  /* candidates re-tested exactly because an FP32 sign was
                                  within the forward-error bound of zero */
    uint64_t exact_candidates; /* candidates classified by pip_classify_exact */
    uint64_t filter_errors;    /* verification mode only (pip_set_verify): straddling pairs whose
                                  trusted fast-path decision (int32 sign, or FP32 sign outside the
                                  error bound) differs from the exact 64/128-bit test; 0 means the
                                  filter was sound on every pair it trusted */
    uint64_t verified_pairs;   /* verification mode only: trusted decisions that were rechecked */
    uint64_t wait_timeouts;    /* large-polygon CTAs whose bounded wait for a bulk copy of edges
                                  gave up (such a CTA stops using its shared tile buffer and decides
                                  its remaining pairs exactly from global memory, so the bits stay
                                  exact, only slower), plus warps of the small-polygon kernel whose
                                  loop guard ended their work early (their bits are then incomplete).
                                  Never expected; 0 in every test */
} pip_stats;

/*
 * pip_classify -- the filtered batched kernels (Method, steps 2-7; Constraint 1).
 * Each polygon is rebased to a local frame at the centre of its bounding box.  When the box
 * is small (width, height < 2^30, width x height < 2^30) every pair test is exact in 32-bit
 * integer arithmetic; when it is below 2^31 on both sides, exact with 64-bit products of
 * 32-bit differences; otherwise the side test (p - R_i) . n runs in FP32 with a proven
 * forward-error bound, and any candidate with a (point, edge) pair whose FP32 value lies
 * within the bound is re-tested exactly with 64/128-bit integers.  The result is exact
 * either way.  Polygons of up to 256 vertices run in one of three small-polygon kernels
 * (pip_set_small_tuning); larger ones (or those with more than 2^18 candidate-edge pairs) in
 * a second kernel that splits their edges across CTAs in tiles, each tile taking the 32-bit
 * test when its own vertices span a box small enough, else the FP32 filter in the tile's
 * frame (two launches on `stream`).  The
 * first call on a stream allocates that stream's work list and must not be captured.
 * Arguments and output layout as described above.  Returns PIP_OK or PIP_ERR_*.
 */
int pip_classify(const int32_t *points, int64_t n_points,
                 const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                 const int32_t *cand_offsets, const int32_t *cand_ids,
                 uint32_t *out_bits, void *stream);

/*
 * pip_classify_exact -- the plain exact kernel (same arguments and output): every
 * (point, edge) pair tests the straddle in int32 and the side of the edge with 64-bit
 * integer products (128-bit when a coordinate difference reaches 2^31).  The reference
 * formulation against which the filtered kernel is compared.
 */
int pip_classify_exact(const int32_t *points, int64_t n_points,
                       const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                       const int32_t *cand_offsets, const int32_t *cand_ids,
                       uint32_t *out_bits, void *stream);

/*
 * pip_classify_paper -- the paper's printed algorithms, evaluated literally, to measure how
 * often their rule for points on the ray or on the boundary differs from the half-open rule of
 * pip_classify (same arguments and output layout, plus `algorithm`):
 *   1  Algorithm 1 (Constraint 1): an edge R_i -> R_{i+1} is a candidate when
 *      f_i f_{i+1} <= 0 with f = y - p_y (horizontal edges on the ray included), the normal
 *      n = (d_y, -d_x) is flipped when n_x < 0, and the edge counts when (p - R_i) . n <= 0;
 *      exact integers.
 *   2  Algorithm 2 (Constraint 2): the same candidates; the edge counts when
 *      x_i + ((p_y - y_i) / d_y) d_x > p_x, evaluated in IEEE float64 with one rounding per
 *      operation (0/0 gives NaN, which never counts).
 * The polygon is R_0 .. R_{m-1} with R_m = R_0 (the paper's convention), as in pip_classify.
 * Both rules agree with pip_classify at points whose y differs from every vertex's y and that
 * lie on no edge; they differ on the boundary and on rays through vertices or along edges.
 * Plain exact kernel; returns PIP_OK, PIP_ERR_INVALID for another `algorithm`, or PIP_ERR_*.
 */
int pip_classify_paper(const int32_t *points, int64_t n_points,
                       const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                       const int32_t *cand_offsets, const int32_t *cand_ids, int32_t algorithm,
                       uint32_t *out_bits, void *stream);

/*
 * y-slab edge index (not in the paper: a step beside the method that changes how many pair
 * tests a point needs, not its answer).  Every polygon with more than 256 vertices gets
 * about m / edges_per_slab slabs of equal height over its y-range (no lower than its mean edge
 * height); each edge is listed in every
 * slab its y-range [min y, max y) meets, or, when it meets more than 8, once in the polygon's
 * list of tall edges.  A point then tests only its slab's edges and the tall list -- exactly
 * the edges that can straddle its ray -- with the exact 64/128-bit side test, so the bits equal
 * pip_classify's while a point of a 100,000-vertex polygon tests tens of edges, not 100,000.
 *
 * pip_slab_index_bytes: size of an index buffer for n_polys polygons with n_verts vertices in
 * all that holds `capacity` (edge, slab) entries (0 on a bad argument).  Typical data needs 1-2
 * entries per vertex of the slabbed polygons; a build reports the exact number.
 *
 * pip_slab_build: builds the index of (poly_offsets, verts) into `index` (device, caller-owned,
 * 256-byte aligned, index_bytes long) on `stream`, and writes the number of entries the
 * polygons need to *d_entries (device int64, may be NULL).  If they exceed the buffer's
 * capacity the index is marked unusable (pip_classify_slab then ignores it and classifies as
 * pip_classify does); rebuild with a larger buffer.  edges_per_slab in 1..256 (8 is a good
 * default).  Returns PIP_OK, PIP_ERR_INVALID, PIP_ERR_WORKSPACE (buffer smaller than its fixed
 * part), or another PIP_ERR_*.
 *
 * pip_classify_slab: pip_classify (same arguments, output and small-polygon kernel) with
 * `slab_index` (device, built by pip_slab_build for the same poly_offsets and verts, or NULL)
 * used for the polygons it covers.
 */
size_t pip_slab_index_bytes(int32_t n_polys, int64_t n_verts, int32_t edges_per_slab, int64_t capacity);
int pip_slab_build(const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys, int64_t n_verts,
                   int32_t edges_per_slab, void *index, size_t index_bytes, int64_t *d_entries,
                   void *stream);
int pip_classify_slab(const int32_t *points, int64_t n_points,
                      const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                      const int32_t *cand_offsets, const int32_t *cand_ids, const void *slab_index,
                      uint32_t *out_bits, void *stream);

/*
 * pip_classify_noalloc -- pip_classify for callers that cannot allocate device memory (the
 * paper has no counterpart).  pip_classify allocates, on its first call on each stream, the
 * device list that hands large polygons to its second kernel (and, once per device, its
 * statistics counters).  Callers that must not trigger cudaMalloc -- applications that
 * manage all device memory through their own allocator or a fixed budget, paths that cannot
 * afford cudaMalloc's implicit synchronisation -- can call
 * this variant instead: same arguments, same bits, same kernels, but the list lives in a
 * fixed array inside the library's device image (512 KiB per device, held until the process
 * exits), so no call allocates.
 *   Limit: n_polys <= PIP_NOALLOC_MAX_POLYS, else PIP_ERR_TOO_LARGE (the array holds one list
 *   entry per polygon of the call).
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *   make that first call before any stream capture that includes this entry point.
 *   Every call shares the one array and clears its header on `stream` first; calls whose
 *   work overlaps on the GPU (different streams, or different host threads) race on it and
 *   must be serialised by the caller.  Its statistics counters live in the same array (they are
 *   not cleared per call); pip_get_stats adds them to pip_classify's, and pip_reset_stats
 *   clears both.
 */
#define PIP_NOALLOC_MAX_POLYS 65536
int pip_classify_noalloc(const int32_t *points, int64_t n_points,
                         const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                         const int32_t *cand_offsets, const int32_t *cand_ids,
                         uint32_t *out_bits, void *stream);

/*
 * pip_quantize_lonlat -- float64 coordinates to the int32 fixed point every other call takes
 * (not in the paper, which computes on float64 lon/lat; the step upstream of the hot path).
 * out[i] = rint(lonlat[i] * scale): the product rounded once in IEEE float64, then rounded to
 * the nearest integer with ties to even.  scale = 1e7 gives 1e-7-degree units.  lonlat and out
 * are device arrays of n_values values (interleaved x, y for points or vertices: n_values = 2 *
 * count).  A value that is NaN, infinite or outside int32 after rounding is written as 0 and
 * ORs a bit into *d_status (device int32, may be NULL; 1 = NaN, 2 = out of range), which the
 * caller zeroes first.  Returns PIP_OK, PIP_ERR_INVALID (scale not positive) or PIP_ERR_*.
 */
int pip_quantize_lonlat(const double *lonlat, int64_t n_values, double scale, int32_t *out,
                        int32_t *d_status, void *stream);

/*
 * Uniform-grid binning (not in the paper; it builds the candidate CSR of a spatial join):
 * candidates of polygon k = every point inside k's CLOSED bounding box, listed by ascending
 * point id, so that repeated calls on the same data give identical arrays.  The polygons, not
 * the points, are binned: a polygon index (their boxes in a hash table of square cells of edge
 * 2^l, l the finest level at which the boxes' cells fit a list of 4 entries per polygon + 1024,
 * boxes of more than 64 cells on a short list of at most 256 that every point tests) is built
 * once and then probed by each batch of points.  cand_offsets is int32: the candidate total
 * must stay below 2^31 (*d_total reports it in int64 regardless).
 *
 * Two-step form (one index, any number of batches, concurrently on several streams when each
 * has its own probe workspace):
 *   pip_bin_index_bytes(n_polys) / pip_bin_index: builds the index (device buffer `index`,
 *     caller-owned, 16-byte aligned) of the polygons; cell_size > 0 asks for cells of at least
 *     that many units (rounded up to a power of two, coarser if the list needs it), 0 = finest.
 *   pip_bin_probe_bytes(n_points, n_polys): size of a batch's probe workspace.
 *   pip_bin_probe_count: writes cand_offsets [n_polys + 1] (device, exclusive prefix sum of
 *     the per-polygon counts) and *d_total (device int64) = the number of candidates, and keeps
 *     the batch's (polygon, point) pairs in the probe workspace (up to n_points / 2 + 1024;
 *     beyond that the fill pass probes the points again).
 *   pip_bin_probe_fill: writes cand_ids (device, capacity `capacity` ids) for the same points,
 *     index and probe workspace.  If the total exceeds `capacity`, ids past the capacity are
 *     dropped and *d_overflow (device int32, may be NULL) is set to 1; otherwise 0.
 * A probe of an index that was not built (or was built for another polygon count) finds no
 * candidates.  n_polys is the indexed polygon count.
 *
 * One-step form: pip_bin_workspace_bytes(n_points, n_polys) = index + one probe workspace;
 * pip_bin_count builds the index and runs the count pass, pip_bin_fill the fill pass, on one
 * workspace (same points and polygons in both calls).
 */
size_t pip_bin_index_bytes(int32_t n_polys);
int pip_bin_index(const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                  int32_t cell_size, void *index, size_t index_bytes, void *stream);
size_t pip_bin_probe_bytes(int64_t n_points, int32_t n_polys);
int pip_bin_probe_count(const int32_t *points, int64_t n_points,
                        const void *index, size_t index_bytes, int32_t n_polys,
                        void *probe, size_t probe_bytes,
                        int32_t *cand_offsets, int64_t *d_total, void *stream);
int pip_bin_probe_fill(const int32_t *points, int64_t n_points,
                       const void *index, size_t index_bytes, int32_t n_polys,
                       void *probe, size_t probe_bytes,
                       const int32_t *cand_offsets, int32_t *cand_ids, int64_t capacity,
                       int32_t *d_overflow, void *stream);
size_t pip_bin_workspace_bytes(int64_t n_points, int32_t n_polys);
int pip_bin_count(const int32_t *points, int64_t n_points,
                  const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                  int32_t cell_size, void *workspace, size_t workspace_bytes,
                  int32_t *cand_offsets, int64_t *d_total, void *stream);
int pip_bin_fill(const int32_t *points, int64_t n_points,
                 const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                 void *workspace, size_t workspace_bytes,
                 const int32_t *cand_offsets, int32_t *cand_ids, int64_t capacity,
                 int32_t *d_overflow, void *stream);

/*
 * Tuning of pip_classify's large-polygon kernel (the autotuner's hook; not in the paper).
 * 0 keeps a value.
 *   edge_tile      edges staged in shared memory per pass (256..8192, a multiple of 32)
 *   pts_per_thread candidates each thread carries through a tile (1, 2, 4)
 *   ctas_per_sm    resident CTAs per SM of its persistent grid (1..8)
 * Applies to later calls on every device; PIP_ERR_INVALID for an out-of-range value.
 */
int pip_set_tuning(int32_t edge_tile, int32_t pts_per_thread, int32_t ctas_per_sm);
int pip_get_tuning(int32_t *edge_tile, int32_t *pts_per_thread, int32_t *ctas_per_sm);

/*
 * Tuning of pip_classify's small-polygon kernel (the autotuner's hook; not in the paper; the
 * bits never depend on it).
 *   kernel       0 (default) = lockstep kernel: every candidate walks its polygon's edges in
 *                rounds of 32 consecutive candidates; 1 = compacting kernel: the candidates of a
 *                slice that lie inside their polygon's box are packed together before the edge
 *                walk, and each slice's loads are issued one slice ahead; 2 = thread-per-polygon
 *                kernel: a thread walks its polygon's edges once for a block of candidates held
 *                in registers (clamped to the polygon's box, which keeps the parity), the
 *                polygons of a CTA sorted by vertex count; -1 keeps the value
 *   slice        candidates per slice (kernels 0 and 1), 128 or 256 (default); kernel 2 takes
 *                slice / 16 candidates per thread (8 or 16); 0 keeps it
 *   ctas_per_sm  resident CTAs per SM of either kernel's persistent grid, 1..16, 0 = as many as
 *                fit (default); -1 keeps it
 * Applies to later calls on every device; PIP_ERR_INVALID for an out-of-range value.
 */
int pip_set_small_tuning(int32_t kernel, int32_t slice, int32_t ctas_per_sm);
int pip_get_small_tuning(int32_t *kernel, int32_t *slice, int32_t *ctas_per_sm);

/* Statistics (device counters of the current device).  pip_get_stats copies them to the
 * host with a synchronous copy: call it after the work of interest has completed. */
int pip_get_stats(pip_stats *out);
int pip_reset_stats(void);

/*
 * pip_validate -- opt-in device-side check of the data arrays of a pip_classify call.
 * n_verts and n_cand_ids are the lengths of the verts and cand_ids allocations (in
 * vertices and ids); the check reads poly_offsets, cand_offsets and at most n_cand_ids ids,
 * never past them.  Writes *d_status (device int32): 0 if valid, else a bit mask:
 *   1  poly_offsets negative or decreasing        2  cand_offsets decreasing or
 *                                                    negative
 *   4  a candidate id outside [0, n_points)       8  poly_offsets[n_polys] > n_verts
 *  16  cand_offsets[n_polys] > n_cand_ids
 * A call that passes makes pip_classify read only inside the given arrays.
 */
int pip_validate(const int32_t *points, int64_t n_points,
                 const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                 int64_t n_verts, const int32_t *cand_offsets, const int32_t *cand_ids,
                 int64_t n_cand_ids, int32_t *d_status, void *stream);

/*
 * pip_set_verify -- verification mode of pip_classify (not in the paper; a test hook for the
 * forward-error bound of the FP32 filter).  With on = 1, later pip_classify calls run copies of
 * the kernels that also recompute, with exact 64/128-bit integers, every straddling pair whose
 * fast-path decision they trust, and count disagreements in pip_stats.filter_errors.  The bits
 * are the same; the kernels are slower.  on = 0 (the default) restores the normal kernels.
 * Returns PIP_OK, or PIP_ERR_INVALID for another value.
 */
int pip_set_verify(int32_t on);

/*
 * pip_xor_words -- dst[i] ^= src[i] for i < n_words (device uint32 arrays, 4-byte aligned), on
 * `stream`.  The parity reduction (step 7) across partitions of a polygon's edges: when a
 * classification is split by edges (each part a chain of the polygon's edges closed through its
 * first vertex, so that the added closing edges cancel in pairs), the inside bit is the XOR of
 * the parts' bits, and multi-GPU callers combine the parts' outputs with this call after an
 * all-gather.  Returns PIP_OK or PIP_ERR_*.
 */
int pip_xor_words(uint32_t *dst, const uint32_t *src, int64_t n_words, void *stream);

/* Human-readable name of a PIP_* status code. */
const char *pip_status_str(int code);

/* The last CUDA runtime error seen by the library on this thread (0 = none). */
int pip_last_cuda_error(void);

/* ABI version (major * 100 + minor). */
int pip_version(void);

/*
 * Number of CUDA kernels the library has enqueued since it was loaded, over all calls,
 * devices and threads (not in the paper; for launch accounting).  A launch recorded into a
 * CUDA graph during stream capture counts once, at capture, not at each replay.
 */
uint64_t pip_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* PIP_H */
