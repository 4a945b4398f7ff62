// Internal launch helpers of libpip (host side; not part of the public C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pipdev {

// Counts kernel launches made by the library (host side; pip_launch_count reads it).
void note_launch(int n = 1);

// Records a CUDA runtime error for pip_last_cuda_error (thread-local) and returns PIP_ERR_CUDA.
int cuda_fail(cudaError_t e);

// Statistics counters that pip_classify_noalloc keeps in its fixed device array (ST_COUNT values
// of the current device): added to `h` (reset to 0 when `reset`), nothing when that entry point
// has not run on this device.  Returns 0 or a CUDA error code.
int noalloc_stats(unsigned long long *h, bool reset);

struct ClassifyArgs;

struct LargeList;

// Tuned shapes of pip_classify's kernels.
struct Tuning {
    int edge_tile;       // large-polygon kernel: edges staged in shared memory per pass
    int pts_per_thread;  // large-polygon kernel: candidates carried by each thread (1, 2, 4)
    int ctas_per_sm;     // large-polygon kernel: resident CTAs per SM
    int verify;          // recheck every trusted decision exactly and count disagreements
    int small_kernel;    // small polygons: 0 = lockstep rounds (k_pip_warp), 1 = compacting (k_pip_cmp),
                         // 2 = thread per polygon (k_pip_tpp)
    int small_slice;     // kernels 0 and 1: candidates per slice (128, 256); kernel 2: slice / 16 per thread
    int small_ctas;      // small-polygon kernel: resident CTAs per SM (0 = as many as fit)
};

int launch_exact(const ClassifyArgs &a, long long total_bits, int grid, cudaStream_t stream, int rule = 0);
int launch_filtered(const ClassifyArgs &a, long long total_bits, const Tuning &t, int n_sm, LargeList *ll,
                    int lcap, cudaStream_t stream);
size_t filtered_smem_bytes(int edge_tile);
int launch_small_cmp(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int slice, int ctas_per_sm,
                     bool verify, cudaStream_t stream);
int launch_small_tpp(const ClassifyArgs &a, LargeList *ll, int lcap, int n_sm, int block, int ctas_per_sm,
                     bool verify, cudaStream_t stream);
Tuning current_tuning();   // the values set by pip_set_tuning
int launch_validate(const ClassifyArgs &a, long long n_verts, long long n_cand_ids, int *d_status, int grid,
                    cudaStream_t stream);

// dst[i] ^= src[i] for i < n (XOR of partial parities)
int launch_xor_words(uint32_t *dst, const uint32_t *src, long long n, int n_sm, cudaStream_t stream);

// exclusive scan of uint32 in place (multi-level); tmp holds scan_tmp_elems(n) values
long long scan_tmp_elems(long long n);
int scan_exclusive(unsigned *d, long long n, unsigned *tmp, cudaStream_t s);

// y-slab edge index
size_t slab_index_bytes(int n_polys, long long n_verts, int edges_per_slab, long long capacity);
int launch_slab_build(const int32_t *poly_offsets, const int2 *verts, int n_polys, long long n_verts,
                      int edges_per_slab, void *index, size_t index_bytes, long long *d_entries, int n_sm,
                      cudaStream_t stream);

// quantisation of float64 lon/lat
int launch_quantize(const double *v, long long n, double scale, int32_t *out, int *status, int n_sm,
                    cudaStream_t stream);

// binning
size_t bin_workspace_bytes(long long n_points, int n_polys);
size_t bin_index_bytes(int n_polys);
size_t bin_probe_bytes(long long n_points, int n_polys);
int launch_bin_index(const int32_t *poly_offsets, const int2 *verts, int n_polys, int cell_size, void *index,
                     size_t index_bytes, int n_sm, cudaStream_t stream);
int launch_bin_probe_count(const int2 *points, long long n_points, const void *index, size_t index_bytes,
                           int n_polys, void *probe, size_t probe_bytes, int32_t *cand_offsets,
                           long long *d_total, int n_sm, cudaStream_t stream);
int launch_bin_probe_fill(const int2 *points, long long n_points, const void *index, size_t index_bytes,
                          int n_polys, void *probe, size_t probe_bytes, const int32_t *cand_offsets,
                          int32_t *cand_ids, long long capacity, int32_t *d_overflow, int n_sm,
                          cudaStream_t stream);
int launch_bin_count(const int2 *points, long long n_points, const int32_t *poly_offsets,
                     const int2 *verts, int n_polys, int cell_size, void *ws, size_t ws_bytes,
                     int32_t *cand_offsets, long long *d_total, int n_sm, cudaStream_t stream);
int launch_bin_fill(const int2 *points, long long n_points, const int32_t *poly_offsets,
                    const int2 *verts, int n_polys, void *ws, size_t ws_bytes,
                    const int32_t *cand_offsets, int32_t *cand_ids, long long capacity,
                    int32_t *d_overflow, int n_sm, cudaStream_t stream);

}  // namespace pipdev
