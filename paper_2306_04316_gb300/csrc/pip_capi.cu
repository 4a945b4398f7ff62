// C ABI of libpip (declared in include/pip.h): argument checks, the per-device
// workspace, tuning state, statistics and the opt-in device-side validation.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>

#include "pip.h"
#include "pip_device.cuh"
#include "pip_launch.h"

using namespace pipdev;

namespace {

constexpr int MAX_DEVICES = 64;
constexpr int LARGE_LIST_CAP = 1 << 16;   // polygons per call handed to the large-polygon kernel

struct DeviceState {
    unsigned long long *stats = nullptr;   // ST_COUNT counters
    int n_sm = 0;
    std::map<cudaStream_t, LargeList *> lists;   // one large-polygon list per stream
};

std::mutex g_mu;
DeviceState g_dev[MAX_DEVICES];
std::atomic<int> g_edge_tile{2048};
std::atomic<int> g_ctas{3};
std::atomic<int> g_ppt{4};
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_verify{0};
std::atomic<int> g_small_kernel{0};
std::atomic<int> g_small_slice{256};
std::atomic<int> g_small_ctas{0};
thread_local int g_last_cuda = 0;

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

// Per-device workspace (statistics counters), created on first use outside capture.
int device_state(cudaStream_t stream, DeviceState **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= MAX_DEVICES) return PIP_ERR_WORKSPACE;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState &s = g_dev[dev];
    if (!s.stats) {
        if (capturing(stream)) return PIP_ERR_WORKSPACE;
        int n_sm = 0;
        e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e);
        unsigned long long *p = nullptr;
        e = cudaMalloc(&p, ST_COUNT * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaMemset(p, 0, ST_COUNT * sizeof(unsigned long long));
        if (e != cudaSuccess) { cudaFree(p); return cuda_fail(e); }
        s.n_sm = n_sm;
        s.stats = p;
    }
    *out = &s;
    return PIP_OK;
}

// The large-polygon list of (current device, stream): created zeroed on the first call on
// that stream, which must not be made during stream capture.
int stream_list(DeviceState *ds, cudaStream_t stream, LargeList **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = ds->lists.find(stream);
    if (it != ds->lists.end()) {
        *out = it->second;
        return PIP_OK;
    }
    if (capturing(stream)) return PIP_ERR_WORKSPACE;
    const size_t bytes = sizeof(LargeList) + (size_t)LARGE_LIST_CAP * 2 * sizeof(int);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMemset(p, 0, bytes);
    if (e != cudaSuccess) { cudaFree(p); return cuda_fail(e); }
    ds->lists[stream] = static_cast<LargeList *>(p);
    *out = static_cast<LargeList *>(p);
    return PIP_OK;
}

bool misaligned(const void *p, size_t a) { return p && (reinterpret_cast<uintptr_t>(p) % a) != 0; }

int check_classify(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                   const int32_t *verts, int32_t n_polys, const int32_t *cand_offsets,
                   const int32_t *cand_ids, const void *out)
{
    if (n_points < 0 || n_polys < 0) return PIP_ERR_SIZE;
    if ((cand_offsets == nullptr) != (cand_ids == nullptr)) return PIP_ERR_NULL;
    if (n_polys > 0 && (!poly_offsets || !verts || !out)) return PIP_ERR_NULL;
    if (n_points > 0 && !points) return PIP_ERR_NULL;
    if (misaligned(points, 8) || misaligned(verts, 8)) return PIP_ERR_ALIGN;
    if (misaligned(poly_offsets, 4) || misaligned(cand_offsets, 4) || misaligned(cand_ids, 4) ||
        misaligned(out, 4))
        return PIP_ERR_ALIGN;
    if (n_points > (int64_t)INT_MAX) return PIP_ERR_TOO_LARGE;   // ids are int32
    return PIP_OK;
}

ClassifyArgs make_args(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                       const int32_t *verts, int32_t n_polys, const int32_t *cand_offsets,
                       const int32_t *cand_ids, uint32_t *out_bits, unsigned long long *stats)
{
    ClassifyArgs a;
    a.points = reinterpret_cast<const int2 *>(points);
    a.n_points = n_points;
    a.poly_offsets = poly_offsets;
    a.verts = reinterpret_cast<const int2 *>(verts);
    a.n_polys = n_polys;
    a.cand_offsets = cand_offsets;
    a.cand_ids = cand_ids;
    a.out_bits = out_bits;
    a.words_per_poly = (n_points + 31) / 32;
    a.stats = stats;
    a.slab = nullptr;
    return a;
}

}  // namespace

void pipdev::note_launch(int n) { g_launches.fetch_add((unsigned long long)n); }

int pipdev::cuda_fail(cudaError_t e)
{
    g_last_cuda = (int)e;
    return PIP_ERR_CUDA;
}

namespace pipdev {
Tuning current_tuning()
{
    return Tuning{g_edge_tile.load(),   g_ppt.load(),         g_ctas.load(),      g_verify.load(),
                  g_small_kernel.load(), g_small_slice.load(), g_small_ctas.load()};
}
}  // namespace pipdev

extern "C" {

int pip_classify(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                 const int32_t *verts, int32_t n_polys, const int32_t *cand_offsets,
                 const int32_t *cand_ids, uint32_t *out_bits, void *stream)
{
    return pip_classify_slab(points, n_points, poly_offsets, verts, n_polys, cand_offsets, cand_ids, nullptr,
                             out_bits, stream);
}

int pip_classify_slab(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                      const int32_t *verts, int32_t n_polys, const int32_t *cand_offsets,
                      const int32_t *cand_ids, const void *slab_index, uint32_t *out_bits, void *stream)
{
    int rc = check_classify(points, n_points, poly_offsets, verts, n_polys, cand_offsets, cand_ids, out_bits);
    if (rc != PIP_OK) return rc;
    if (misaligned(slab_index, 256)) return PIP_ERR_ALIGN;
    if (n_polys == 0) return PIP_OK;
    const bool dense = cand_offsets == nullptr;
    const long long total_bits = dense ? (long long)n_polys * 32 * ((n_points + 31) / 32) : 0;
    if (dense && total_bits == 0) return PIP_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    LargeList *ll = nullptr;
    rc = stream_list(ds, s, &ll);
    if (rc != PIP_OK) return rc;
    ClassifyArgs a = make_args(points, n_points, poly_offsets, verts, n_polys, cand_offsets, cand_ids,
                               out_bits, ds->stats);
    a.slab = static_cast<const unsigned char *>(slab_index);
    Tuning t = current_tuning();
    int e = launch_filtered(a, total_bits, t, ds->n_sm, ll, LARGE_LIST_CAP, s);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}

int pip_quantize_lonlat(const double *lonlat, int64_t n_values, double scale, int32_t *out, int32_t *d_status,
                        void *stream)
{
    if (n_values < 0) return PIP_ERR_SIZE;
    if (!(scale > 0.0) || scale != scale) return PIP_ERR_INVALID;
    if (n_values > 0 && (!lonlat || !out)) return PIP_ERR_NULL;
    if (misaligned(lonlat, 8) || misaligned(out, 4) || misaligned(d_status, 4)) return PIP_ERR_ALIGN;
    if (n_values == 0) return PIP_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    int rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    int e = launch_quantize(lonlat, n_values, scale, out, d_status, ds->n_sm, s);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}

size_t pip_slab_index_bytes(int32_t n_polys, int64_t n_verts, int32_t edges_per_slab, int64_t capacity)
{
    if (n_polys < 0 || n_verts < 0 || edges_per_slab < 1 || edges_per_slab > 256 || capacity < 0) return 0;
    return slab_index_bytes(n_polys, n_verts, edges_per_slab, capacity);
}

int pip_slab_build(const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys, int64_t n_verts,
                   int32_t edges_per_slab, void *index, size_t index_bytes, int64_t *d_entries, void *stream)
{
    if (n_polys < 0 || n_verts < 0) return PIP_ERR_SIZE;
    if (edges_per_slab < 1 || edges_per_slab > 256) return PIP_ERR_INVALID;
    if (!index || (n_polys > 0 && (!poly_offsets || !verts))) return PIP_ERR_NULL;
    if (n_verts > (int64_t)INT_MAX) return PIP_ERR_TOO_LARGE;
    if (misaligned(index, 256) || misaligned(verts, 8) || misaligned(poly_offsets, 4) || misaligned(d_entries, 8))
        return PIP_ERR_ALIGN;
    if (index_bytes < slab_index_bytes(n_polys, n_verts, edges_per_slab, 0)) return PIP_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    int rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    int e = launch_slab_build(poly_offsets, reinterpret_cast<const int2 *>(verts), n_polys, n_verts, edges_per_slab,
                              index, index_bytes, reinterpret_cast<long long *>(d_entries), ds->n_sm, s);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}

}  // extern "C"

namespace {
int classify_exact_rule(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                        const int32_t *verts, int32_t n_polys, const int32_t *cand_offsets,
                        const int32_t *cand_ids, uint32_t *out_bits, void *stream, int rule)
{
    int rc = check_classify(points, n_points, poly_offsets, verts, n_polys, cand_offsets, cand_ids, out_bits);
    if (rc != PIP_OK) return rc;
    if (n_polys == 0) return PIP_OK;
    const bool dense = cand_offsets == nullptr;
    const long long total_bits = dense ? (long long)n_polys * 32 * ((n_points + 31) / 32) : 0;
    if (dense && total_bits == 0) return PIP_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    ClassifyArgs a = make_args(points, n_points, poly_offsets, verts, n_polys, cand_offsets, cand_ids,
                               out_bits, rule == 0 ? ds->stats : nullptr);
    long long grid = (long long)ds->n_sm * 8;
    if (dense) grid = std::min(grid, (total_bits / 32 + 7) / 8);
    if (grid < 1) grid = 1;
    int e = launch_exact(a, total_bits, (int)grid, s, rule);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}
}  // namespace

extern "C" {

int pip_classify_exact(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                       const int32_t *verts, int32_t n_polys, const int32_t *cand_offsets,
                       const int32_t *cand_ids, uint32_t *out_bits, void *stream)
{
    return classify_exact_rule(points, n_points, poly_offsets, verts, n_polys, cand_offsets, cand_ids,
                               out_bits, stream, 0);
}

int pip_classify_paper(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                       const int32_t *verts, int32_t n_polys, const int32_t *cand_offsets,
                       const int32_t *cand_ids, int32_t algorithm, uint32_t *out_bits, void *stream)
{
    if (algorithm != 1 && algorithm != 2) return PIP_ERR_INVALID;
    return classify_exact_rule(points, n_points, poly_offsets, verts, n_polys, cand_offsets, cand_ids,
                               out_bits, stream, algorithm);
}

int pip_set_tuning(int32_t edge_tile, int32_t pts_per_thread, int32_t ctas_per_sm)
{
    if (edge_tile != 0 && (edge_tile < 256 || edge_tile > 8192 || edge_tile % 32 != 0)) return PIP_ERR_INVALID;
    if (pts_per_thread != 0 && pts_per_thread != 1 && pts_per_thread != 2 && pts_per_thread != 4)
        return PIP_ERR_INVALID;
    if (ctas_per_sm != 0 && (ctas_per_sm < 1 || ctas_per_sm > 8)) return PIP_ERR_INVALID;
    if (edge_tile) g_edge_tile.store(edge_tile);
    if (pts_per_thread) g_ppt.store(pts_per_thread);
    if (ctas_per_sm) g_ctas.store(ctas_per_sm);
    return PIP_OK;
}

int pip_set_small_tuning(int32_t kernel, int32_t slice, int32_t ctas_per_sm)
{
    if (kernel < -1 || kernel > 2) return PIP_ERR_INVALID;
    if (slice != 0 && slice != 128 && slice != 256) return PIP_ERR_INVALID;
    if (ctas_per_sm < -1 || ctas_per_sm > 16) return PIP_ERR_INVALID;
    if (kernel >= 0) g_small_kernel.store(kernel);
    if (slice) g_small_slice.store(slice);
    if (ctas_per_sm >= 0) g_small_ctas.store(ctas_per_sm);
    return PIP_OK;
}

int pip_get_small_tuning(int32_t *kernel, int32_t *slice, int32_t *ctas_per_sm)
{
    if (!kernel || !slice || !ctas_per_sm) return PIP_ERR_NULL;
    *kernel = g_small_kernel.load();
    *slice = g_small_slice.load();
    *ctas_per_sm = g_small_ctas.load();
    return PIP_OK;
}

int pip_get_tuning(int32_t *edge_tile, int32_t *pts_per_thread, int32_t *ctas_per_sm)
{
    if (!edge_tile || !pts_per_thread || !ctas_per_sm) return PIP_ERR_NULL;
    *edge_tile = g_edge_tile.load();
    *pts_per_thread = g_ppt.load();
    *ctas_per_sm = g_ctas.load();
    return PIP_OK;
}

int pip_get_stats(pip_stats *out)
{
    if (!out) return PIP_ERR_NULL;
    DeviceState *ds = nullptr;
    int rc = device_state(nullptr, &ds);
    if (rc != PIP_OK) return rc;
    unsigned long long h[ST_COUNT];
    cudaError_t e = cudaMemcpy(h, ds->stats, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    const int en = noalloc_stats(h, false);   // pip_classify_noalloc's own counters
    if (en) return cuda_fail((cudaError_t)en);
    out->candidates = h[ST_CANDIDATES];
    out->bbox_rejects = h[ST_BBOX_REJECTS];
    out->fallback_points = h[ST_FALLBACK_POINTS];
    out->exact_candidates = h[ST_EXACT_CANDIDATES];
    out->filter_errors = h[ST_FILTER_ERRORS];
    out->verified_pairs = h[ST_VERIFIED];
    out->wait_timeouts = h[ST_WAIT_TIMEOUTS];
    return PIP_OK;
}

int pip_set_verify(int32_t on)
{
    if (on != 0 && on != 1) return PIP_ERR_INVALID;
    g_verify.store(on);
    return PIP_OK;
}

int pip_reset_stats(void)
{
    DeviceState *ds = nullptr;
    int rc = device_state(nullptr, &ds);
    if (rc != PIP_OK) return rc;
    cudaError_t e = cudaMemset(ds->stats, 0, ST_COUNT * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e);
    unsigned long long h[ST_COUNT] = {0};
    const int en = noalloc_stats(h, true);
    return en == 0 ? PIP_OK : cuda_fail((cudaError_t)en);
}

int pip_validate(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                 const int32_t *verts, int32_t n_polys, int64_t n_verts, const int32_t *cand_offsets,
                 const int32_t *cand_ids, int64_t n_cand_ids, int32_t *d_status, void *stream)
{
    if (!d_status) return PIP_ERR_NULL;
    if (n_verts < 0 || n_cand_ids < 0) return PIP_ERR_SIZE;
    int rc = check_classify(points, n_points, poly_offsets, verts, n_polys, cand_offsets, cand_ids,
                            d_status);
    if (rc != PIP_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (n_polys == 0) return PIP_OK;
    ClassifyArgs a = make_args(points, n_points, poly_offsets, verts, n_polys, cand_offsets, cand_ids,
                               nullptr, nullptr);
    int err = launch_validate(a, n_verts, n_cand_ids, d_status, ds->n_sm * 4, s);
    return err == 0 ? PIP_OK : cuda_fail((cudaError_t)err);
}

size_t pip_bin_workspace_bytes(int64_t n_points, int32_t n_polys)
{
    if (n_points < 0 || n_polys < 0) return 0;
    return bin_workspace_bytes(n_points, n_polys);
}

int pip_bin_count(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                  const int32_t *verts, int32_t n_polys, int32_t cell_size, void *workspace,
                  size_t workspace_bytes, int32_t *cand_offsets, int64_t *d_total, void *stream)
{
    if (n_points < 0 || n_polys < 0 || cell_size < 0) return PIP_ERR_SIZE;
    if (n_points > (int64_t)INT_MAX) return PIP_ERR_TOO_LARGE;
    if (!cand_offsets || !d_total || !workspace) return PIP_ERR_NULL;
    if (n_polys > 0 && (!poly_offsets || !verts)) return PIP_ERR_NULL;
    if (n_points > 0 && !points) return PIP_ERR_NULL;
    if (misaligned(points, 8) || misaligned(verts, 8) || misaligned(workspace, 16) ||
        misaligned(d_total, 8) || misaligned(cand_offsets, 4) || misaligned(poly_offsets, 4))
        return PIP_ERR_ALIGN;
    if (workspace_bytes < bin_workspace_bytes(n_points, n_polys)) return PIP_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    int rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    int e = launch_bin_count(reinterpret_cast<const int2 *>(points), n_points, poly_offsets,
                             reinterpret_cast<const int2 *>(verts), n_polys, cell_size, workspace,
                             workspace_bytes, cand_offsets, reinterpret_cast<long long *>(d_total),
                             ds->n_sm, s);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}

int pip_bin_fill(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                 const int32_t *verts, int32_t n_polys, void *workspace, size_t workspace_bytes,
                 const int32_t *cand_offsets, int32_t *cand_ids, int64_t capacity,
                 int32_t *d_overflow, void *stream)
{
    if (n_points < 0 || n_polys < 0 || capacity < 0) return PIP_ERR_SIZE;
    if (n_points > (int64_t)INT_MAX) return PIP_ERR_TOO_LARGE;
    if (!cand_offsets || !workspace || (capacity > 0 && !cand_ids)) return PIP_ERR_NULL;
    if (n_polys > 0 && (!poly_offsets || !verts)) return PIP_ERR_NULL;
    if (n_points > 0 && !points) return PIP_ERR_NULL;
    if (misaligned(points, 8) || misaligned(verts, 8) || misaligned(workspace, 16) ||
        misaligned(cand_ids, 4) || misaligned(cand_offsets, 4) || misaligned(poly_offsets, 4) ||
        misaligned(d_overflow, 4))
        return PIP_ERR_ALIGN;
    if (workspace_bytes < bin_workspace_bytes(n_points, n_polys)) return PIP_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    int rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    int e = launch_bin_fill(reinterpret_cast<const int2 *>(points), n_points, poly_offsets,
                            reinterpret_cast<const int2 *>(verts), n_polys, workspace, workspace_bytes,
                            cand_offsets, cand_ids, capacity, d_overflow, ds->n_sm, s);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}

size_t pip_bin_index_bytes(int32_t n_polys)
{
    if (n_polys < 0) return 0;
    return bin_index_bytes(n_polys);
}

size_t pip_bin_probe_bytes(int64_t n_points, int32_t n_polys)
{
    if (n_points < 0 || n_polys < 0) return 0;
    return bin_probe_bytes(n_points, n_polys);
}

int pip_bin_index(const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys, int32_t cell_size,
                  void *index, size_t index_bytes, void *stream)
{
    if (n_polys < 0 || cell_size < 0) return PIP_ERR_SIZE;
    if (!index) return PIP_ERR_NULL;
    if (n_polys > 0 && (!poly_offsets || !verts)) return PIP_ERR_NULL;
    if (misaligned(verts, 8) || misaligned(index, 16) || misaligned(poly_offsets, 4)) return PIP_ERR_ALIGN;
    if (index_bytes < bin_index_bytes(n_polys)) return PIP_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    int rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    int e = launch_bin_index(poly_offsets, reinterpret_cast<const int2 *>(verts), n_polys, cell_size, index,
                             index_bytes, ds->n_sm, s);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}

int pip_bin_probe_count(const int32_t *points, int64_t n_points, const void *index, size_t index_bytes,
                        int32_t n_polys, void *probe, size_t probe_bytes, int32_t *cand_offsets,
                        int64_t *d_total, void *stream)
{
    if (n_points < 0 || n_polys < 0) return PIP_ERR_SIZE;
    if (n_points > (int64_t)INT_MAX) return PIP_ERR_TOO_LARGE;
    if (!index || !probe || !cand_offsets || !d_total) return PIP_ERR_NULL;
    if (n_points > 0 && !points) return PIP_ERR_NULL;
    if (misaligned(points, 8) || misaligned(index, 16) || misaligned(probe, 16) || misaligned(d_total, 8) ||
        misaligned(cand_offsets, 4))
        return PIP_ERR_ALIGN;
    if (index_bytes < bin_index_bytes(n_polys) || probe_bytes < bin_probe_bytes(n_points, n_polys))
        return PIP_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    int rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    int e = launch_bin_probe_count(reinterpret_cast<const int2 *>(points), n_points, index, index_bytes, n_polys,
                                   probe, probe_bytes, cand_offsets, reinterpret_cast<long long *>(d_total),
                                   ds->n_sm, s);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}

int pip_bin_probe_fill(const int32_t *points, int64_t n_points, const void *index, size_t index_bytes,
                       int32_t n_polys, void *probe, size_t probe_bytes, const int32_t *cand_offsets,
                       int32_t *cand_ids, int64_t capacity, int32_t *d_overflow, void *stream)
{
    if (n_points < 0 || n_polys < 0 || capacity < 0) return PIP_ERR_SIZE;
    if (n_points > (int64_t)INT_MAX) return PIP_ERR_TOO_LARGE;
    if (!index || !probe || !cand_offsets || (capacity > 0 && !cand_ids)) return PIP_ERR_NULL;
    if (n_points > 0 && !points) return PIP_ERR_NULL;
    if (misaligned(points, 8) || misaligned(index, 16) || misaligned(probe, 16) || misaligned(cand_ids, 4) ||
        misaligned(cand_offsets, 4) || misaligned(d_overflow, 4))
        return PIP_ERR_ALIGN;
    if (index_bytes < bin_index_bytes(n_polys) || probe_bytes < bin_probe_bytes(n_points, n_polys))
        return PIP_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    int rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    int e = launch_bin_probe_fill(reinterpret_cast<const int2 *>(points), n_points, index, index_bytes, n_polys,
                                  probe, probe_bytes, cand_offsets, cand_ids, capacity, d_overflow, ds->n_sm, s);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}

int pip_xor_words(uint32_t *dst, const uint32_t *src, int64_t n_words, void *stream)
{
    if (n_words < 0) return PIP_ERR_SIZE;
    if (n_words > 0 && (!dst || !src)) return PIP_ERR_NULL;
    if (misaligned(dst, 4) || misaligned(src, 4)) return PIP_ERR_ALIGN;
    if (n_words == 0) return PIP_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *ds = nullptr;
    int rc = device_state(s, &ds);
    if (rc != PIP_OK) return rc;
    const int e = launch_xor_words(dst, src, n_words, ds->n_sm, s);
    return e == 0 ? PIP_OK : cuda_fail((cudaError_t)e);
}

const char *pip_status_str(int code)
{
    switch (code) {
        case PIP_OK: return "PIP_OK";
        case PIP_ERR_NULL: return "PIP_ERR_NULL: a required pointer is NULL";
        case PIP_ERR_SIZE: return "PIP_ERR_SIZE: negative size or capacity too small";
        case PIP_ERR_ALIGN: return "PIP_ERR_ALIGN: misaligned pointer";
        case PIP_ERR_TOO_LARGE: return "PIP_ERR_TOO_LARGE: count beyond int32 addressing";
        case PIP_ERR_WORKSPACE: return "PIP_ERR_WORKSPACE: workspace missing or too small";
        case PIP_ERR_CUDA: return "PIP_ERR_CUDA: CUDA runtime error";
        case PIP_ERR_INVALID: return "PIP_ERR_INVALID: invalid value";
        default: return "unknown status";
    }
}

int pip_last_cuda_error(void) { return g_last_cuda; }

int pip_version(void) { return 104; }

uint64_t pip_launch_count(void) { return g_launches.load(); }

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// opt-in device-side validation of the data arrays
// ---------------------------------------------------------------------------------------------
namespace pipdev {

__global__ void k_validate(ClassifyArgs a, long long n_verts, long long n_cand_ids, int *status)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    int bad = 0;
    for (long long k = tid; k < a.n_polys; k += nthr) {
        const int p0 = a.poly_offsets[k], p1 = a.poly_offsets[k + 1];
        if (p0 < 0 || p1 < p0) bad |= 1;
        if (a.cand_offsets) {
            const int c0 = a.cand_offsets[k], c1 = a.cand_offsets[k + 1];
            if (c1 < c0 || c0 < 0) bad |= 2;
        }
    }
    if (tid == 0 && (long long)a.poly_offsets[a.n_polys] > n_verts) bad |= 8;
    if (a.cand_offsets) {
        if (tid == 0 && a.cand_offsets[0] < 0) bad |= 2;
        long long C = a.cand_offsets[a.n_polys];
        if (C > n_cand_ids) {
            if (tid == 0) bad |= 16;
            C = n_cand_ids;
        }
        for (long long c = tid; c < C; c += nthr) {
            const int id = a.cand_ids[c];
            if (id < 0 || (long long)id >= a.n_points) bad |= 4;
        }
    }
    if (bad) atomicOr(status, bad);
}

// dst[i] ^= src[i]: the parity reduction of step 7 across edge partitions (16-byte words where
// both arrays allow it, a grid-stride loop over 32-bit words otherwise)
__global__ void k_xor_words(uint32_t *dst, const uint32_t *src, long long n)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0;
    long long done = 0;
    if (vec) {
        const long long n4 = n / 4;
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        for (long long i = tid; i < n4; i += nthr) {
            uint4 a = d4[i];
            const uint4 b = s4[i];
            a.x ^= b.x; a.y ^= b.y; a.z ^= b.z; a.w ^= b.w;
            d4[i] = a;
        }
        done = n4 * 4;
    }
    for (long long i = done + tid; i < n; i += nthr) dst[i] ^= src[i];
}

int launch_xor_words(uint32_t *dst, const uint32_t *src, long long n, int n_sm, cudaStream_t stream)
{
    const long long blocks = std::min<long long>((long long)n_sm * 4, (n / 4 + 255) / 256 + 1);
    k_xor_words<<<(int)std::max(1LL, blocks), 256, 0, stream>>>(dst, src, n);
    note_launch();
    return (int)cudaGetLastError();
}

int launch_validate(const ClassifyArgs &a, long long n_verts, long long n_cand_ids, int *d_status, int grid,
                    cudaStream_t stream)
{
    k_validate<<<grid, 256, 0, stream>>>(a, n_verts, n_cand_ids, d_status);
    note_launch();
    return (int)cudaGetLastError();
}

}  // namespace pipdev
