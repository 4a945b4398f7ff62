// pip_classify_noalloc: pip_classify for callers that cannot allocate device memory.
//
// pip_classify keeps the list of polygons that go to its large-polygon kernel in memory the
// library allocates with cudaMalloc on the first call on each stream (and its statistics
// counters on the first call on each device).  Some callers cannot let a library do that:
// applications that own every byte of device memory through their own allocator or a fixed
// budget, and latency-critical paths where the implicit synchronisation of cudaMalloc is not
// acceptable.  This entry point
// classifies with the same kernels but takes that list, and its statistics counters, from a
// fixed array in the library's own device image (below), so it never allocates: no cudaMalloc,
// cudaFree or allocating library routine is called on its path.  The paper has no counterpart; the limit is
// PIP_NOALLOC_MAX_POLYS polygons per call, enough for the list to hold every polygon of the
// call, so it can never overflow.
#include <climits>
#include <mutex>

#include "pip.h"
#include "pip_device.cuh"
#include "pip_launch.h"

using namespace pipdev;

namespace {

// The statistics counters (ST_COUNT values, so that pip_get_stats also reports this entry
// point's work and any timed-out tile wait), then the list header, PIP_NOALLOC_MAX_POLYS entries
// and as many work counters: 64 B + 32 B + 2 * 4 B * 65536 = 512 KiB + 96 B in every device's
// copy of the module, held until the process exits.  Every call shares it.
constexpr int NOALLOC_CAP = PIP_NOALLOC_MAX_POLYS;
constexpr size_t NOALLOC_STATS_BYTES = ST_COUNT * sizeof(unsigned long long);
static __device__ __align__(256) unsigned char
    g_noalloc_scratch[NOALLOC_STATS_BYTES + sizeof(LargeList) + 2 * sizeof(int) * NOALLOC_CAP];

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_scratch_ptr[MAX_DEVICES] = {nullptr};   // device address of the array, per device
int g_noalloc_sm[MAX_DEVICES] = {0};

// Once per device, with that device current: the device address of the array (the host-side
// name is only a stand-in and must never reach a kernel).
int noalloc_setup(unsigned char **scratch, int *n_sm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= MAX_DEVICES) return PIP_ERR_WORKSPACE;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        if (!p) return PIP_ERR_WORKSPACE;
        int sm = 0;
        e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e);
        g_noalloc_sm[dev] = sm;
        g_scratch_ptr[dev] = p;
    }
    *scratch = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    *n_sm = g_noalloc_sm[dev];
    return PIP_OK;
}

bool misaligned(const void *p, size_t a) { return p && (reinterpret_cast<uintptr_t>(p) % a) != 0; }

}  // namespace

extern "C" int pip_classify_noalloc(const int32_t *points, int64_t n_points, const int32_t *poly_offsets,
                                    const int32_t *verts, int32_t n_polys, const int32_t *cand_offsets,
                                    const int32_t *cand_ids, uint32_t *out_bits, void *stream)
{
    if (n_points < 0 || n_polys < 0) return PIP_ERR_SIZE;
    if (n_polys > NOALLOC_CAP) return PIP_ERR_TOO_LARGE;
    if (n_points > (int64_t)INT_MAX) return PIP_ERR_TOO_LARGE;
    if ((cand_offsets == nullptr) != (cand_ids == nullptr)) return PIP_ERR_NULL;
    if (n_polys > 0 && (!poly_offsets || !verts || !out_bits)) return PIP_ERR_NULL;
    if (n_points > 0 && !points) return PIP_ERR_NULL;
    if (misaligned(points, 8) || misaligned(verts, 8) || misaligned(poly_offsets, 4) ||
        misaligned(cand_offsets, 4) || misaligned(cand_ids, 4) || misaligned(out_bits, 4))
        return PIP_ERR_ALIGN;
    if (n_polys == 0) return PIP_OK;
    const bool dense = cand_offsets == nullptr;
    const long long total_bits = dense ? (long long)n_polys * 32 * ((n_points + 31) / 32) : 0;
    if (dense && total_bits == 0) return PIP_OK;
    unsigned char *scratch = nullptr;
    int n_sm = 0;
    int rc = noalloc_setup(&scratch, &n_sm);
    if (rc != PIP_OK) return rc;
    LargeList *ll = reinterpret_cast<LargeList *>(scratch + NOALLOC_STATS_BYTES);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the list must start empty: the array keeps whatever the last call left in it (a call whose
    // kernels never ran to the end would leave entries behind)
    cudaError_t e = cudaMemsetAsync(ll, 0, sizeof(LargeList), s);
    if (e != cudaSuccess) return cuda_fail(e);
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
    a.stats = reinterpret_cast<unsigned long long *>(scratch);   // counters in the same array
    a.slab = nullptr;
    const int err = launch_filtered(a, total_bits, current_tuning(), n_sm, ll, NOALLOC_CAP, s);
    return err == 0 ? PIP_OK : cuda_fail((cudaError_t)err);
}

int pipdev::noalloc_stats(unsigned long long *h, bool reset)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    void *p = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (dev >= 0 && dev < MAX_DEVICES) p = g_scratch_ptr[dev];
    }
    if (!p) return 0;   // pip_classify_noalloc has not run on this device
    unsigned long long v[ST_COUNT];
    e = cudaMemcpy(v, p, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return (int)e;
    for (int i = 0; i < ST_COUNT; ++i) h[i] += v[i];
    if (reset) {
        e = cudaMemset(p, 0, sizeof v);
        if (e != cudaSuccess) return (int)e;
    }
    return 0;
}
