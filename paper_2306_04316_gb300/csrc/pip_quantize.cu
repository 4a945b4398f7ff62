// Quantisation of float64 longitude/latitude to the int32 fixed point the kernels take
// (pip_quantize_lonlat).  Not part of the paper's method, which runs on float64 lon/lat (its
// Simulation section); this is the step upstream of the hot path.  Each coordinate becomes
// rint(v * scale): the product rounded to float64 once, then rounded to the nearest integer with
// ties to even -- a plain IEEE definition, so any IEEE-754 implementation gives the same int32.
// A coordinate that is NaN, infinite, or outside int32 after rounding sets a status bit and is
// written as 0.
#include <cstdint>
#include <cuda_runtime.h>

#include "pip_device.cuh"
#include "pip_launch.h"

namespace pipdev {

__global__ void k_quantize(const double *__restrict__ v, long long n, double scale, int32_t *out, int *status)
{
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double q = rint(__dmul_rn(__ldg(v + i), scale));
        int32_t r = 0;
        if (q != q) bad |= 1;                                        // NaN
        else if (q < -2147483648.0 || q > 2147483647.0) bad |= 2;    // infinite or out of range
        else r = (int32_t)q;
        out[i] = r;
    }
    bad = __reduce_or_sync(FULL, bad);
    if ((threadIdx.x & 31) == 0 && bad && status) atomicOr(status, bad);
}

int launch_quantize(const double *v, long long n, double scale, int32_t *out, int *status, int n_sm,
                    cudaStream_t stream)
{
    const long long need = (n + 255) / 256;
    const int grid = (int)(need < (long long)n_sm * 8 ? (need > 0 ? need : 1) : (long long)n_sm * 8);
    k_quantize<<<grid, 256, 0, stream>>>(v, n, scale, out, status);
    note_launch();
    return (int)cudaGetLastError();
}

}  // namespace pipdev
