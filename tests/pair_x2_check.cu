// Test kernel: the packed pair (core_x2.cuh) against the scalar pair
// (core.cuh) on every binary32 input, bit for bit (NaN results compared as
// NaN).  Built by tests/test_gpu_pair_x2.py with the library's own numerics
// flags.  Thread k evaluates the inputs with bit patterns 2k and 2k + 1 as
// one packed pair and as two scalar pairs; it touches no memory but the two
// counters.
#include <cuda_runtime.h>
#include <stdint.h>

#include "core_x2.cuh"

using namespace sincos_gb300;

namespace {

__device__ __forceinline__ bool same(float a, float b)
{
    return (a != a && b != b) || __float_as_uint(a) == __float_as_uint(b);
}

template <int RED, int COEF>
__global__ void k_check(unsigned long long *mismatches, unsigned *first_bad)
{
    const uint64_t npairs = 1ull << 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npairs; k += stride) {
        const float x0 = __uint_as_float((unsigned)(2 * k));
        const float x1 = __uint_as_float((unsigned)(2 * k + 1));
        float s0, c0, s1, c1;
        pair<RED, COEF>(x0, s0, c0);
        pair<RED, COEF>(x1, s1, c1);
        float2 s, c;
        pair_x2<RED, COEF>(make_float2(x0, x1), s, c);
        const bool ok0 = same(s.x, s0) && same(c.x, c0);
        const bool ok1 = same(s.y, s1) && same(c.y, c1);
        if (!ok0 || !ok1) {
            atomicAdd(mismatches, 1ull);
            atomicMin(first_bad, ok0 ? (unsigned)(2 * k + 1) : (unsigned)(2 * k));
        }
    }
}

}  // namespace

// Runs the check for one reduction (0 plain, 1 compensated) and coefficient
// set (0 normalized, 1 dagger); returns 0 and the mismatch count and the
// smallest mismatching bit pattern (0xffffffff if none), or a CUDA error code.
extern "C" int pair_x2_check(int red, int coef, unsigned long long *mismatches_out,
                             unsigned *first_bad_out)
{
    unsigned long long *d_mis = nullptr;
    unsigned *d_first = nullptr;
    cudaError_t e = cudaMalloc((void **)&d_mis, sizeof *d_mis);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_first, sizeof *d_first);
    if (e == cudaSuccess) e = cudaMemset(d_mis, 0, sizeof *d_mis);
    if (e == cudaSuccess) e = cudaMemset(d_first, 0xff, sizeof *d_first);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if (red == 1 && coef == 1)
            k_check<RED_COMPENSATED, COEF_DAGGER><<<sms * 8, 256>>>(d_mis, d_first);
        else if (red == 1)
            k_check<RED_COMPENSATED, COEF_NORMALIZED><<<sms * 8, 256>>>(d_mis, d_first);
        else if (coef == 1)
            k_check<RED_PLAIN, COEF_DAGGER><<<sms * 8, 256>>>(d_mis, d_first);
        else
            k_check<RED_PLAIN, COEF_NORMALIZED><<<sms * 8, 256>>>(d_mis, d_first);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(mismatches_out, d_mis, sizeof *d_mis, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(first_bad_out, d_first, sizeof *d_first, cudaMemcpyDeviceToHost);
    cudaFree(d_mis);
    cudaFree(d_first);
    return (int)e;
}
