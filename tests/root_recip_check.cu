// Test kernel: the Huygens term's r = sqrt(a) and w = 1/r (core_rt.cuh,
// scalar and packed forms) against the correctly rounded operations
// __fsqrt_rn(a) and __frcp_rn(__fsqrt_rn(a)) on every binary32 bit pattern,
// bit for bit (NaN results compared as NaN).  Built by
// tests/test_gpu_root_recip.py with the library's own numerics flags.  Thread
// k takes the patterns 2k and 2k + 1, as two scalar evaluations and as one
// packed pair; it touches no memory but the counters.
#include <cuda_runtime.h>
#include <stdint.h>

#include "core_rt.cuh"

using namespace sincos_gb300;

namespace {

__device__ __forceinline__ bool same(float a, float b)
{
    return (a != a && b != b) || __float_as_uint(a) == __float_as_uint(b);
}

// counters: [0] scalar mismatches, [1] packed mismatches, [2] first bad
// pattern (scalar), [3] first bad pattern (packed)
__global__ void k_check(unsigned long long *mis, unsigned *first)
{
    const uint64_t npairs = 1ull << 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long ms = 0, mp = 0;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npairs; k += stride) {
        const unsigned b0 = (unsigned)(2 * k), b1 = b0 + 1;
        const float a0 = __uint_as_float(b0), a1 = __uint_as_float(b1);
        const float r0 = __fsqrt_rn(a0), r1 = __fsqrt_rn(a1);
        const float w0 = __frcp_rn(r0), w1 = __frcp_rn(r1);
        float sr0, sw0, sr1, sw1;
        root_recip(a0, sr0, sw0);
        root_recip(a1, sr1, sw1);
        float2 pr, pw;
        root_recip_x2(make_float2(a0, a1), pr, pw);
        const bool s0 = same(sr0, r0) && same(sw0, w0), s1 = same(sr1, r1) && same(sw1, w1);
        const bool p0 = same(pr.x, r0) && same(pw.x, w0), p1 = same(pr.y, r1) && same(pw.y, w1);
        if (!s0 || !s1) {
            ms += (!s0) + (!s1);
            atomicMin(&first[0], s0 ? b1 : b0);
        }
        if (!p0 || !p1) {
            mp += (!p0) + (!p1);
            atomicMin(&first[1], p0 ? b1 : b0);
        }
    }
    if (ms) atomicAdd(&mis[0], ms);
    if (mp) atomicAdd(&mis[1], mp);
}

}  // namespace

// Runs the check; returns 0 (or a CUDA error code) and writes the scalar and
// packed mismatch counts and their smallest mismatching patterns
// (0xffffffff if none).
extern "C" int root_recip_check(unsigned long long *mis_out, unsigned *first_out)
{
    unsigned long long *d_mis = nullptr;
    unsigned *d_first = nullptr;
    cudaError_t e = cudaMalloc((void **)&d_mis, 2 * sizeof *d_mis);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_first, 2 * sizeof *d_first);
    if (e == cudaSuccess) e = cudaMemset(d_mis, 0, 2 * sizeof *d_mis);
    if (e == cudaSuccess) e = cudaMemset(d_first, 0xff, 2 * sizeof *d_first);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        k_check<<<sms * 8, 256>>>(d_mis, d_first);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(mis_out, d_mis, 2 * sizeof *d_mis, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(first_out, d_first, 2 * sizeof *d_first, cudaMemcpyDeviceToHost);
    cudaFree(d_mis);
    cudaFree(d_first);
    return (int)e;
}
