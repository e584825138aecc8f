// cuda_libm.cu -- CUDA's own sincosf and __sincosf in the same streaming
// layout as the library's forward kernel, used only as a context figure by
// the benchmark (speed and error of the vendor functions on the same GPU).
// The functions are called, not reimplemented.  Built with nvcc's default
// floating-point flags, as ordinary user code would be.
#include <cuda_runtime.h>
#include <stdint.h>

template <bool FAST>
__global__ void k_libm(const float4 *x, float4 *s, float4 *c, int64_t nvec)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
        const float4 a = x[v];
        float4 sv, cv;
        if (FAST) {
            __sincosf(a.x, &sv.x, &cv.x);
            __sincosf(a.y, &sv.y, &cv.y);
            __sincosf(a.z, &sv.z, &cv.z);
            __sincosf(a.w, &sv.w, &cv.w);
        } else {
            sincosf(a.x, &sv.x, &cv.x);
            sincosf(a.y, &sv.y, &cv.y);
            sincosf(a.z, &sv.z, &cv.z);
            sincosf(a.w, &sv.w, &cv.w);
        }
        s[v] = sv;
        c[v] = cv;
    }
}

// x, s, c: device, 16-byte aligned, n a multiple of 4.  fast = 0: sincosf,
// fast = 1: __sincosf.  Returns the cudaError_t of the launch.
extern "C" int context_libm_sincos(const float *x, float *s, float *c, int64_t n, int fast,
                                   cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nvec = n / 4;
    int64_t grid = (int64_t)sms * 8;
    const int64_t need = (nvec + 255) / 256;
    if (need < grid) grid = need > 0 ? need : 1;
    if (fast)
        k_libm<true><<<(unsigned)grid, 256, 0, stream>>>((const float4 *)x, (float4 *)s,
                                                          (float4 *)c, nvec);
    else
        k_libm<false><<<(unsigned)grid, 256, 0, stream>>>((const float4 *)x, (float4 *)s,
                                                           (float4 *)c, nvec);
    return (int)cudaGetLastError();
}
