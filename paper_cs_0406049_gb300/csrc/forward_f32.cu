// forward_f32.cu -- binary32-output forward kernels and the dtype dispatch.
#include "forward.cuh"

namespace sincos_gb300 {

int launch_forward_bf16(const float *x, void *s, void *c, int64_t n, int red, int coef,
                        const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st);
int launch_forward_f16(const float *x, void *s, void *c, int64_t n, int red, int coef,
                       const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st);

int launch_forward(const float *x, void *s, void *c, int64_t n, int dtype, int red, int coef,
                   bool in_place, const sincos_plan &plan, const DeviceInfo &dev,
                   cudaStream_t st)
{
    if (dtype == SINCOS_F32)
        return launch_forward_t<float>(x, (float *)s, (float *)c, n, red, coef, in_place, plan, dev,
                                       st);
    if (dtype == SINCOS_BF16) return launch_forward_bf16(x, s, c, n, red, coef, plan, dev, st);
    return launch_forward_f16(x, s, c, n, red, coef, plan, dev, st);
}

unsigned take_timeouts_forward_f32() { return take_bulk_wait_timeouts_here(); }

}  // namespace sincos_gb300
