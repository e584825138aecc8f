// forward_bf16.cu -- bf16-output forward kernels.  Each pair is computed in
// binary32 exactly as for binary32 output, then rounded to nearest even.
#include "forward.cuh"

namespace sincos_gb300 {

int launch_forward_bf16(const float *x, void *s, void *c, int64_t n, int red, int coef,
                        const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    return launch_forward_t<__nv_bfloat16>(x, (__nv_bfloat16 *)s, (__nv_bfloat16 *)c, n, red, coef,
                                           false, plan, dev, st);
}

unsigned take_timeouts_forward_bf16() { return take_bulk_wait_timeouts_here(); }

}  // namespace sincos_gb300
