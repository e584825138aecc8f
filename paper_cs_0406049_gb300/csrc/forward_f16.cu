// forward_f16.cu -- fp16-output forward kernels.  Each pair is computed in
// binary32 exactly as for binary32 output, then rounded to nearest even.
#include "forward.cuh"

namespace sincos_gb300 {

int launch_forward_f16(const float *x, void *s, void *c, int64_t n, int red, int coef,
                       const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    return launch_forward_t<__half>(x, (__half *)s, (__half *)c, n, red, coef, false, plan, dev,
                                    st);
}

unsigned take_timeouts_forward_f16() { return take_bulk_wait_timeouts_here(); }

}  // namespace sincos_gb300
