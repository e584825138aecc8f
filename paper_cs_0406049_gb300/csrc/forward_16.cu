// forward_16.cu -- bf16- and fp16-output forward kernels.  Each pair is
// computed in binary32 exactly as for binary32 output and then rounded to
// nearest even (cvt.rn), eight results per 16-byte store.
#include "forward.cuh"

namespace sincos_gb300 {

int launch_forward_16(const float *x, void *s, void *c, int64_t n, int dtype, int red, int coef,
                      const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    if (dtype == SINCOS_BF16)
        return launch_forward_t<__nv_bfloat16>(x, (__nv_bfloat16 *)s, (__nv_bfloat16 *)c, n, red,
                                               coef, false, plan, dev, st);
    return launch_forward_t<__half>(x, (__half *)s, (__half *)c, n, red, coef, false, plan, dev, st);
}

}  // namespace sincos_gb300
