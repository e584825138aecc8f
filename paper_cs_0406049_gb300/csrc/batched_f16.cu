// batched_f16.cu -- fp16-output batched kernels.
#include "batched.cuh"

namespace sincos_gb300 {

int launch_batched_f16(const sincos_seg *segs, const int64_t *lens, int count, int red, int coef,
                       int64_t *sched, const sincos_plan &plan, const DeviceInfo &dev,
                       cudaStream_t st)
{
    return launch_batched_t<__half>(segs, lens, count, red, coef, sched, plan, dev, st);
}

unsigned take_timeouts_batched_f16() { return take_bulk_wait_timeouts_here(); }
unsigned take_bad_segments_batched_f16() { return take_bad_segments_here(); }

}  // namespace sincos_gb300
