// batched_f32.cu -- binary32-output batched kernels and the dtype dispatch.
#include "batched.cuh"

namespace sincos_gb300 {

int launch_batched_bf16(const sincos_seg *segs, const int64_t *lens, int count, int red, int coef,
                        int64_t *sched, const sincos_plan &plan, const DeviceInfo &dev,
                        cudaStream_t st);
int launch_batched_f16(const sincos_seg *segs, const int64_t *lens, int count, int red, int coef,
                       int64_t *sched, const sincos_plan &plan, const DeviceInfo &dev,
                       cudaStream_t st);

int launch_batched(const sincos_seg *segs, const int64_t *lens, int count, int dtype, int red,
                   int coef, int64_t *sched, const sincos_plan &plan, const DeviceInfo &dev,
                   cudaStream_t st)
{
    if (dtype == SINCOS_F32)
        return launch_batched_t<float>(segs, lens, count, red, coef, sched, plan, dev, st);
    if (dtype == SINCOS_BF16)
        return launch_batched_bf16(segs, lens, count, red, coef, sched, plan, dev, st);
    return launch_batched_f16(segs, lens, count, red, coef, sched, plan, dev, st);
}

unsigned take_timeouts_batched_f32() { return take_bulk_wait_timeouts_here(); }
unsigned take_bad_segments_batched_f32() { return take_bad_segments_here(); }

}  // namespace sincos_gb300
