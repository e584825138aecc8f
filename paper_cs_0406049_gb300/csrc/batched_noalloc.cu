// batched_noalloc.cu -- the batched forward for callers that must not
// allocate device memory.
//
// sincos_batched keeps its tile-prefix scratch in a buffer the library
// obtains with cudaMalloc the first time a stream needs it.  Some callers
// cannot allow that: a plug-in running inside a host application that owns
// every device allocation, a real-time thread that must never hit the
// implicit device synchronization cudaMalloc/cudaFree can cause, or code that
// runs under a memory budget fixed at start-up.  For them the scratch here is
// a fixed file-scope device array, sized for up to
// SINCOS_NOALLOC_MAX_SEGMENTS arrays; it exists on every GPU that loads the
// library, for as long as the library stays loaded.
//
// Host code must not pass the array's name to a kernel: on the host that name
// is only a stand-in for the device symbol.  The device address is looked up
// once per device with cudaGetSymbolAddress, with that device current, and
// cached.
#include <mutex>

#include "trace.h"
#include "internal.h"

namespace sincos_gb300 {

namespace {

// The batched schedule (tile prefix of up to SINCOS_NOALLOC_MAX_SEGMENTS
// segments, then the per-CTA starts; see batched.cuh).  Only register plans
// (vec_bytes 16 or 32) use it; the ring kernel of bulk plans schedules itself
// and touches no scratch.  Every call writes all the entries it later reads,
// so nothing needs clearing between calls.
__device__ __align__(256) int64_t g_noalloc_prefix[SINCOS_NOALLOC_MAX_SEGMENTS + 1 +
                                                   2 * (kMaxBatchedCtas + 1)];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
int64_t *g_noalloc_ptr[kMaxDevices] = {nullptr};

bool stream_is_capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Device address of g_noalloc_prefix on the current device (looked up on the
// first call for that device).  The lookup may load the library's device
// code onto the GPU, which must not happen inside a stream capture: a first
// call on a capturing stream is refused with SINCOS_ECAPTURE.
int noalloc_scratch(int dev, cudaStream_t st, int64_t **out)
{
    if (dev < 0 || dev >= kMaxDevices) return SINCOS_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        if (stream_is_capturing(st)) return SINCOS_ECAPTURE;
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_prefix);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (no-alloc scratch)");
        g_noalloc_ptr[dev] = (int64_t *)p;
    }
    *out = g_noalloc_ptr[dev];
    return SINCOS_OK;
}

}  // namespace

}  // namespace sincos_gb300

using namespace sincos_gb300;

extern "C" int sincos_batched_noalloc(const sincos_seg *segs, const int64_t *lens, int count,
                                      int out_dtype, int reduction, int coef,
                                      sincos_stream_t stream)
{
    SINCOS_TRACE("sincos_batched_noalloc");
    if (count < 0 || !valid_dtype(out_dtype) || !valid_reduction(reduction) || !valid_coef(coef))
        return SINCOS_EINVAL;
    if (count == 0) return SINCOS_OK;
    if (!segs || !lens) return SINCOS_EINVAL;
    if (!aligned_to(segs, 8) || !aligned_to(lens, 8)) return SINCOS_EINVAL;
    if (count > SINCOS_NOALLOC_MAX_SEGMENTS)
        return fail_with(SINCOS_EUNSUPPORTED,
                         "sincos_batched_noalloc: count exceeds SINCOS_NOALLOC_MAX_SEGMENTS "
                         "(65536 arrays), the size of the library's fixed scratch array");
    const DeviceInfo *dev = nullptr;
    int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    int64_t *prefix = nullptr;
    rc = noalloc_scratch(dev->ordinal, (cudaStream_t)stream, &prefix);
    if (rc != SINCOS_OK) return rc;
    const sincos_plan plan = plan_for(*dev, SINCOS_OP_BATCHED, out_dtype, count);
    return launch_batched(segs, lens, count, out_dtype, reduction, coef, prefix, plan, *dev,
                          (cudaStream_t)stream);
}
