// api.cu -- C ABI entry points for the single-array forward and backward,
// argument validation, device facts, error reporting and launch counting.
#include <atomic>
#include <mutex>
#include <string>
#include <map>
#include <tuple>

#include "bulk.cuh"
#include "seg_check.h"
#include "trace.h"
#include "internal.h"

namespace sincos_gb300 {

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

constexpr int kMaxDevices = 64;
std::mutex g_dev_mu;
DeviceInfo g_devices[kMaxDevices];
bool g_dev_ready[kMaxDevices] = {false};

// Resident CTAs per SM of a kernel at a block size on a device, with no
// dynamic shared memory (kind 0) or with the bulk kernels' fixed amount
// (kind 1).
using OccKey = std::tuple<const void *, int, int, int>;   // kernel, block, device, kind
std::mutex g_occ_mu;
std::map<OccKey, int> g_occ;

}  // namespace

int cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return SINCOS_ECUDA;
}

int fail_with(int status, const char *what)
{
    g_last_error = what;
    return status;
}

void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int check_launch(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    count_launches(1);
    return SINCOS_OK;
}

int current_device(const DeviceInfo **info)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return SINCOS_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_dev_mu);
    DeviceInfo &d = g_devices[dev];
    if (!g_dev_ready[dev]) {
        cudaDeviceProp prop;
        e = cudaGetDeviceProperties(&prop, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
        d.ordinal = dev;
        d.sms = prop.multiProcessorCount;
        d.major = prop.major;
        d.minor = prop.minor;
        d.max_threads_per_sm = prop.maxThreadsPerMultiProcessor;
        int pageable = 0;
        if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
            cudaGetLastError();
            pageable = 0;
        }
        d.pageable_access = pageable == 1;
        snprintf(d.name, sizeof d.name, "%s", prop.name);
        g_dev_ready[dev] = true;
    }
    // The library carries sm_103a code only.
    if (d.major != 10 || d.minor != 3) {
        g_last_error = std::string("device ") + d.name + " is sm_" + std::to_string(d.major) +
                       std::to_string(d.minor) + "; this library is built for sm_103a only";
        return SINCOS_EUNSUPPORTED;
    }
    *info = &d;
    return SINCOS_OK;
}

int resident_ctas(const void *kernel, int block, int want)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const OccKey key(kernel, block, dev, 0);
    int per_sm = -1;
    {
        std::lock_guard<std::mutex> lock(g_occ_mu);
        auto it = g_occ.find(key);
        if (it != g_occ.end()) per_sm = it->second;
    }
    if (per_sm < 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
        }
        std::lock_guard<std::mutex> lock(g_occ_mu);
        g_occ[key] = per_sm;
    }
    return per_sm < want ? per_sm : want;
}

int bulk_resident_ctas(const void *kernel, int block, size_t smem)
{
    int dev = 0;
    cudaGetDevice(&dev);
    // The calling thread's last answer first (repeated calls of one kind).
    thread_local const void *last_kernel = nullptr;
    thread_local int last_block = -1, last_dev = -1, last_ctas = 0;
    thread_local size_t last_smem = 0;
    if (kernel == last_kernel && block == last_block && dev == last_dev && smem == last_smem)
        return last_ctas;
    const OccKey key(kernel, block, dev, 1);
    {
        std::lock_guard<std::mutex> lock(g_occ_mu);
        auto it = g_occ.find(key);
        if (it != g_occ.end()) {
            last_kernel = kernel;
            last_block = block;
            last_dev = dev;
            last_smem = smem;
            last_ctas = it->second;
            return it->second;
        }
    }
    int per_sm = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    std::lock_guard<std::mutex> lock(g_occ_mu);
    g_occ[key] = per_sm;
    return per_sm;
}

sincos_plan fit_plan(const void *kernel, const sincos_plan &plan, int *per_sm)
{
    sincos_plan p = plan;
    *per_sm = resident_ctas(kernel, p.block, p.ctas_per_sm);
    while (*per_sm <= 0 && p.block > 32) {
        p.block = (p.block / 2 + 31) / 32 * 32;
        *per_sm = resident_ctas(kernel, p.block, p.ctas_per_sm);
    }
    return p;
}

// One CTA waits on an mbarrier that nothing ever arrives on, with the given
// time limit, exactly as the bulk kernels wait on their stages; the wait gives
// up and counts a timeout.  Exercises the timeout path without a fault.
__global__ void k_selftest_wait(unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(smem_addr(&bar), 0u, limit_ns))
        atomicAdd(&g_bulk_wait_timeouts, 1u);
}

bool valid_dtype(int d) { return d == SINCOS_F32 || d == SINCOS_BF16 || d == SINCOS_F16; }
bool valid_reduction(int r) { return r == SINCOS_RED_PLAIN || r == SINCOS_RED_COMPENSATED; }
bool valid_coef(int c) { return c == SINCOS_COEF_NORMALIZED || c == SINCOS_COEF_DAGGER; }

}  // namespace sincos_gb300

using namespace sincos_gb300;

extern "C" {

int sincos_pairs_ex(const float *x, void *s, void *c, int64_t n, int out_dtype, int reduction,
                    int coef, sincos_stream_t stream)
{
    SINCOS_TRACE("sincos_pairs_ex");
    if (n < 0 || !valid_dtype(out_dtype) || !valid_reduction(reduction) || !valid_coef(coef))
        return SINCOS_EINVAL;
    if (n == 0) return SINCOS_OK;
    if (!x || !s || !c) return SINCOS_EINVAL;
    const size_t osz = (size_t)dtype_size(out_dtype);
    if (!aligned_to(x, 4) || !aligned_to(s, osz) || !aligned_to(c, osz)) return SINCOS_EINVAL;
    const size_t xb = (size_t)n * 4, ob = (size_t)n * osz;
    if (ranges_overlap(s, ob, c, ob)) return SINCOS_EOVERLAP;
    bool in_place = false;
    for (const void *o : {(const void *)s, (const void *)c}) {
        if (!ranges_overlap(x, xb, o, ob)) continue;
        if (o == (const void *)x && out_dtype == SINCOS_F32) in_place = true;
        else return SINCOS_EOVERLAP;
    }
    const DeviceInfo *dev = nullptr;
    int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    const sincos_plan plan = plan_for(*dev, SINCOS_OP_PAIRS, out_dtype, n);
    return launch_forward(x, s, c, n, out_dtype, reduction, coef, in_place, plan, *dev,
                          (cudaStream_t)stream);
}

int sincos_pairs(const float *x, float *s, float *c, int64_t n, sincos_stream_t stream)
{
    return sincos_pairs_ex(x, s, c, n, SINCOS_F32, SINCOS_RED_PLAIN, SINCOS_COEF_NORMALIZED, stream);
}

int sincos_backward(const float *gs, const float *gc, const float *s, const float *c, float *gx,
                    int64_t n, sincos_stream_t stream)
{
    SINCOS_TRACE("sincos_backward");
    if (n < 0) return SINCOS_EINVAL;
    if (n == 0) return SINCOS_OK;
    if (!gx || ((gs || gc) && (!s || !c))) return SINCOS_EINVAL;
    if (!all_float_aligned({gs, gc, s, c, gx})) return SINCOS_EINVAL;
    const size_t b = (size_t)n * 4;
    bool in_place = false;
    for (const float *in : {gs, gc, gs ? c : nullptr, gc ? s : nullptr}) {
        if (!in || !ranges_overlap(in, b, gx, b)) continue;
        if (in == gx) in_place = true;
        else return SINCOS_EOVERLAP;
    }
    const DeviceInfo *dev = nullptr;
    int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    const sincos_plan plan = plan_for(*dev, SINCOS_OP_BACKWARD, SINCOS_F32, n);
    return launch_backward(gs, gc, s, c, gx, n, in_place, plan, *dev, (cudaStream_t)stream);
}

const char *sincos_strerror(int status)
{
    switch (status) {
    case SINCOS_OK: return "ok";
    case SINCOS_EINVAL: return "invalid argument";
    case SINCOS_EOVERLAP: return "input and output arrays overlap in a way that is not allowed";
    case SINCOS_ECUDA: return "a CUDA runtime call failed (see sincos_last_error)";
    case SINCOS_EUNSUPPORTED: return "unsupported device or configuration";
    case SINCOS_ECAPTURE:
        return "the call would allocate or do first-use set-up while its stream is being captured";
    default: return "unknown status";
    }
}

const char *sincos_last_error(void) { return g_last_error.c_str(); }

uint32_t sincos_device_wait_timeouts(void)
{
    return take_timeouts_forward_f32() + take_timeouts_forward_bf16() + take_timeouts_forward_f16() +
           take_timeouts_batched_f32() + take_timeouts_batched_bf16() + take_timeouts_batched_f16() +
           take_timeouts_expi() + take_bulk_wait_timeouts_here();
}

uint32_t sincos_device_bad_segments(void)
{
    return take_bad_segments_batched_f32() + take_bad_segments_batched_bf16() +
           take_bad_segments_batched_f16();
}

int sincos_seg_check(const sincos_seg *seg, int64_t len, int out_dtype)
{
    if (!seg || !valid_dtype(out_dtype)) return SINCOS_EINVAL;
    return seg_usable(seg->x, seg->s, seg->c, len, (unsigned)dtype_size(out_dtype))
               ? SINCOS_OK : SINCOS_EINVAL;
}

int sincos_selftest_wait_timeout(uint32_t limit_us, sincos_stream_t stream)
{
    if (limit_us == 0 || limit_us > 1000000u) return SINCOS_EINVAL;
    const DeviceInfo *dev = nullptr;
    const int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    k_selftest_wait<<<1, 32, 0, (cudaStream_t)stream>>>(1000ull * limit_us);
    return check_launch("wait self-test launch");
}

uint64_t sincos_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int sincos_version(void) { return 10000; }

}  // extern "C"
