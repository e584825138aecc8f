// host_path.cu -- the forward on host arrays.
//
// Host buffers the kernel can reach are read and written by the kernel itself
// across the host link (zero-copy), with the register path's plain vector
// loads and stores: page-locked, mapped buffers (cudaHostAlloc,
// cudaMallocHost, or cudaHostRegister with mapping) on any device, and
// ordinary pageable memory on devices that access it through the host's page
// tables (cudaDevAttrPageableMemoryAccess, as GB300 with Grace over
// NVLink-C2C).  There that moves 272 GB/s for either kind of memory, against
// 262 for the copy pipeline with page-locked buffers (it loses its fill and
// drain) and 28 for the pipeline with pageable ones (the driver stages those
// copies).  Otherwise, or when the caller asks for it
// (sincos_host_route_set), the buffers go through the pipeline: chunked host
// -> device copy, kernel, device -> host copy, with consecutive chunks on
// three rotating internal streams, so that one chunk's upload, another's
// kernel and a third's download proceed at once.  The device side of the
// pipeline uses only the caller's workspace.
#include <atomic>
#include <mutex>

#include "trace.h"
#include "internal.h"

namespace sincos_gb300 {

namespace {

constexpr int kSlots = 3;
constexpr int kMaxDevices = 64;

// The route the calling thread's last sincos_pairs_host call took.
thread_local int g_last_path = SINCOS_HOST_PATH_NONE;
// The process-wide route policy (sincos_host_route_set).
std::atomic<int> g_route_policy{SINCOS_HOST_ROUTE_AUTO};

struct Pipe {
    bool ready = false;
    cudaStream_t st[kSlots] = {nullptr, nullptr, nullptr};
    cudaEvent_t done[kSlots] = {nullptr, nullptr, nullptr};
    cudaEvent_t start = nullptr;
    std::mutex mu;   // one enqueue sequence at a time per device
};

std::mutex g_pipe_mu;
Pipe g_pipes[kMaxDevices];

int get_pipe(int dev, Pipe **out)
{
    std::lock_guard<std::mutex> lock(g_pipe_mu);
    Pipe &p = g_pipes[dev];
    if (!p.ready) {
        cudaError_t e = cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming);
        for (int k = 0; e == cudaSuccess && k < kSlots; ++k) {
            e = cudaStreamCreateWithFlags(&p.st[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.done[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "host path stream/event creation");
        p.ready = true;
    }
    *out = &p;
    return SINCOS_OK;
}

// Device address of a host buffer the GPU can access directly: its mapped
// address if it is page-locked and mapped, the host address itself if it is
// pageable memory and the device reads pageable memory through the host's
// page tables; else false (then the copy pipeline is used).  *pinned tells
// which of the first two it was.
bool reachable_host(const void *p, bool pageable_access, void **dev, bool *pinned)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *dev = a.devicePointer;
        *pinned = true;
        return true;
    }
    if (a.type == cudaMemoryTypeUnregistered && pageable_access) {
        *dev = const_cast<void *>(p);
        *pinned = false;
        return true;
    }
    return false;
}

// The zero-copy plan: the register path with 16-byte plain loads and
// stores (every plan of that path measured the same over the host link).
// Host memory is only ever touched by such loads and stores: the bulk
// (TMA-staged) kernels are for device memory, and this plan never selects
// them.
constexpr sincos_plan kZeroCopyPlan = {256, 4, 4, 16};

int64_t slot_elems_for(int dtype, size_t ws_bytes)
{
    const int64_t per = 4 + 2 * (int64_t)dtype_size(dtype);
    int64_t m = (int64_t)(ws_bytes / kSlots) / per;
    return m - m % 64;   // keeps every sub-buffer 128-byte aligned
}

}  // namespace

}  // namespace sincos_gb300

using namespace sincos_gb300;

extern "C" {

size_t sincos_host_workspace_bytes(int out_dtype, int64_t chunk_elems)
{
    if (!valid_dtype(out_dtype) || chunk_elems <= 0) return 0;
    int64_t m = chunk_elems + 63;
    m -= m % 64;
    return (size_t)kSlots * (size_t)m * (size_t)(4 + 2 * dtype_size(out_dtype));
}

int sincos_pairs_host(const float *x_host, void *s_host, void *c_host, int64_t n, int out_dtype,
                      int reduction, int coef, void *dev_ws, size_t ws_bytes,
                      sincos_stream_t stream)
{
    SINCOS_TRACE("sincos_pairs_host");
    g_last_path = SINCOS_HOST_PATH_NONE;
    if (n < 0 || !valid_dtype(out_dtype) || !valid_reduction(reduction) || !valid_coef(coef))
        return SINCOS_EINVAL;
    if (n == 0) return SINCOS_OK;
    if (!x_host || !s_host || !c_host || !dev_ws || ((uintptr_t)dev_ws & 255u)) return SINCOS_EINVAL;
    if (!aligned_to(x_host, 4) || !aligned_to(s_host, (size_t)dtype_size(out_dtype)) ||
        !aligned_to(c_host, (size_t)dtype_size(out_dtype)))
        return SINCOS_EINVAL;
    const int64_t slot = slot_elems_for(out_dtype, ws_bytes);
    if (slot < 64) return SINCOS_EINVAL;
    const size_t osz = (size_t)dtype_size(out_dtype);
    if (ranges_overlap(s_host, (size_t)n * osz, c_host, (size_t)n * osz)) return SINCOS_EOVERLAP;
    const DeviceInfo *dev = nullptr;
    int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    cudaStream_t user = (cudaStream_t)stream;

    void *xd = nullptr, *sd = nullptr, *cd = nullptr;
    bool px = false, ps = false, pc = false;
    const bool pa = dev->pageable_access;
    if (g_route_policy.load(std::memory_order_relaxed) == SINCOS_HOST_ROUTE_AUTO &&
        reachable_host(x_host, pa, &xd, &px) && reachable_host(s_host, pa, &sd, &ps) &&
        reachable_host(c_host, pa, &cd, &pc)) {
        // zero-copy: the same aliasing rules as sincos_pairs_ex
        const size_t xb = (size_t)n * 4, ob = (size_t)n * osz;
        bool in_place = false;
        for (const void *o : {(const void *)s_host, (const void *)c_host}) {
            if (!ranges_overlap(x_host, xb, o, ob)) continue;
            if (o == (const void *)x_host && out_dtype == SINCOS_F32) in_place = true;
            else return SINCOS_EOVERLAP;
        }
        rc = launch_forward((const float *)xd, sd, cd, n, out_dtype, reduction, coef, in_place,
                            kZeroCopyPlan, *dev, user);
        if (rc == SINCOS_OK)
            g_last_path = px && ps && pc ? SINCOS_HOST_PATH_ZERO_COPY
                                         : SINCOS_HOST_PATH_ZERO_COPY_PAGEABLE;
        return rc;
    }

    Pipe *pipe = nullptr;
    rc = get_pipe(dev->ordinal, &pipe);
    if (rc != SINCOS_OK) return rc;

    char *ws = (char *)dev_ws;
    const size_t slot_bytes = (size_t)slot * (4 + 2 * osz);

    std::lock_guard<std::mutex> lock(pipe->mu);
    cudaError_t e = cudaEventRecord(pipe->start, user);
    for (int k = 0; e == cudaSuccess && k < kSlots; ++k) e = cudaStreamWaitEvent(pipe->st[k], pipe->start, 0);
    if (e != cudaSuccess) return cuda_fail(e, "host path ordering after the caller's stream");

    for (int64_t off = 0, j = 0; off < n; off += slot, ++j) {
        const int k = (int)(j % kSlots);
        cudaStream_t st = pipe->st[k];
        const int64_t m = (n - off < slot) ? n - off : slot;
        float *xd = (float *)(ws + k * slot_bytes);
        char *sd = (char *)xd + (size_t)slot * 4;
        char *cd = sd + (size_t)slot * osz;
        e = cudaMemcpyAsync(xd, x_host + off, (size_t)m * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "host path upload");
        const sincos_plan plan = plan_for(*dev, SINCOS_OP_PAIRS, out_dtype, m);
        rc = launch_forward(xd, sd, cd, m, out_dtype, reduction, coef, false, plan, *dev, st);
        if (rc != SINCOS_OK) return rc;
        e = cudaMemcpyAsync((char *)s_host + (size_t)off * osz, sd, (size_t)m * osz,
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char *)c_host + (size_t)off * osz, cd, (size_t)m * osz,
                                cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "host path download");
    }
    for (int k = 0; k < kSlots; ++k) {
        e = cudaEventRecord(pipe->done[k], pipe->st[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(user, pipe->done[k], 0);
        if (e != cudaSuccess) return cuda_fail(e, "host path ordering before the caller's stream");
    }
    g_last_path = SINCOS_HOST_PATH_PIPELINE;
    return SINCOS_OK;
}

int sincos_host_last_path(void) { return g_last_path; }

int sincos_host_route_set(int policy)
{
    if (policy != SINCOS_HOST_ROUTE_AUTO && policy != SINCOS_HOST_ROUTE_PIPELINE)
        return SINCOS_EINVAL;
    g_route_policy.store(policy, std::memory_order_relaxed);
    return SINCOS_OK;
}

}  // extern "C"
