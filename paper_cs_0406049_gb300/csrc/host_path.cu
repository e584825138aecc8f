// host_path.cu -- the forward on host arrays.
//
// Page-locked, mapped buffers (cudaHostAlloc, cudaMallocHost, or
// cudaHostRegister with mapping) are read and written by the kernel itself
// across the host link (zero-copy), with the register path's plain vector
// loads and stores.  On GB300's NVLink-C2C that moves 272 GB/s against 262
// for the copy pipeline, which loses its fill and drain.  Other host memory
// goes through the pipeline: chunked host -> device copy, kernel, device ->
// host copy, with consecutive chunks on three rotating internal streams, so
// that one chunk's upload, another's kernel and a third's download proceed at
// once.  The device side of the pipeline uses only the caller's workspace.
#include <mutex>

#include "trace.h"
#include "internal.h"

namespace sincos_gb300 {

namespace {

constexpr int kSlots = 3;
constexpr int kMaxDevices = 64;

// The route the calling thread's last sincos_pairs_host call took.
thread_local int g_last_path = SINCOS_HOST_PATH_NONE;

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

// Device address of a host buffer the GPU can access directly (page-locked
// and mapped), or false (then the copy pipeline is used).
bool mapped_host(const void *p, void **dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dev = a.devicePointer;
    return true;
}

// The zero-copy plan: the register path with 16-byte plain loads and
// stores (every plan of that path measured the same over the host link).
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
    if (mapped_host(x_host, &xd) && mapped_host(s_host, &sd) && mapped_host(c_host, &cd)) {
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
        if (rc == SINCOS_OK) g_last_path = SINCOS_HOST_PATH_ZERO_COPY;
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

}  // extern "C"
