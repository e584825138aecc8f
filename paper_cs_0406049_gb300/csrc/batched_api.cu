// batched_api.cu -- C ABI of the batched forward: the per-(device, stream)
// prefix scratch, the direct entry points and the CUDA-graph wrapper.
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "trace.h"
#include "internal.h"

namespace sincos_gb300 {

namespace {

struct Scratch {
    int64_t *ptr = nullptr;
    size_t bytes = 0;
};

std::mutex g_scratch_mu;
std::map<std::pair<int, uintptr_t>, Scratch> g_scratch;

bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

int validate(const sincos_seg *segs, const int64_t *lens, int count, int dtype, int red, int coef)
{
    if (count < 0 || !valid_dtype(dtype) || !valid_reduction(red) || !valid_coef(coef))
        return SINCOS_EINVAL;
    if (count > 0 && (!segs || !lens)) return SINCOS_EINVAL;
    if (count > 0 && (!aligned_to(segs, 8) || !aligned_to(lens, 8))) return SINCOS_EINVAL;
    return SINCOS_OK;
}

// Kernel nodes of a captured graph.
int graph_kernel_nodes(cudaGraph_t graph, int *kernels)
{
    size_t nn = 0;
    cudaError_t e = cudaGraphGetNodes(graph, nullptr, &nn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphGetNodes");
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphGetNodes");
    int k = 0;
    for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[i], &t);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphNodeGetType");
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    *kernels = k;
    return SINCOS_OK;
}

}  // namespace

// Device scratch of at least batched_scratch_elems(count) int64 for `st` on
// the current device.
// Grows (after synchronizing `st`, whose earlier batched work may still read
// the old buffer) when too small; refuses to allocate while `st` is captured.
int batched_scratch(cudaStream_t st, int count, int64_t **prefix)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    const size_t need = sizeof(int64_t) * batched_scratch_elems(count);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    Scratch &sc = g_scratch[std::make_pair(dev, (uintptr_t)st)];
    if (sc.bytes < need) {
        if (capturing(st)) return SINCOS_ECAPTURE;
        if (sc.ptr) {
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize (scratch growth)");
            cudaFree(sc.ptr);
            sc.ptr = nullptr;
            sc.bytes = 0;
        }
        size_t bytes = 4096;
        while (bytes < need) bytes *= 2;
        void *p = nullptr;
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (batched scratch)");
        sc.ptr = (int64_t *)p;
        sc.bytes = bytes;
    }
    *prefix = sc.ptr;
    return SINCOS_OK;
}

}  // namespace sincos_gb300

using namespace sincos_gb300;

struct sincos_graph_s {
    int device = -1;
    int64_t *prefix = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

extern "C" {

int sincos_batched_ex(const sincos_seg *segs, const int64_t *lens, int count, int out_dtype,
                      int reduction, int coef, sincos_stream_t stream)
{
    SINCOS_TRACE("sincos_batched_ex");
    int rc = validate(segs, lens, count, out_dtype, reduction, coef);
    if (rc != SINCOS_OK || count == 0) return rc;
    const DeviceInfo *dev = nullptr;
    rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // Batched plans are keyed by the segment count (the lengths live on the
    // device and are not read back).  Only register plans use the schedule
    // scratch; the ring kernel schedules itself.
    const sincos_plan plan = plan_for(*dev, SINCOS_OP_BATCHED, out_dtype, count);
    int64_t *prefix = nullptr;
    if (plan_vec_bytes(plan) != 0) {
        rc = batched_scratch(st, count, &prefix);
        if (rc != SINCOS_OK) return rc;
    }
    return launch_batched(segs, lens, count, out_dtype, reduction, coef, prefix, plan, *dev, st);
}

int sincos_batched(const sincos_seg *segs, const int64_t *lens, int count, sincos_stream_t stream)
{
    return sincos_batched_ex(segs, lens, count, SINCOS_F32, SINCOS_RED_PLAIN,
                             SINCOS_COEF_NORMALIZED, stream);
}

int sincos_batched_release(void)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    int prev = 0;
    cudaGetDevice(&prev);
    int rc = SINCOS_OK;
    for (auto &kv : g_scratch) {
        if (!kv.second.ptr) continue;
        cudaSetDevice(kv.first.first);
        const cudaError_t e = cudaFree(kv.second.ptr);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaFree (batched scratch)");
    }
    g_scratch.clear();
    cudaSetDevice(prev);
    return rc;
}

int sincos_batched_graph_create(const sincos_seg *segs, const int64_t *lens, int count,
                                int out_dtype, int reduction, int coef, sincos_graph *out)
{
    SINCOS_TRACE("sincos_batched_graph_create");
    if (!out) return SINCOS_EINVAL;
    *out = nullptr;
    int rc = validate(segs, lens, count, out_dtype, reduction, coef);
    if (rc != SINCOS_OK) return rc;
    if (count == 0) return SINCOS_EINVAL;
    const DeviceInfo *dev = nullptr;
    rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;

    sincos_graph g = new sincos_graph_s;
    g->device = dev->ordinal;
    cudaStream_t cap = nullptr;
    const sincos_plan plan = plan_for(*dev, SINCOS_OP_BATCHED, out_dtype, count);
    cudaError_t e = cudaSuccess;
    if (plan_vec_bytes(plan) != 0)      // the schedule scratch of register plans
        e = cudaMalloc((void **)&g->prefix, sizeof(int64_t) * batched_scratch_elems(count));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "graph create (scratch or stream)");
        sincos_batched_graph_destroy(g);
        if (cap) cudaStreamDestroy(cap);
        return rc;
    }
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = launch_batched(segs, lens, count, out_dtype, reduction, coef, g->prefix, plan, *dev,
                            cap);
        const cudaError_t e2 = cudaStreamEndCapture(cap, &g->graph);
        if (rc == SINCOS_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
        // Captured kernels are not launches; replays are counted instead.
        // launch_batched counted each kernel it enqueued (one for the ring
        // plan, two for register plans), and each is one kernel node.
        if (rc == SINCOS_OK) rc = graph_kernel_nodes(g->graph, &g->launches);
        if (rc == SINCOS_OK) count_launches((uint64_t)0 - (uint64_t)g->launches);
    } else {
        rc = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (rc == SINCOS_OK) {
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
    }
    cudaStreamDestroy(cap);
    if (rc != SINCOS_OK) {
        sincos_batched_graph_destroy(g);
        return rc;
    }
    *out = g;
    return SINCOS_OK;
}

int sincos_batched_graph_launch(sincos_graph g, sincos_stream_t stream)
{
    SINCOS_TRACE("sincos_batched_graph_launch");
    if (!g || !g->exec) return SINCOS_EINVAL;
    const cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    count_launches((uint64_t)g->launches);
    return SINCOS_OK;
}

int sincos_batched_graph_destroy(sincos_graph g)
{
    if (!g) return SINCOS_EINVAL;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->prefix) cudaFree(g->prefix);
    delete g;
    return SINCOS_OK;
}

}  // extern "C"
