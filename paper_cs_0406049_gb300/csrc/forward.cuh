// forward.cuh -- the forward kernels (one array of angles) and their launcher,
// instantiated per output type by forward_f32.cu, forward_bf16.cu and
// forward_f16.cu.
//
// Work layout.  After a scalar head of h elements that brings x, s and c to a
// 128-byte line boundary (or at least to vector alignment; see vector_head),
// the array is a sequence of E-element vectors (E pairs = W bytes of sines
// and W of cosines, W = 16 or 32 from the launch plan).  A
// "chunk" is block * UNROLL consecutive vectors; thread t of a CTA owns
// vectors t, t + block, ..., t + (UNROLL-1)*block of the chunk, so each load
// is coalesced across the warp and all UNROLL loads are in flight before the
// first pair is computed.  CTAs stride over whole chunks (grid = resident
// CTAs per SM x SMs, or fewer for small arrays).  The last partial chunk, the
// head and the tail (< E elements) go to the CTA that would have had the next
// chunk; it handles them after its vector work.  Pointer triples with no
// common vector alignment take the element-wise kernel.
#pragma once

#include "bulk.cuh"
#include "core.cuh"
#include "internal.h"

namespace sincos_gb300 {

template <class OutT, int RED, int COEF, int UNROLL, int LD, int W>
__global__ void k_forward(const float *x, OutT *s, OutT *c, int64_t n, int64_t head,
                          int64_t nvec)
{
    constexpr int E = Vec<OutT, W>::E;
    const float *xv = x + head;
    OutT *sv = s + head;
    OutT *cv = c + head;
    const int64_t chunk = (int64_t)blockDim.x * UNROLL;
    const int64_t nfull = nvec / chunk;

    for (int64_t ch = blockIdx.x; ch < nfull; ch += gridDim.x) {
        const int64_t v0 = ch * chunk + threadIdx.x;
        float in[UNROLL][E];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            load_vec<OutT, W, LD>(in[u], xv + (v0 + (int64_t)u * blockDim.x) * E);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t e = (v0 + (int64_t)u * blockDim.x) * E;
            compute_store<RED, COEF, OutT, W>(in[u], sv + e, cv + e);
        }
    }

    if (blockIdx.x == (unsigned)(nfull % gridDim.x)) {
        for (int64_t v = nfull * chunk + threadIdx.x; v < nvec; v += blockDim.x) {
            float in[E];
            load_vec<OutT, W, LD>(in, xv + v * E);
            compute_store<RED, COEF, OutT, W>(in, sv + v * E, cv + v * E);
        }
        for (int64_t i = threadIdx.x; i < head; i += blockDim.x)
            scalar_elem<RED, COEF>(x, s, c, i);
        for (int64_t i = head + nvec * E + threadIdx.x; i < n; i += blockDim.x)
            scalar_elem<RED, COEF>(x, s, c, i);
    }
}

// Element-wise fallback for pointer triples with no common vector alignment.
template <class OutT, int RED, int COEF>
__global__ void k_forward_scalar(const float *x, OutT *s, OutT *c, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        scalar_elem<RED, COEF>(x, s, c, i);
}

template <class OutT, int RED, int COEF, int UNROLL, int LD, int W>
static int launch_forward_vec(const float *x, OutT *s, OutT *c, int64_t n, int64_t head,
                              const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    constexpr int E = Vec<OutT, W>::E;
    const void *fn = (const void *)k_forward<OutT, RED, COEF, UNROLL, LD, W>;
    int per_sm = 0;
    const sincos_plan p = fit_plan(fn, plan, &per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t nvec = (n - head) / E;
    const int64_t chunks = nvec / ((int64_t)p.block * UNROLL);
    int64_t grid = (int64_t)per_sm * dev.sms;
    if (chunks < grid) grid = chunks > 0 ? chunks : 1;
    k_forward<OutT, RED, COEF, UNROLL, LD, W><<<(unsigned)grid, p.block, 0, st>>>(
        x, s, c, n, head, nvec);
    return check_launch("forward kernel launch");
}

template <class OutT, int RED, int COEF, int W>
static int launch_forward_w(const float *x, OutT *s, OutT *c, int64_t n, int h, bool in_place,
                            const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    const int64_t head = h < n ? h : n;
    // In place (x == s or x == c): every element is read before the same
    // thread overwrites it, but the non-coherent load path is only defined
    // for memory the kernel does not write, so use coherent loads.
    if (in_place)
        return launch_forward_vec<OutT, RED, COEF, 4, LD_COHERENT, W>(x, s, c, n, head, plan, dev,
                                                                      st);
    switch (plan.unroll) {
    case 1: return launch_forward_vec<OutT, RED, COEF, 1, LD_NC, W>(x, s, c, n, head, plan, dev, st);
    case 2: return launch_forward_vec<OutT, RED, COEF, 2, LD_NC, W>(x, s, c, n, head, plan, dev, st);
    case 4: return launch_forward_vec<OutT, RED, COEF, 4, LD_NC, W>(x, s, c, n, head, plan, dev, st);
    case 8: return launch_forward_vec<OutT, RED, COEF, 8, LD_NC, W>(x, s, c, n, head, plan, dev, st);
    default: return SINCOS_EINVAL;
    }
}

template <class OutT, int RED, int COEF>
static int launch_forward_rc(const float *x, OutT *s, OutT *c, int64_t n, bool in_place,
                             const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    // Bulk (TMA-staged) path when the plan asks for it and the array holds at
    // least one whole chunk after its aligned start.  ctas_per_sm >= 2 asks
    // for the small-stage variant (several CTAs per SM).
    if (plan_vec_bytes(plan) == 0 && plan.ctas_per_sm >= 2) {
        const int h = vector_head<OutT, 16>(x, s, c);
        if (h >= 0 && n - h >= kBulkSmallChunk) {
            switch (plan.block) {
            case 128:
                return launch_forward_bulk_nt<OutT, RED, COEF, 128, kBulkSmallChunk>(x, s, c, n, h,
                                                                                      dev, st);
            case 256:
                return launch_forward_bulk_nt<OutT, RED, COEF, 256, kBulkSmallChunk>(x, s, c, n, h,
                                                                                      dev, st);
            default:
                return launch_forward_bulk_nt<OutT, RED, COEF, 512, kBulkSmallChunk>(x, s, c, n, h,
                                                                                      dev, st);
            }
        }
    } else if (plan_vec_bytes(plan) == 0) {
        const int h = vector_head<OutT, 16>(x, s, c);
        if (h >= 0 && n - h >= kBulkChunk) {
            switch (plan.block) {
            case 128: return launch_forward_bulk_nt<OutT, RED, COEF, 128>(x, s, c, n, h, dev, st);
            case 512: return launch_forward_bulk_nt<OutT, RED, COEF, 512>(x, s, c, n, h, dev, st);
            case 1024: return launch_forward_bulk_nt<OutT, RED, COEF, 1024>(x, s, c, n, h, dev, st);
            default: return launch_forward_bulk_nt<OutT, RED, COEF, 256>(x, s, c, n, h, dev, st);
            }
        }
    }
    // The plan's access width first; a 16-byte vector path if the pointers
    // only admit that; element-wise otherwise.
    if (plan_vec_bytes(plan) == 32) {
        const int h = vector_head<OutT, 32>(x, s, c);
        if (h >= 0)
            return launch_forward_w<OutT, RED, COEF, 32>(x, s, c, n, h, in_place, plan, dev, st);
    }
    const int h = vector_head<OutT, 16>(x, s, c);
    if (h >= 0)
        return launch_forward_w<OutT, RED, COEF, 16>(x, s, c, n, h, in_place, plan, dev, st);
    const void *fn = (const void *)k_forward_scalar<OutT, RED, COEF>;
    int per_sm = 0;
    const sincos_plan p = fit_plan(fn, plan, &per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    int64_t grid = (int64_t)per_sm * dev.sms;
    const int64_t need = (n + p.block - 1) / p.block;
    if (need < grid) grid = need;
    k_forward_scalar<OutT, RED, COEF><<<(unsigned)grid, p.block, 0, st>>>(x, s, c, n);
    return check_launch("forward scalar kernel launch");
}

template <class OutT>
int launch_forward_t(const float *x, OutT *s, OutT *c, int64_t n, int red, int coef,
                     bool in_place, const sincos_plan &plan, const DeviceInfo &dev,
                     cudaStream_t st)
{
    if (red == RED_PLAIN && coef == COEF_NORMALIZED)
        return launch_forward_rc<OutT, RED_PLAIN, COEF_NORMALIZED>(x, s, c, n, in_place, plan, dev, st);
    if (red == RED_COMPENSATED && coef == COEF_NORMALIZED)
        return launch_forward_rc<OutT, RED_COMPENSATED, COEF_NORMALIZED>(x, s, c, n, in_place, plan,
                                                                         dev, st);
    if (red == RED_PLAIN && coef == COEF_DAGGER)
        return launch_forward_rc<OutT, RED_PLAIN, COEF_DAGGER>(x, s, c, n, in_place, plan, dev, st);
    return launch_forward_rc<OutT, RED_COMPENSATED, COEF_DAGGER>(x, s, c, n, in_place, plan, dev, st);
}

}  // namespace sincos_gb300
