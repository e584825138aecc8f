// forward.cuh -- the forward kernels (one array of angles) and their launcher,
// instantiated per output type by forward_f32.cu and forward_16.cu.
//
// Work layout.  After a scalar head of h < kVec elements that brings x, s and
// c to 16-byte alignment, the array is a sequence of kVec-element vectors.
// A "chunk" is block * UNROLL consecutive vectors; thread t of a CTA owns
// vectors t, t + block, ..., t + (UNROLL-1)*block of the chunk, so each of
// its UNROLL 16-byte loads is coalesced across the warp and all UNROLL loads
// are in flight before the first pair is computed.  CTAs stride over whole
// chunks (grid = resident CTAs per SM x SMs, or fewer for small arrays).  The
// last partial chunk, the head and the tail (< kVec elements) go to the CTA
// that would have had the next chunk.  Arrays whose three pointers admit no
// common 16-byte alignment take the scalar kernel.
#pragma once

#include "core.cuh"
#include "internal.h"

namespace sincos_gb300 {

template <class OutT, int RED, int COEF, int UNROLL, int LD>
__global__ void k_forward(const float *x, OutT *s, OutT *c, int64_t n, int64_t head,
                          int64_t nvec)
{
    constexpr int V = Out<OutT>::kVec;
    const float *xv = x + head;
    OutT *sv = s + head;
    OutT *cv = c + head;
    const int64_t chunk = (int64_t)blockDim.x * UNROLL;
    const int64_t nfull = nvec / chunk;

    for (int64_t ch = blockIdx.x; ch < nfull; ch += gridDim.x) {
        const int64_t v0 = ch * chunk + threadIdx.x;
        InVec<OutT> in[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            load_vec<LD>(in[u], xv + (v0 + (int64_t)u * blockDim.x) * V);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t e = (v0 + (int64_t)u * blockDim.x) * V;
            compute_store<RED, COEF>(in[u], sv + e, cv + e);
        }
    }

    if (blockIdx.x == (unsigned)(nfull % gridDim.x)) {
        for (int64_t v = nfull * chunk + threadIdx.x; v < nvec; v += blockDim.x) {
            InVec<OutT> in;
            load_vec<LD>(in, xv + v * V);
            compute_store<RED, COEF>(in, sv + v * V, cv + v * V);
        }
        for (int64_t i = threadIdx.x; i < head; i += blockDim.x)
            scalar_elem<RED, COEF>(x, s, c, i);
        for (int64_t i = head + nvec * V + threadIdx.x; i < n; i += blockDim.x)
            scalar_elem<RED, COEF>(x, s, c, i);
    }
}

// Element-wise fallback for pointer triples with no common 16-byte alignment.
template <class OutT, int RED, int COEF>
__global__ void k_forward_scalar(const float *x, OutT *s, OutT *c, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        scalar_elem<RED, COEF>(x, s, c, i);
}

template <class OutT, int RED, int COEF, int UNROLL, int LD>
static int launch_forward_vec(const float *x, OutT *s, OutT *c, int64_t n, int64_t head,
                              const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    constexpr int V = Out<OutT>::kVec;
    const void *fn = (const void *)k_forward<OutT, RED, COEF, UNROLL, LD>;
    const int per_sm = resident_ctas(fn, plan.block, plan.ctas_per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t nvec = (n - head) / V;
    const int64_t chunks = nvec / ((int64_t)plan.block * UNROLL);
    int64_t grid = (int64_t)per_sm * dev.sms;
    if (chunks < grid) grid = chunks > 0 ? chunks : 1;
    k_forward<OutT, RED, COEF, UNROLL, LD><<<(unsigned)grid, plan.block, 0, st>>>(x, s, c, n, head,
                                                                                 nvec);
    return check_launch("forward kernel launch");
}

template <class OutT, int RED, int COEF>
static int launch_forward_rc(const float *x, OutT *s, OutT *c, int64_t n, bool in_place,
                             const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    const int h = vector_head<OutT>(x, s, c);
    if (h < 0) {
        const void *fn = (const void *)k_forward_scalar<OutT, RED, COEF>;
        const int per_sm = resident_ctas(fn, plan.block, plan.ctas_per_sm);
        if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
        int64_t grid = (int64_t)per_sm * dev.sms;
        const int64_t need = (n + plan.block - 1) / plan.block;
        if (need < grid) grid = need;
        k_forward_scalar<OutT, RED, COEF><<<(unsigned)grid, plan.block, 0, st>>>(x, s, c, n);
        return check_launch("forward scalar kernel launch");
    }
    const int64_t head = h < n ? h : n;
    // In place (x == s or x == c): every element is read before the same
    // thread overwrites it, but the non-coherent load path is only defined
    // for memory the kernel does not write, so use coherent loads.
    if (in_place)
        return launch_forward_vec<OutT, RED, COEF, 4, LD_COHERENT>(x, s, c, n, head, plan, dev, st);
    switch (plan.unroll) {
    case 1: return launch_forward_vec<OutT, RED, COEF, 1, LD_NC>(x, s, c, n, head, plan, dev, st);
    case 2: return launch_forward_vec<OutT, RED, COEF, 2, LD_NC>(x, s, c, n, head, plan, dev, st);
    case 4: return launch_forward_vec<OutT, RED, COEF, 4, LD_NC>(x, s, c, n, head, plan, dev, st);
    case 8: return launch_forward_vec<OutT, RED, COEF, 8, LD_NC>(x, s, c, n, head, plan, dev, st);
    default: return SINCOS_EINVAL;
    }
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
