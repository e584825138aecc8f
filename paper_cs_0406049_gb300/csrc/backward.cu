// backward.cu -- gradient of the pair with respect to the angle.
//
// d/dx [gs sin x + gc cos x] = gs cos x - gc sin x, evaluated on the forward's
// own outputs (s, c) as gx = fma(gs, c, -(gc*s)).  The method is smooth
// inside each period (Sec. Methodology: no seams except the wrap at odd
// multiples of pi), so this is the derivative a caller differentiating
// through the pair expects.  Four streams in (gs, gc, s, c), one out; a null
// gs or gc stands for zeros and its stream is not read.  Same chunked
// 16-byte layout as the forward kernels (see forward.cuh).
#include "core.cuh"
#include "internal.h"

namespace sincos_gb300 {

template <bool GS, bool GC>
__device__ __forceinline__ float grad(float gs, float gc, float s, float c)
{
    if (GS && GC) return __fmaf_rn(gs, c, -__fmul_rn(gc, s));
    if (GC) return -__fmul_rn(gc, s);
    if (GS) return __fmul_rn(gs, c);
    return 0.0f;
}

template <bool GS, bool GC, int LD>
__device__ __forceinline__ void grad_vec(const float *gs, const float *gc, const float *s,
                                         const float *c, float *gx, int64_t e)
{
    float4 vgs = make_float4(0.f, 0.f, 0.f, 0.f), vgc = vgs, vs = vgs, vc = vgs;
    if (GS) vgs = ld16<LD>(gs + e);
    if (GC) vgc = ld16<LD>(gc + e);
    if (GC) vs = ld16<LD>(s + e);
    if (GS) vc = ld16<LD>(c + e);
    st16(gx + e, grad<GS, GC>(vgs.x, vgc.x, vs.x, vc.x), grad<GS, GC>(vgs.y, vgc.y, vs.y, vc.y),
         grad<GS, GC>(vgs.z, vgc.z, vs.z, vc.z), grad<GS, GC>(vgs.w, vgc.w, vs.w, vc.w));
}

template <bool GS, bool GC>
__device__ __forceinline__ void grad_elem(const float *gs, const float *gc, const float *s,
                                          const float *c, float *gx, int64_t i)
{
    gx[i] = grad<GS, GC>(GS ? gs[i] : 0.f, GC ? gc[i] : 0.f, GC ? s[i] : 0.f, GS ? c[i] : 0.f);
}

template <bool GS, bool GC, int UNROLL, int LD>
__global__ void k_backward(const float *gs, const float *gc, const float *s, const float *c,
                           float *gx, int64_t n, int64_t head, int64_t nvec)
{
    const int64_t chunk = (int64_t)blockDim.x * UNROLL;
    const int64_t nfull = nvec / chunk;
    for (int64_t ch = blockIdx.x; ch < nfull; ch += gridDim.x) {
        const int64_t v0 = ch * chunk + threadIdx.x;
        float4 vgs[UNROLL], vgc[UNROLL], vs[UNROLL], vc[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t e = head + (v0 + (int64_t)u * blockDim.x) * 4;
            if (GS) vgs[u] = ld16<LD>(gs + e);
            if (GC) vgc[u] = ld16<LD>(gc + e);
            if (GC) vs[u] = ld16<LD>(s + e);
            if (GS) vc[u] = ld16<LD>(c + e);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t e = head + (v0 + (int64_t)u * blockDim.x) * 4;
            if (!GS) vgs[u] = vc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!GC) vgc[u] = vs[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            st16(gx + e, grad<GS, GC>(vgs[u].x, vgc[u].x, vs[u].x, vc[u].x),
                 grad<GS, GC>(vgs[u].y, vgc[u].y, vs[u].y, vc[u].y),
                 grad<GS, GC>(vgs[u].z, vgc[u].z, vs[u].z, vc[u].z),
                 grad<GS, GC>(vgs[u].w, vgc[u].w, vs[u].w, vc[u].w));
        }
    }
    if (blockIdx.x == (unsigned)(nfull % gridDim.x)) {
        for (int64_t v = nfull * chunk + threadIdx.x; v < nvec; v += blockDim.x)
            grad_vec<GS, GC, LD>(gs, gc, s, c, gx, head + v * 4);
        for (int64_t i = threadIdx.x; i < head; i += blockDim.x)
            grad_elem<GS, GC>(gs, gc, s, c, gx, i);
        for (int64_t i = head + nvec * 4 + threadIdx.x; i < n; i += blockDim.x)
            grad_elem<GS, GC>(gs, gc, s, c, gx, i);
    }
}

template <bool GS, bool GC>
__global__ void k_backward_scalar(const float *gs, const float *gc, const float *s,
                                  const float *c, float *gx, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        grad_elem<GS, GC>(gs, gc, s, c, gx, i);
}

// Smallest h in [0, 4) with every used pointer + h 16-byte aligned, or -1.
static int backward_head(const float *const *ptrs, int k)
{
    for (int h = 0; h < 4; ++h) {
        bool ok = true;
        for (int i = 0; i < k; ++i)
            ok = ok && ((((uintptr_t)ptrs[i]) + 4u * h) & 15u) == 0;
        if (ok) return h;
    }
    return -1;
}

template <bool GS, bool GC, int UNROLL, int LD>
static int launch_bwd_vec(const float *gs, const float *gc, const float *s, const float *c,
                          float *gx, int64_t n, int64_t head, const sincos_plan &plan,
                          const DeviceInfo &dev, cudaStream_t st)
{
    const void *fn = (const void *)k_backward<GS, GC, UNROLL, LD>;
    const int per_sm = resident_ctas(fn, plan.block, plan.ctas_per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t nvec = (n - head) / 4;
    const int64_t chunks = nvec / ((int64_t)plan.block * UNROLL);
    int64_t grid = (int64_t)per_sm * dev.sms;
    if (chunks < grid) grid = chunks > 0 ? chunks : 1;
    k_backward<GS, GC, UNROLL, LD><<<(unsigned)grid, plan.block, 0, st>>>(gs, gc, s, c, gx, n,
                                                                          head, nvec);
    return check_launch("backward kernel launch");
}

template <bool GS, bool GC>
static int launch_bwd_gc(const float *gs, const float *gc, const float *s, const float *c,
                         float *gx, int64_t n, bool in_place, const sincos_plan &plan,
                         const DeviceInfo &dev, cudaStream_t st)
{
    const float *ptrs[5];
    int k = 0;
    if (GS) { ptrs[k++] = gs; ptrs[k++] = c; }
    if (GC) { ptrs[k++] = gc; ptrs[k++] = s; }
    ptrs[k++] = gx;
    const int h = backward_head(ptrs, k);
    if (h < 0) {
        const void *fn = (const void *)k_backward_scalar<GS, GC>;
        const int per_sm = resident_ctas(fn, plan.block, plan.ctas_per_sm);
        if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
        int64_t grid = (int64_t)per_sm * dev.sms;
        const int64_t need = (n + plan.block - 1) / plan.block;
        if (need < grid) grid = need;
        k_backward_scalar<GS, GC><<<(unsigned)grid, plan.block, 0, st>>>(gs, gc, s, c, gx, n);
        return check_launch("backward scalar kernel launch");
    }
    const int64_t head = h < n ? h : n;
    if (in_place)
        return launch_bwd_vec<GS, GC, 2, LD_COHERENT>(gs, gc, s, c, gx, n, head, plan, dev, st);
    switch (plan.unroll) {
    case 1: return launch_bwd_vec<GS, GC, 1, LD_NC>(gs, gc, s, c, gx, n, head, plan, dev, st);
    case 2: return launch_bwd_vec<GS, GC, 2, LD_NC>(gs, gc, s, c, gx, n, head, plan, dev, st);
    case 4: return launch_bwd_vec<GS, GC, 4, LD_NC>(gs, gc, s, c, gx, n, head, plan, dev, st);
    case 8: return launch_bwd_vec<GS, GC, 8, LD_NC>(gs, gc, s, c, gx, n, head, plan, dev, st);
    default: return SINCOS_EINVAL;
    }
}

int launch_backward(const float *gs, const float *gc, const float *s, const float *c, float *gx,
                    int64_t n, bool in_place, const sincos_plan &plan, const DeviceInfo &dev,
                    cudaStream_t st)
{
    if (gs && gc) return launch_bwd_gc<true, true>(gs, gc, s, c, gx, n, in_place, plan, dev, st);
    if (gs) return launch_bwd_gc<true, false>(gs, gc, s, c, gx, n, in_place, plan, dev, st);
    if (gc) return launch_bwd_gc<false, true>(gs, gc, s, c, gx, n, in_place, plan, dev, st);
    return launch_bwd_gc<false, false>(gs, gc, s, c, gx, n, in_place, plan, dev, st);
}

}  // namespace sincos_gb300
