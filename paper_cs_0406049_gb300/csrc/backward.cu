// backward.cu -- gradient of the pair with respect to the angle.
//
// d/dx [gs sin x + gc cos x] = gs cos x - gc sin x, evaluated on the forward's
// own outputs (s, c) as gx = fma(gs, c, -(gc*s)).  The method is smooth
// inside each period (Sec. Methodology: no seams except the wrap at odd
// multiples of pi), so this is the derivative a caller differentiating
// through the pair expects.  Four streams in (gs, gc, s, c), one out; a null
// gs or gc stands for zeros and its stream is not read.  Same chunked vector
// layout as the forward kernels (see forward.cuh), E = W/4 gradients per
// 16- or 32-byte vector.
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

// One W-byte vector of gradients from W-byte vectors of the used inputs.
template <bool GS, bool GC, int LD, int W>
__device__ __forceinline__ void grad_load(float (&vgs)[W / 4], float (&vgc)[W / 4],
                                          float (&vs)[W / 4], float (&vc)[W / 4],
                                          const float *gs, const float *gc, const float *s,
                                          const float *c, int64_t e)
{
    if (GS) load_f32<W, LD>(vgs, gs + e);
    if (GC) load_f32<W, LD>(vgc, gc + e);
    if (GC) load_f32<W, LD>(vs, s + e);
    if (GS) load_f32<W, LD>(vc, c + e);
}

template <bool GS, bool GC, int W>
__device__ __forceinline__ void grad_store(const float (&vgs)[W / 4], const float (&vgc)[W / 4],
                                           const float (&vs)[W / 4], const float (&vc)[W / 4],
                                           float *gx)
{
    uint32_t w[W / 4];
#pragma unroll
    for (int i = 0; i < W / 4; ++i)
        w[i] = __float_as_uint(grad<GS, GC>(GS ? vgs[i] : 0.f, GC ? vgc[i] : 0.f,
                                            GC ? vs[i] : 0.f, GS ? vc[i] : 0.f));
    store_words<W>(gx, w);
}

template <bool GS, bool GC>
__device__ __forceinline__ void grad_elem(const float *gs, const float *gc, const float *s,
                                          const float *c, float *gx, int64_t i)
{
    gx[i] = grad<GS, GC>(GS ? gs[i] : 0.f, GC ? gc[i] : 0.f, GC ? s[i] : 0.f, GS ? c[i] : 0.f);
}

// Same chunked layout as k_forward with E = W/4 gradients per vector.
template <bool GS, bool GC, int UNROLL, int LD, int W>
__global__ void k_backward(const float *gs, const float *gc, const float *s, const float *c,
                           float *gx, int64_t n, int64_t head, int64_t nvec)
{
    constexpr int E = W / 4;
    const int64_t chunk = (int64_t)blockDim.x * UNROLL;
    const int64_t nfull = nvec / chunk;
    for (int64_t ch = blockIdx.x; ch < nfull; ch += gridDim.x) {
        const int64_t v0 = ch * chunk + threadIdx.x;
        float vgs[UNROLL][E], vgc[UNROLL][E], vs[UNROLL][E], vc[UNROLL][E];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            grad_load<GS, GC, LD, W>(vgs[u], vgc[u], vs[u], vc[u], gs, gc, s, c,
                                     head + (v0 + (int64_t)u * blockDim.x) * E);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            grad_store<GS, GC, W>(vgs[u], vgc[u], vs[u], vc[u],
                                  gx + head + (v0 + (int64_t)u * blockDim.x) * E);
    }
    if (blockIdx.x == (unsigned)(nfull % gridDim.x)) {
        for (int64_t v = nfull * chunk + threadIdx.x; v < nvec; v += blockDim.x) {
            float vgs[E], vgc[E], vs[E], vc[E];
            grad_load<GS, GC, LD, W>(vgs, vgc, vs, vc, gs, gc, s, c, head + v * E);
            grad_store<GS, GC, W>(vgs, vgc, vs, vc, gx + head + v * E);
        }
        for (int64_t i = threadIdx.x; i < head; i += blockDim.x)
            grad_elem<GS, GC>(gs, gc, s, c, gx, i);
        for (int64_t i = head + nvec * E + threadIdx.x; i < n; i += blockDim.x)
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

// Smallest h with every used pointer + h on a 128-byte line if their line
// offsets agree, else in [0, W/4) with every pointer + h W-byte aligned, or
// -1 (no common vector alignment).
static int backward_head(const float *const *ptrs, int k, int w)
{
    bool same_line_offset = true;
    for (int i = 1; i < k; ++i)
        same_line_offset = same_line_offset &&
                           (((uintptr_t)ptrs[i] & 127u) == ((uintptr_t)ptrs[0] & 127u));
    if (same_line_offset && ((uintptr_t)ptrs[0] & 3u) == 0)
        return (int)(((128u - ((uintptr_t)ptrs[0] & 127u)) & 127u) / 4u);
    for (int h = 0; h < w / 4; ++h) {
        bool ok = true;
        for (int i = 0; i < k; ++i)
            ok = ok && ((((uintptr_t)ptrs[i]) + 4u * h) % (unsigned)w) == 0;
        if (ok) return h;
    }
    return -1;
}

template <bool GS, bool GC, int UNROLL, int LD, int W>
static int launch_bwd_vec(const float *gs, const float *gc, const float *s, const float *c,
                          float *gx, int64_t n, int64_t head, const sincos_plan &plan,
                          const DeviceInfo &dev, cudaStream_t st)
{
    const void *fn = (const void *)k_backward<GS, GC, UNROLL, LD, W>;
    int per_sm = 0;
    const sincos_plan p = fit_plan(fn, plan, &per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t nvec = (n - head) / (W / 4);
    const int64_t chunks = nvec / ((int64_t)p.block * UNROLL);
    int64_t grid = (int64_t)per_sm * dev.sms;
    if (chunks < grid) grid = chunks > 0 ? chunks : 1;
    k_backward<GS, GC, UNROLL, LD, W><<<(unsigned)grid, p.block, 0, st>>>(gs, gc, s, c, gx, n,
                                                                          head, nvec);
    return check_launch("backward kernel launch");
}

template <bool GS, bool GC, int W>
static int launch_bwd_w(const float *gs, const float *gc, const float *s, const float *c,
                        float *gx, int64_t n, int h, bool in_place, const sincos_plan &plan,
                        const DeviceInfo &dev, cudaStream_t st)
{
    const int64_t head = h < n ? h : n;
    if (in_place)
        return launch_bwd_vec<GS, GC, 2, LD_COHERENT, W>(gs, gc, s, c, gx, n, head, plan, dev, st);
    switch (plan.unroll) {
    case 1: return launch_bwd_vec<GS, GC, 1, LD_NC, W>(gs, gc, s, c, gx, n, head, plan, dev, st);
    case 2: return launch_bwd_vec<GS, GC, 2, LD_NC, W>(gs, gc, s, c, gx, n, head, plan, dev, st);
    case 4: return launch_bwd_vec<GS, GC, 4, LD_NC, W>(gs, gc, s, c, gx, n, head, plan, dev, st);
    case 8: return launch_bwd_vec<GS, GC, 8, LD_NC, W>(gs, gc, s, c, gx, n, head, plan, dev, st);
    default: return SINCOS_EINVAL;
    }
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
    if (reg_vec_bytes(plan) == 32) {
        const int h = backward_head(ptrs, k, 32);
        if (h >= 0) return launch_bwd_w<GS, GC, 32>(gs, gc, s, c, gx, n, h, in_place, plan, dev, st);
    }
    const int h = backward_head(ptrs, k, 16);
    if (h >= 0) return launch_bwd_w<GS, GC, 16>(gs, gc, s, c, gx, n, h, in_place, plan, dev, st);
    const void *fn = (const void *)k_backward_scalar<GS, GC>;
    int per_sm = 0;
    const sincos_plan p = fit_plan(fn, plan, &per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    int64_t grid = (int64_t)per_sm * dev.sms;
    const int64_t need = (n + p.block - 1) / p.block;
    if (need < grid) grid = need;
    k_backward_scalar<GS, GC><<<(unsigned)grid, p.block, 0, st>>>(gs, gc, s, c, gx, n);
    return check_launch("backward scalar kernel launch");
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
