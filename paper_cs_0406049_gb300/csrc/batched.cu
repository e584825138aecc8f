// batched.cu -- the forward over many independent arrays in one launch pair.
//
// Element space.  Each array (segment) is cut into tiles of T = block *
// UNROLL * kVec elements (the last tile of a segment may be short).  Tile
// numbers are global: a prefix kernel writes prefix[i] = number of tiles in
// segments 0 .. i-1 into device scratch, so segment i owns tiles
// [prefix[i], prefix[i+1]).
//
// Schedule.  The tile kernel is persistent: CTA b of G takes the contiguous
// run of tiles [total*b/G, total*(b+1)/G).  It finds the segment of its first
// tile by binary search over the prefix array once, then walks forward (one
// comparison per tile, one extra load when it crosses into the next
// segment), so the per-tile bookkeeping is a few L1-resident loads.  Within a
// tile thread t owns vectors t, t + block, ... exactly as in the single-array
// kernel, after a scalar head that aligns the segment's three pointers.  No
// CTA waits on another and no counter is shared, so nothing can spin.
#include "core.cuh"
#include "internal.h"

namespace sincos_gb300 {

// prefix[0] = 0; prefix[i+1] = prefix[i] + ceil(max(lens[i], 0) / tile).
// One CTA of 1024 threads scans the lengths 1024 at a time.
__global__ void k_batched_prefix(const int64_t *lens, int count, int64_t tile, int64_t *prefix)
{
    __shared__ int64_t warp_total[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        carry = 0;
        prefix[0] = 0;
    }
    __syncthreads();
    for (int base = 0; base < count; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int64_t v = 0;
        if (i < count) {
            const int64_t len = lens[i];
            v = len > 0 ? (len + tile - 1) / tile : 0;
        }
        int64_t incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) warp_total[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = lane < nwarps ? warp_total[lane] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t t = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += t;
            }
            warp_total[lane] = w;   // inclusive over warps
        }
        __syncthreads();
        const int64_t mine = carry + (warp > 0 ? warp_total[warp - 1] : 0) + incl;
        if (i < count) prefix[i + 1] = mine;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = mine;
        __syncthreads();
    }
}

template <class OutT, int RED, int COEF, int UNROLL>
__device__ __forceinline__ void tile_work(const float *x, OutT *s, OutT *c, int64_t m)
{
    constexpr int V = Out<OutT>::kVec;
    int h = vector_head<OutT>(x, s, c);
    if (h < 0) {
        for (int64_t i = threadIdx.x; i < m; i += blockDim.x)
            scalar_elem<RED, COEF>(x, s, c, i);
        return;
    }
    if (h > m) h = (int)m;
    const int64_t nv = (m - h) / V;
    const float *xv = x + h;
    OutT *sv = s + h;
    OutT *cv = c + h;
    InVec<OutT> in[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
        const int64_t j = threadIdx.x + (int64_t)u * blockDim.x;
        if (j < nv) load_vec<LD_NC>(in[u], xv + j * V);
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
        const int64_t j = threadIdx.x + (int64_t)u * blockDim.x;
        if (j < nv) compute_store<RED, COEF>(in[u], sv + j * V, cv + j * V);
    }
    if ((int)threadIdx.x < h) scalar_elem<RED, COEF>(x, s, c, threadIdx.x);
    for (int64_t i = h + nv * V + threadIdx.x; i < m; i += blockDim.x)
        scalar_elem<RED, COEF>(x, s, c, i);
}

template <class OutT, int RED, int COEF, int UNROLL>
__global__ void k_batched(const sincos_seg *segs, const int64_t *lens, const int64_t *prefix,
                          int count)
{
    constexpr int V = Out<OutT>::kVec;
    const int64_t tile = (int64_t)blockDim.x * UNROLL * V;
    const int64_t total = prefix[count];
    const int64_t t0 = total * blockIdx.x / gridDim.x;
    const int64_t t1 = total * (blockIdx.x + 1) / gridDim.x;
    if (t0 >= t1) return;

    // Segment of tile t0: the last i in [0, count) with prefix[i] <= t0.
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t0) lo = mid;
        else hi = mid - 1;
    }
    int seg = lo;
    int64_t seg_first = prefix[seg];
    int64_t seg_end = prefix[seg + 1];
    for (int64_t t = t0; t < t1; ++t) {
        while (t >= seg_end) {          // also skips empty segments
            ++seg;
            seg_first = seg_end;
            seg_end = prefix[seg + 1];
        }
        const sincos_seg d = segs[seg];
        const int64_t e0 = (t - seg_first) * tile;
        const int64_t rest = lens[seg] - e0;
        const int64_t m = rest < tile ? rest : tile;
        tile_work<OutT, RED, COEF, UNROLL>(d.x + e0, (OutT *)d.s + e0, (OutT *)d.c + e0, m);
    }
}

int64_t batched_tile_elems(const sincos_plan &plan, int dtype)
{
    return (int64_t)plan.block * plan.unroll * (dtype == SINCOS_F32 ? 4 : 8);
}

template <class OutT, int RED, int COEF, int UNROLL>
static int launch_tiles(const sincos_seg *segs, const int64_t *lens, int count, int64_t *prefix,
                        const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    const void *fn = (const void *)k_batched<OutT, RED, COEF, UNROLL>;
    const int per_sm = resident_ctas(fn, plan.block, plan.ctas_per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const unsigned grid = (unsigned)per_sm * (unsigned)dev.sms;
    k_batched<OutT, RED, COEF, UNROLL><<<grid, plan.block, 0, st>>>(segs, lens, prefix, count);
    return check_launch("batched tile kernel launch");
}

template <class OutT, int RED, int COEF>
static int launch_tiles_u(const sincos_seg *segs, const int64_t *lens, int count, int64_t *prefix,
                          const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    switch (plan.unroll) {
    case 1: return launch_tiles<OutT, RED, COEF, 1>(segs, lens, count, prefix, plan, dev, st);
    case 2: return launch_tiles<OutT, RED, COEF, 2>(segs, lens, count, prefix, plan, dev, st);
    case 4: return launch_tiles<OutT, RED, COEF, 4>(segs, lens, count, prefix, plan, dev, st);
    case 8: return launch_tiles<OutT, RED, COEF, 8>(segs, lens, count, prefix, plan, dev, st);
    default: return SINCOS_EINVAL;
    }
}

template <class OutT>
static int launch_tiles_t(const sincos_seg *segs, const int64_t *lens, int count, int64_t *prefix,
                          int red, int coef, const sincos_plan &plan, const DeviceInfo &dev,
                          cudaStream_t st)
{
    if (red == RED_PLAIN && coef == COEF_NORMALIZED)
        return launch_tiles_u<OutT, RED_PLAIN, COEF_NORMALIZED>(segs, lens, count, prefix, plan, dev, st);
    if (red == RED_COMPENSATED && coef == COEF_NORMALIZED)
        return launch_tiles_u<OutT, RED_COMPENSATED, COEF_NORMALIZED>(segs, lens, count, prefix, plan,
                                                                      dev, st);
    if (red == RED_PLAIN && coef == COEF_DAGGER)
        return launch_tiles_u<OutT, RED_PLAIN, COEF_DAGGER>(segs, lens, count, prefix, plan, dev, st);
    return launch_tiles_u<OutT, RED_COMPENSATED, COEF_DAGGER>(segs, lens, count, prefix, plan, dev,
                                                              st);
}

int launch_batched(const sincos_seg *segs, const int64_t *lens, int count, int dtype, int red,
                   int coef, int64_t *prefix, const sincos_plan &plan, const DeviceInfo &dev,
                   cudaStream_t st)
{
    k_batched_prefix<<<1, 1024, 0, st>>>(lens, count, batched_tile_elems(plan, dtype), prefix);
    int rc = check_launch("batched prefix kernel launch");
    if (rc != SINCOS_OK) return rc;
    if (dtype == SINCOS_F32)
        rc = launch_tiles_t<float>(segs, lens, count, prefix, red, coef, plan, dev, st);
    else if (dtype == SINCOS_BF16)
        rc = launch_tiles_t<__nv_bfloat16>(segs, lens, count, prefix, red, coef, plan, dev, st);
    else
        rc = launch_tiles_t<__half>(segs, lens, count, prefix, red, coef, plan, dev, st);
    return rc;
}

}  // namespace sincos_gb300
