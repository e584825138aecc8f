// batched.cu -- the forward over many independent arrays in one launch pair.
//
// Element space.  Each array (segment) is cut into tiles of T = block *
// UNROLL * E elements, E pairs per W-byte output vector, laid on the
// segment's own vector grid (see seg_tiles; the last tile may be short).
// Tile numbers are global: a prefix kernel writes prefix[i] = number of tiles
// in segments 0 .. i-1 into device scratch, so segment i owns tiles
// [prefix[i], prefix[i+1]).
//
// Schedule.  The tile kernel is persistent: CTA b of G takes the contiguous
// run of tiles [total*b/G, total*(b+1)/G).  It finds the segment of its first
// tile by binary search over the prefix array once, then walks forward (one
// comparison per tile, one extra load when it crosses into the next
// segment), so the per-tile bookkeeping is register arithmetic except at
// segment changes.  Within a tile thread t owns vectors t, t + block, ...
// exactly as in the single-array kernel.  No CTA waits on another and no
// counter is shared, so nothing can spin.
#include "core.cuh"
#include "internal.h"

namespace sincos_gb300 {

// Where a segment's vector grid starts: the element h at which x, s and c
// all start a 128-byte line, or failing that are W-byte vector aligned, or -1
// when they admit no common alignment (then tiles start at multiples of T
// from element 0 and take the 16-byte or element-wise path).
template <class OutT, int W>
__device__ __forceinline__ int seg_head(const sincos_seg &d)
{
    return vector_head<OutT, W>(d.x, d.s, d.c);
}

// Tiles of a segment of length len with grid start h: tile 0 is the scalar
// head [0, h) plus the first T aligned elements, tile k >= 1 is
// [h + kT, h + (k+1)T) clipped to len.  So every tile boundary inside a
// segment falls on a vector boundary of all three arrays, and no 32-byte
// sector is written by two tiles except at the segment's own two ends.
__device__ __forceinline__ int64_t seg_tiles(int64_t len, int h, int64_t tile)
{
    if (len <= 0) return 0;
    const int64_t a = h > 0 ? h : 0;
    if (len <= a) return 1;
    return (len - a + tile - 1) / tile;
}

// prefix[0] = 0; prefix[i+1] = prefix[i] + seg_tiles(lens[i], head of segs[i]).
// One CTA of 1024 threads scans the segments 1024 at a time.
template <class OutT, int W>
__global__ void k_batched_prefix(const sincos_seg *segs, const int64_t *lens, int count,
                                 int64_t tile, int64_t *prefix)
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
        if (i < count) v = seg_tiles(lens[i], seg_head<OutT, W>(segs[i]), tile);
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

// Tile k of a segment whose three pointers share the vector grid starting at
// element h: vectors [h + kT, min(len, h + (k+1)T)), all UNROLL loads of a
// thread issued first; after them tile 0 also does the scalar head [0, h)
// and the last tile the scalar tail after its last whole vector.
template <class OutT, int RED, int COEF, int UNROLL, int W>
__device__ __forceinline__ void tile_aligned(const float *x, OutT *s, OutT *c, int64_t len,
                                             int h, int64_t k, int64_t tile)
{
    constexpr int E = Vec<OutT, W>::E;
    const int64_t v0 = h + k * tile;                    // first element of the vector run
    const int64_t end = len < v0 + tile ? len : v0 + tile;
    const int64_t nv = end > v0 ? (end - v0) / E : 0;
    const float *xv = x + v0;
    OutT *sv = s + v0;
    OutT *cv = c + v0;
    float in[UNROLL][E];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
        const int64_t j = threadIdx.x + (int64_t)u * blockDim.x;
        if (j < nv) load_vec<OutT, W, LD_NC>(in[u], xv + j * E);
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
        const int64_t j = threadIdx.x + (int64_t)u * blockDim.x;
        if (j < nv) compute_store<RED, COEF, OutT, W>(in[u], sv + j * E, cv + j * E);
    }
    if (k == 0) {
        const int64_t hh = h < len ? h : len;
        for (int64_t i = threadIdx.x; i < hh; i += blockDim.x)
            scalar_elem<RED, COEF>(x, s, c, i);
    }
    for (int64_t i = v0 + nv * E + threadIdx.x; i < end; i += blockDim.x)
        scalar_elem<RED, COEF>(x, s, c, i);
}

// Tile k of a segment with no common W-byte alignment: elements
// [kT, min(len, (k+1)T)) through 16-byte vectors if the pointers admit them,
// else element by element.
template <class OutT, int RED, int COEF>
__device__ __forceinline__ void tile_unaligned(const float *x, OutT *s, OutT *c, int64_t len,
                                               int64_t k, int64_t tile)
{
    constexpr int E16 = Vec<OutT, 16>::E;
    const int64_t e0 = k * tile;
    const int64_t m = len - e0 < tile ? len - e0 : tile;
    x += e0;
    s += e0;
    c += e0;
    int h16 = vector_head<OutT, 16>(x, s, c);
    if (h16 < 0) {
        for (int64_t i = threadIdx.x; i < m; i += blockDim.x)
            scalar_elem<RED, COEF>(x, s, c, i);
        return;
    }
    if (h16 > m) h16 = (int)m;
    const int64_t nv = (m - h16) / E16;
    for (int64_t j = threadIdx.x; j < nv; j += blockDim.x) {
        float in[E16];
        load_vec<OutT, 16, LD_NC>(in, x + h16 + j * E16);
        compute_store<RED, COEF, OutT, 16>(in, s + h16 + j * E16, c + h16 + j * E16);
    }
    if ((int)threadIdx.x < h16) scalar_elem<RED, COEF>(x, s, c, threadIdx.x);
    for (int64_t i = h16 + nv * E16 + threadIdx.x; i < m; i += blockDim.x)
        scalar_elem<RED, COEF>(x, s, c, i);
}

template <class OutT, int RED, int COEF, int UNROLL, int W>
__global__ void k_batched(const sincos_seg *segs, const int64_t *lens, const int64_t *prefix,
                          int count)
{
    constexpr int E = Vec<OutT, W>::E;
    const int64_t tile = (int64_t)blockDim.x * UNROLL * E;
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
    sincos_seg d = segs[seg];
    int64_t len = lens[seg];
    int h = seg_head<OutT, W>(d);
    for (int64_t t = t0; t < t1; ++t) {
        if (t >= seg_end) {
            do {                        // also skips empty segments
                ++seg;
                seg_first = seg_end;
                seg_end = prefix[seg + 1];
            } while (t >= seg_end);
            d = segs[seg];
            len = lens[seg];
            h = seg_head<OutT, W>(d);
        }
        if (h >= 0)
            tile_aligned<OutT, RED, COEF, UNROLL, W>(d.x, (OutT *)d.s, (OutT *)d.c, len, h,
                                                     t - seg_first, tile);
        else
            tile_unaligned<OutT, RED, COEF>(d.x, (OutT *)d.s, (OutT *)d.c, len, t - seg_first,
                                            tile);
    }
}

int64_t batched_tile_elems(const sincos_plan &plan, int dtype)
{
    return (int64_t)plan.block * plan.unroll * (reg_vec_bytes(plan) / dtype_size(dtype));
}

template <class OutT, int RED, int COEF, int W>
static const void *tiles_kernel_w(int unroll)
{
    switch (unroll) {
    case 1: return (const void *)k_batched<OutT, RED, COEF, 1, W>;
    case 2: return (const void *)k_batched<OutT, RED, COEF, 2, W>;
    case 4: return (const void *)k_batched<OutT, RED, COEF, 4, W>;
    case 8: return (const void *)k_batched<OutT, RED, COEF, 8, W>;
    default: return nullptr;
    }
}

template <class OutT, int RED, int COEF>
static const void *tiles_kernel_rc(const sincos_plan &plan)
{
    if (reg_vec_bytes(plan) == 32) return tiles_kernel_w<OutT, RED, COEF, 32>(plan.unroll);
    return tiles_kernel_w<OutT, RED, COEF, 16>(plan.unroll);
}

template <class OutT>
static const void *tiles_kernel_t(int red, int coef, const sincos_plan &plan)
{
    if (red == RED_PLAIN && coef == COEF_NORMALIZED)
        return tiles_kernel_rc<OutT, RED_PLAIN, COEF_NORMALIZED>(plan);
    if (red == RED_COMPENSATED && coef == COEF_NORMALIZED)
        return tiles_kernel_rc<OutT, RED_COMPENSATED, COEF_NORMALIZED>(plan);
    if (red == RED_PLAIN && coef == COEF_DAGGER)
        return tiles_kernel_rc<OutT, RED_PLAIN, COEF_DAGGER>(plan);
    return tiles_kernel_rc<OutT, RED_COMPENSATED, COEF_DAGGER>(plan);
}

int launch_batched(const sincos_seg *segs, const int64_t *lens, int count, int dtype, int red,
                   int coef, int64_t *prefix, const sincos_plan &plan, const DeviceInfo &dev,
                   cudaStream_t st)
{
    const void *fn = dtype == SINCOS_F32    ? tiles_kernel_t<float>(red, coef, plan)
                     : dtype == SINCOS_BF16 ? tiles_kernel_t<__nv_bfloat16>(red, coef, plan)
                                            : tiles_kernel_t<__half>(red, coef, plan);
    if (!fn) return SINCOS_EINVAL;
    // The tile size follows the CTA size actually launched.
    int per_sm = 0;
    const sincos_plan p = fit_plan(fn, plan, &per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t tile = batched_tile_elems(p, dtype);
    const bool w32 = reg_vec_bytes(p) == 32;
    if (dtype == SINCOS_F32)
        (w32 ? k_batched_prefix<float, 32> : k_batched_prefix<float, 16>)
            <<<1, 1024, 0, st>>>(segs, lens, count, tile, prefix);
    else if (dtype == SINCOS_BF16)
        (w32 ? k_batched_prefix<__nv_bfloat16, 32> : k_batched_prefix<__nv_bfloat16, 16>)
            <<<1, 1024, 0, st>>>(segs, lens, count, tile, prefix);
    else
        (w32 ? k_batched_prefix<__half, 32> : k_batched_prefix<__half, 16>)
            <<<1, 1024, 0, st>>>(segs, lens, count, tile, prefix);
    int rc = check_launch("batched prefix kernel launch");
    if (rc != SINCOS_OK) return rc;
    void *args[] = {(void *)&segs, (void *)&lens, (void *)&prefix, (void *)&count};
    const cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)per_sm * (unsigned)dev.sms),
                                           dim3((unsigned)p.block), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "batched tile kernel launch");
    return check_launch("batched tile kernel launch");
}

}  // namespace sincos_gb300
