// batched.cuh -- the forward over many independent arrays, instantiated per
// output type by batched_f32.cu, batched_bf16.cu and batched_f16.cu.
//
// Element space.  Each array (segment) is cut into tiles of T elements laid
// on the segment's own vector grid (see seg_tiles; the last tile may be
// short).  Two kernels walk these tiles:
//
// * k_batched_ring (plans with vec_bytes 0, the default for binary32): one
//   launch.  Each CTA first computes its own run of tiles from the lengths
//   (ring_run), then a producer warp streams the run's angles through a TMA
//   ring of full stages to the consumer threads (see the ring section below).
//   T = kBulkChunk.  No scratch.
// * k_batched (register plans): a schedule kernel writes prefix[i] = number
//   of tiles in segments 0 .. i-1 into device scratch, and for each CTA its
//   first tile and that tile's segment, cutting the tiles into runs of equal
//   count (k_batched_prefix with ce = 0, ct = 1).  T = block * UNROLL * E,
//   E pairs per W-byte output vector.  The CTA walks forward from its first
//   segment (one comparison per tile, one extra load when it crosses into
//   the next segment); within a tile thread t owns vectors t, t + block, ...
//   exactly as in the single-array kernel.
//
// No CTA waits on another and no counter is shared between CTAs.
#pragma once

#include "batched_common.cuh"
#include "batched_ring.cuh"

namespace sincos_gb300 {

// The schedule of one batched launch over `grid` tile-kernel CTAs, by one CTA
// of 1024 threads, into sched = prefix[0 .. count], first_tile[0 .. grid],
// first_seg[0 .. grid]:
//   prefix[i] = tiles of segments 0 .. i-1 (seg_tiles with tile size T);
//   first_tile[b] = the first tile starting at or after cost floor(C b / grid)
//     of the concatenation, where a tile costs ce per element plus ct and C
//     is the total; the boundaries so cut the work into equal parts to within
//     a tile (ce = 0, ct = 1: equal tile counts);
//   first_seg[b] = the segment holding that point (the tile kernel walks
//     forward from it when the tile lies further on).
// Pass 1 sums the costs; pass 2 scans tiles and costs together, and each
// segment writes the boundaries whose point falls inside it.
template <class OutT, int W>
__global__ void k_batched_prefix(const sincos_seg *segs, const int64_t *lens, int count,
                                 int64_t tile, int grid, int64_t ce, int64_t ct, int64_t *sched)
{
    int64_t *prefix = sched;
    int64_t *first_tile = sched + count + 1;
    int64_t *first_seg = first_tile + grid + 1;
    __shared__ int64_t wa[32], wb[32];

    // An array whose descriptor fails seg_ok gets no tiles (it is skipped);
    // pass 2 counts it once.
    int64_t mine = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const sincos_seg d = segs[i];
        int64_t ne = lens[i] > 0 ? lens[i] : 0;
        if (!seg_ok<OutT>(d, ne)) ne = 0;
        mine += ce * ne + ct * seg_tiles(ne, seg_head<OutT, W>(d), tile);
    }
    int64_t zero = 0, all = 0, unused = 0;
    cta_scan2(mine, zero, wa, wb, &all, &unused);

    if (threadIdx.x == 0) prefix[0] = 0;
    int64_t carry_t = 0, carry_w = 0;
    for (int base = 0; base < count; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int64_t nt = 0, nw = 0;
        int h = -1;
        if (i < count) {
            const sincos_seg d = segs[i];
            int64_t ne = lens[i] > 0 ? lens[i] : 0;
            if (!seg_ok<OutT>(d, ne)) {
                atomicAdd(&g_bad_segments, 1u);
                ne = 0;
            }
            h = seg_head<OutT, W>(d);
            nt = seg_tiles(ne, h, tile);
            nw = ce * ne + ct * nt;
        }
        int64_t it = nt, iw = nw, tot_t = 0, tot_w = 0;
        cta_scan2(it, iw, wa, wb, &tot_t, &tot_w);
        const int64_t t0 = carry_t + it - nt;    // first tile of segment i
        const int64_t w0 = carry_w + iw - nw;    // cost before segment i
        if (i < count) {
            prefix[i + 1] = t0 + nt;
            if (nw > 0) {
                for (int64_t b = (w0 * grid + all - 1) / all; b < grid; ++b) {
                    const int64_t at = all * b / grid;
                    if (at >= w0 + nw) break;
                    first_tile[b] = t0 + first_tile_from(at - w0, h, tile, nt, ce, ct);
                    first_seg[b] = i;
                }
            }
        }
        carry_t += tot_t;
        carry_w += tot_w;
    }
    // The end of the last run; with no work at all every run is empty.
    for (int b = threadIdx.x; b <= grid; b += blockDim.x) {
        if (b == grid || all == 0) {
            first_tile[b] = carry_t;
            first_seg[b] = 0;
        }
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
__global__ void k_batched(const sincos_seg *segs, const int64_t *lens, const int64_t *sched,
                          int count)
{
    constexpr int E = Vec<OutT, W>::E;
    const int64_t tile = (int64_t)blockDim.x * UNROLL * E;
    const int64_t *prefix = sched;
    const int64_t *first_tile = sched + count + 1;
    const int64_t t0 = first_tile[blockIdx.x];
    const int64_t t1 = first_tile[blockIdx.x + 1];
    if (t0 >= t1) return;

    // A segment at or before tile t0's; the loop walks forward from it.
    int seg = (int)first_tile[gridDim.x + 1 + blockIdx.x];
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

// Both kernels of one batched launch for output type OutT.
template <class OutT>
int launch_batched_t(const sincos_seg *segs, const int64_t *lens, int count, int red, int coef,
                     int64_t *sched, const sincos_plan &plan, const DeviceInfo &dev,
                     cudaStream_t st)
{
    if (plan_vec_bytes(plan) == 0)
        return launch_batched_ring<OutT>(segs, lens, count, red, coef, sched, plan, dev, st);
    const void *fn = tiles_kernel_t<OutT>(red, coef, plan);
    if (!fn) return SINCOS_EINVAL;
    // The tile size follows the CTA size actually launched.
    int per_sm = 0;
    const sincos_plan p = fit_plan(fn, plan, &per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t tile = (int64_t)p.block * p.unroll * (reg_vec_bytes(p) / (int)sizeof(OutT));
    const int grid = batched_grid(per_sm, dev);
    if (reg_vec_bytes(p) == 32)
        k_batched_prefix<OutT, 32><<<1, 1024, 0, st>>>(segs, lens, count, tile, grid, 0, 1,
                                                       sched);
    else
        k_batched_prefix<OutT, 16><<<1, 1024, 0, st>>>(segs, lens, count, tile, grid, 0, 1,
                                                       sched);
    int rc = check_launch("batched schedule kernel launch");
    if (rc != SINCOS_OK) return rc;
    void *args[] = {(void *)&segs, (void *)&lens, (void *)&sched, (void *)&count};
    const cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((unsigned)p.block),
                                           args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "batched tile kernel launch");
    return check_launch("batched tile kernel launch");
}

}  // namespace sincos_gb300
