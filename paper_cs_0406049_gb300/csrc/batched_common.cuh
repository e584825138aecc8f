// batched_common.cuh -- pieces shared by the two batched kernels: where a
// segment's vector grid starts, how it is cut into tiles, the tile at a given
// work offset, a CTA-wide scan, and the grid size.
#pragma once

#include "bulk.cuh"
#include "core.cuh"
#include "internal.h"
#include "seg_check.h"

namespace sincos_gb300 {

// Arrays skipped because their descriptor failed seg_usable, per translation
// unit (each batched TU reports its own; a read clears it).
static __device__ unsigned int g_bad_segments = 0;

// seg_usable for a descriptor of the batch's output type.
template <class OutT>
__device__ __forceinline__ bool seg_ok(const sincos_seg &d, int64_t len)
{
    return seg_usable(d.x, d.s, d.c, len, (unsigned)sizeof(OutT));
}

// Reads and clears this translation unit's skipped-array counter.
static inline unsigned take_bad_segments_here()
{
    unsigned v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_bad_segments, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaMemcpyToSymbol(g_bad_segments, &zero, sizeof zero);
    return v;
}

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

// First tile of a segment (len > 0 elements, grid start h, tile size T,
// ntiles tiles) that starts at or after cost r into the segment, a tile
// costing ce per element plus ct; ntiles if none does.  Tile 0 starts at 0,
// tile k >= 1 at element a + kT (a = max(h, 0)), after cost ce (a + kT) + ct k.
__device__ __forceinline__ int64_t first_tile_from(int64_t r, int h, int64_t tile,
                                                   int64_t ntiles, int64_t ce, int64_t ct)
{
    if (r <= 0) return 0;
    const int64_t a = h > 0 ? h : 0;
    const int64_t per = ce * tile + ct;
    const int64_t r1 = r - ce * a;
    int64_t k = r1 > 0 ? (r1 + per - 1) / per : 1;
    if (k < 1) k = 1;
    return k < ntiles ? k : ntiles;
}

// Inclusive scan of (a, b) over the CTA's threads in thread order; `wa`, `wb`
// are 32-entry shared arrays.  Returns the CTA totals in *ta, *tb.
__device__ __forceinline__ void cta_scan2(int64_t &a, int64_t &b, int64_t *wa, int64_t *wb,
                                          int64_t *ta, int64_t *tb)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, a, d);
        const int64_t v = __shfl_up_sync(0xffffffffu, b, d);
        if (lane >= d) {
            a += u;
            b += v;
        }
    }
    if (lane == 31) {
        wa[warp] = a;
        wb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        int64_t u = lane < nwarps ? wa[lane] : 0;
        int64_t v = lane < nwarps ? wb[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t pu = __shfl_up_sync(0xffffffffu, u, d);
            const int64_t pv = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) {
                u += pu;
                v += pv;
            }
        }
        wa[lane] = u;   // inclusive over warps
        wb[lane] = v;
    }
    __syncthreads();
    if (warp > 0) {
        a += wa[warp - 1];
        b += wb[warp - 1];
    }
    *ta = wa[nwarps - 1];
    *tb = wb[nwarps - 1];
    __syncthreads();
}

// CTAs of a batched tile kernel: all resident ones, at most kMaxBatchedCtas.
static inline int batched_grid(int per_sm, const DeviceInfo &dev)
{
    const int64_t g = (int64_t)per_sm * dev.sms;
    return (int)(g < kMaxBatchedCtas ? g : kMaxBatchedCtas);
}

}  // namespace sincos_gb300
