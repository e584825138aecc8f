// batched.cuh -- the forward over many independent arrays in one launch pair,
// instantiated per output type by batched_f32.cu, batched_bf16.cu and
// batched_f16.cu.
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
#pragma once

#include "bulk.cuh"
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

// ---------------------------------------------------------------------------
// Bulk (TMA-staged) variant: the same tiles with T = kBulkChunk, each tile's
// 16-byte-aligned middle moved through a two-stage shared-memory ring by bulk
// copies and written back by bulk stores; heads, tails and segments without
// a common 16-byte alignment are done directly from global memory.  Thread 0
// walks the tile run two tiles ahead of the others to issue the loads.
// ---------------------------------------------------------------------------

// Position of a walk over a CTA's contiguous tile run.
struct TileWalk {
    int seg;
    int64_t seg_first, seg_end, len;
    sincos_seg d;
    int h;
};

template <class OutT>
__device__ __forceinline__ void walk_start(TileWalk &w, const sincos_seg *segs,
                                           const int64_t *lens, const int64_t *prefix, int count,
                                           int64_t t)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    w.seg = lo;
    w.seg_first = prefix[lo];
    w.seg_end = prefix[lo + 1];
    w.d = segs[lo];
    w.len = lens[lo];
    w.h = seg_head<OutT, 16>(w.d);
}

template <class OutT>
__device__ __forceinline__ void walk_to(TileWalk &w, const sincos_seg *segs, const int64_t *lens,
                                        const int64_t *prefix, int64_t t)
{
    if (t < w.seg_end) return;
    do {
        ++w.seg;
        w.seg_first = w.seg_end;
        w.seg_end = prefix[w.seg + 1];
    } while (t >= w.seg_end);
    w.d = segs[w.seg];
    w.len = lens[w.seg];
    w.h = seg_head<OutT, 16>(w.d);
}

// The bulk-copied part of tile t of the walk's segment: angles
// [v0, v0 + mb), mb a multiple of the 16-byte vector (0 if none).
template <class OutT>
__device__ __forceinline__ void tile_bulk_part(const TileWalk &w, int64_t t, int64_t *v0,
                                               int64_t *mb)
{
    constexpr int E = Vec<OutT, 16>::E;
    if (w.h < 0) {
        *v0 = 0;
        *mb = 0;
        return;
    }
    const int64_t start = w.h + (t - w.seg_first) * kBulkChunk;
    const int64_t end = w.len < start + kBulkChunk ? w.len : start + kBulkChunk;
    *v0 = start;
    *mb = end > start ? (end - start) / E * E : 0;
}

// Tiles whose bulk part is at least this many angles go through the TMA
// ring; smaller ones (mostly the short last tile of a segment, and short
// segments) are done straight from global memory, so a nearly empty tile
// never holds one of the two ring stages.
constexpr int64_t kBulkMinAngles = kBulkChunk / 4;

// Pairs of the E angles at element e of a staged input tile into the staged
// output tiles (16-byte shared-memory accesses).
template <int RED, int COEF, class OutT>
__device__ __forceinline__ void bulk_tile_vec(const float *xi, OutT *so, OutT *co, int e)
{
    constexpr int E = Vec<OutT, 16>::E;
    float in[E];
#pragma unroll
    for (int q = 0; q < E; q += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(xi + e + q);
        in[q] = v.x;
        in[q + 1] = v.y;
        in[q + 2] = v.z;
        in[q + 3] = v.w;
    }
    float sv[E], cv[E];
#pragma unroll
    for (int i = 0; i < E; ++i) pair<RED, COEF>(in[i], sv[i], cv[i]);
    uint32_t ws[4], wc[4];
    if constexpr (sizeof(OutT) == 4) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ws[i] = __float_as_uint(sv[i]);
            wc[i] = __float_as_uint(cv[i]);
        }
    } else {
        OutT *tag = nullptr;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ws[i] = pack2(tag, sv[2 * i], sv[2 * i + 1]);
            wc[i] = pack2(tag, cv[2 * i], cv[2 * i + 1]);
        }
    }
    *reinterpret_cast<uint4 *>(so + e) = make_uint4(ws[0], ws[1], ws[2], ws[3]);
    *reinterpret_cast<uint4 *>(co + e) = make_uint4(wc[0], wc[1], wc[2], wc[3]);
}

// Thread 0: find the next ring-worthy tile at or after *tp (advancing the
// producer walk) and start its bulk load into `dst`; false if none is left.
template <class OutT>
__device__ __forceinline__ bool issue_next_bulk_tile(TileWalk &pw, int64_t *tp, int64_t t1,
                                                     const sincos_seg *segs, const int64_t *lens,
                                                     const int64_t *prefix, float *dst,
                                                     uint32_t bar)
{
    while (*tp < t1) {
        const int64_t t = (*tp)++;
        walk_to<OutT>(pw, segs, lens, prefix, t);
        int64_t v0, mb;
        tile_bulk_part<OutT>(pw, t, &v0, &mb);
        if (mb >= kBulkMinAngles) {
            bulk_load(dst, pw.d.x + v0, (uint32_t)(mb * 4), bar);
            return true;
        }
    }
    return false;
}

// The pairs of angles [v0, v0 + m) of one segment, 16-byte vectors straight
// from global memory (v0 is on the segment's 16-byte grid), then the scalar
// remainder.
template <class OutT, int RED, int COEF, int NT>
__device__ __forceinline__ void direct_run(const float *x, OutT *s, OutT *c, int64_t v0,
                                           int64_t m)
{
    constexpr int E = Vec<OutT, 16>::E;
    const int64_t nv = m / E;
    for (int64_t j = threadIdx.x; j < nv; j += NT) {
        float in[E];
        load_vec<OutT, 16, LD_NC>(in, x + v0 + j * E);
        compute_store<RED, COEF, OutT, 16>(in, s + v0 + j * E, c + v0 + j * E);
    }
    for (int64_t i = v0 + nv * E + threadIdx.x; i < v0 + m; i += NT)
        scalar_elem<RED, COEF>(x, s, c, i);
}

template <class OutT, int RED, int COEF, int NT>
__global__ void __launch_bounds__(NT)
k_batched_bulk(const sincos_seg *segs, const int64_t *lens, const int64_t *prefix, int count)
{
    constexpr int E = Vec<OutT, 16>::E;
    extern __shared__ __align__(128) unsigned char smem[];
    float *xin = (float *)smem;                                        // [stages][chunk]
    OutT *sout = (OutT *)(xin + kBulkStages * kBulkChunk);              // [2][chunk]
    OutT *cout = sout + 2 * kBulkChunk;                                 // [2][chunk]
    __shared__ __align__(8) uint64_t full[kBulkStages];
    __shared__ int64_t issued[kBulkStages];
    __shared__ int give_up;

    const int64_t total = prefix[count];
    const int64_t t0 = total * blockIdx.x / gridDim.x;
    const int64_t t1 = total * (blockIdx.x + 1) / gridDim.x;
    if (t0 >= t1) return;
    const int tid = threadIdx.x;
    if (tid == 0) {
        give_up = 0;
        for (int i = 0; i < kBulkStages; ++i) {
            issued[i] = 0;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&full[i]))
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    TileWalk cw, pw;                      // consumer (all threads), producer (thread 0)
    int64_t tp = t0;                      // producer: next tile to examine
    walk_start<OutT>(cw, segs, lens, prefix, count, t0);
    if (tid == 0) {
        pw = cw;
        for (int st = 0; st < kBulkStages; ++st)
            if (issue_next_bulk_tile<OutT>(pw, &tp, t1, segs, lens, prefix,
                                           xin + st * kBulkChunk, smem_addr(&full[st])))
                issued[st] += 1;
    }

    int64_t kb = 0;                       // ring tiles consumed so far
    for (int64_t t = t0; t < t1; ++t) {
        walk_to<OutT>(cw, segs, lens, prefix, t);
        const float *xs = cw.d.x;
        OutT *ss = (OutT *)cw.d.s;
        OutT *cs = (OutT *)cw.d.c;
        if (cw.h < 0) {                   // no common 16-byte grid
            tile_unaligned<OutT, RED, COEF>(xs, ss, cs, cw.len, t - cw.seg_first, kBulkChunk);
            continue;
        }
        int64_t v0, mb;
        tile_bulk_part<OutT>(cw, t, &v0, &mb);
        if (t == cw.seg_first) {          // the segment's scalar head
            const int64_t hh = cw.h < cw.len ? cw.h : cw.len;
            for (int64_t i = tid; i < hh; i += NT) scalar_elem<RED, COEF>(xs, ss, cs, i);
        }
        const int64_t end = cw.len < v0 + kBulkChunk ? cw.len : v0 + kBulkChunk;
        if (mb < kBulkMinAngles) {        // short tile: straight from global memory
            if (end > v0) direct_run<OutT, RED, COEF, NT>(xs, ss, cs, v0, end - v0);
            continue;
        }
        const int st = (int)(kb % kBulkStages);
        if (!mbar_wait_bounded(smem_addr(&full[st]), (uint32_t)((kb / kBulkStages) & 1))) {
            atomicAdd(&g_bulk_wait_timeouts, 1u);
            give_up = 1;
        }
        const int b = (int)(kb & 1);
        if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncthreads();
        if (give_up) break;
        const float *xi = xin + st * kBulkChunk;
        OutT *so = sout + b * kBulkChunk;
        OutT *co = cout + b * kBulkChunk;
        if (mb == kBulkChunk) {           // a whole tile: fixed, fully unrolled trip count
#pragma unroll
            for (int j = 0; j < kBulkChunk / (NT * E); ++j)
                bulk_tile_vec<RED, COEF, OutT>(xi, so, co, (j * NT + tid) * E);
        } else {
#pragma unroll 2
            for (int64_t e = (int64_t)tid * E; e < mb; e += (int64_t)NT * E)
                bulk_tile_vec<RED, COEF, OutT>(xi, so, co, (int)e);
        }
        for (int64_t i = v0 + mb + tid; i < end; i += NT) scalar_elem<RED, COEF>(xs, ss, cs, i);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            bulk_store(ss + v0, so, (uint32_t)(mb * sizeof(OutT)));
            bulk_store(cs + v0, co, (uint32_t)(mb * sizeof(OutT)));
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            if (issue_next_bulk_tile<OutT>(pw, &tp, t1, segs, lens, prefix,
                                           xin + st * kBulkChunk, smem_addr(&full[st])))
                issued[st] += 1;
        }
        ++kb;
    }
    if (give_up && tid == 0) {
        for (int st = 0; st < kBulkStages; ++st) {
            const int64_t consumed = kb / kBulkStages + ((kb % kBulkStages) > st ? 1 : 0);
            for (int64_t j = consumed; j < issued[st]; ++j)
                mbar_wait_bounded(smem_addr(&full[st]), (uint32_t)(j & 1));
        }
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

template <class OutT, int RED, int COEF>
static const void *bulk_tiles_kernel_rc(int block)
{
    switch (block) {
    case 128: return (const void *)k_batched_bulk<OutT, RED, COEF, 128>;
    case 512: return (const void *)k_batched_bulk<OutT, RED, COEF, 512>;
    case 1024: return (const void *)k_batched_bulk<OutT, RED, COEF, 1024>;
    default: return (const void *)k_batched_bulk<OutT, RED, COEF, 256>;
    }
}

template <class OutT>
static const void *bulk_tiles_kernel_t(int red, int coef, int block)
{
    if (red == RED_PLAIN && coef == COEF_NORMALIZED)
        return bulk_tiles_kernel_rc<OutT, RED_PLAIN, COEF_NORMALIZED>(block);
    if (red == RED_COMPENSATED && coef == COEF_NORMALIZED)
        return bulk_tiles_kernel_rc<OutT, RED_COMPENSATED, COEF_NORMALIZED>(block);
    if (red == RED_PLAIN && coef == COEF_DAGGER)
        return bulk_tiles_kernel_rc<OutT, RED_PLAIN, COEF_DAGGER>(block);
    return bulk_tiles_kernel_rc<OutT, RED_COMPENSATED, COEF_DAGGER>(block);
}

template <class OutT>
static int launch_batched_bulk(const sincos_seg *segs, const int64_t *lens, int count, int red,
                               int coef, int64_t *prefix, const sincos_plan &plan,
                               const DeviceInfo &dev, cudaStream_t st)
{
    const void *fn = bulk_tiles_kernel_t<OutT>(red, coef, plan.block);
    const int block = (plan.block == 128 || plan.block == 512 || plan.block == 1024) ? plan.block
                                                                                       : 256;
    constexpr size_t smem = bulk_smem_bytes<OutT>();
    const int per_sm = bulk_resident_ctas(fn, block, smem);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    k_batched_prefix<OutT, 16><<<1, 1024, 0, st>>>(segs, lens, count, kBulkChunk, prefix);
    int rc = check_launch("batched prefix kernel launch");
    if (rc != SINCOS_OK) return rc;
    void *args[] = {(void *)&segs, (void *)&lens, (void *)&prefix, (void *)&count};
    const cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)per_sm * (unsigned)dev.sms),
                                           dim3((unsigned)block), args, smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "batched bulk kernel launch");
    return check_launch("batched bulk kernel launch");
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
                     int64_t *prefix, const sincos_plan &plan, const DeviceInfo &dev,
                     cudaStream_t st)
{
    if (plan_vec_bytes(plan) == 0)
        return launch_batched_bulk<OutT>(segs, lens, count, red, coef, prefix, plan, dev, st);
    const void *fn = tiles_kernel_t<OutT>(red, coef, plan);
    if (!fn) return SINCOS_EINVAL;
    // The tile size follows the CTA size actually launched.
    int per_sm = 0;
    const sincos_plan p = fit_plan(fn, plan, &per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t tile = (int64_t)p.block * p.unroll * (reg_vec_bytes(p) / (int)sizeof(OutT));
    if (reg_vec_bytes(p) == 32)
        k_batched_prefix<OutT, 32><<<1, 1024, 0, st>>>(segs, lens, count, tile, prefix);
    else
        k_batched_prefix<OutT, 16><<<1, 1024, 0, st>>>(segs, lens, count, tile, prefix);
    int rc = check_launch("batched prefix kernel launch");
    if (rc != SINCOS_OK) return rc;
    void *args[] = {(void *)&segs, (void *)&lens, (void *)&prefix, (void *)&count};
    const cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)per_sm * (unsigned)dev.sms),
                                           dim3((unsigned)p.block), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "batched tile kernel launch");
    return check_launch("batched tile kernel launch");
}

}  // namespace sincos_gb300
