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

    int64_t mine = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const int64_t ne = lens[i] > 0 ? lens[i] : 0;
        mine += ce * ne + ct * seg_tiles(ne, seg_head<OutT, W>(segs[i]), tile);
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
            const int64_t ne = lens[i] > 0 ? lens[i] : 0;
            h = seg_head<OutT, W>(segs[i]);
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

// ---------------------------------------------------------------------------
// Ring (TMA-staged) variant: NT consumer threads and one producer warp.
//
// The producer warp walks the CTA's tile run (tile size T = kBulkChunk) with
// the metadata of 32 segments at a time in its lanes (one load per lane for
// 32 segments, then register shuffles).  It streams the run's elements, one
// element range per segment, through a ring of kRingStages input stages of
// kRingCap angles.  Each stage is filled to capacity: it takes the rest of
// one range and the start of the next ("parts", up to kRingMaxParts), and a
// range that does not fit is split on a 32-angle boundary of its vector
// grid.  So the ring carries full stages however the arrays are sized, as in
// the single-array kernel, and a short array costs a descriptor, not a
// round trip.  Of each part the producer bulk-copies the middle (the angles
// from the segment's vector grid on, or from the first 16-byte boundary of
// x when x, s and c share no grid, a whole number of vectors) into the
// stage.  The few angles before and after the middle ("edges": the scalar
// head up to the segment's line boundary, a tail shorter than one vector)
// the consumers load from global memory at the start of the stage, so that
// latency overlaps the stage's main work.  Consumers write the pairs of a
// middle on the shared grid into an output stage that consumer thread 0
// bulk-stores; the other pairs go straight to global memory.  Consumers
// never read segment metadata.
//
// Synchronization: per stage, full[st] (the producer arrives after arming it
// with the stage's byte count) and empty[st] (every consumer arrives once it
// has read the stage's input); descriptor slots that outlive their stage by
// one round (see kRingSlots); a named barrier among the consumers; bulk-store
// groups for the two output stages.  Every
// wait is bounded.  A wait that gives up counts a timeout and stops its side;
// the producer then waits (bounded) for every copy it issued before the CTA
// may exit.
// ---------------------------------------------------------------------------

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

constexpr int kRingStages = 2;
constexpr int kRingCap = kBulkChunk;           // angles per stage
constexpr int kRingMaxParts = 32;              // parts per stage
// Descriptor slots: the producer builds the parts of stage k in slot
// k % kRingSlots while stage k - kRingStages is still being consumed, so once
// that stage is released it only has to start the copies.
constexpr int kRingSlots = 2 * kRingStages;

// Cost of a tile in the schedule of the ring kernel, in angles on top of its
// angles: a part's descriptor, its edges and its bulk store.
constexpr int64_t kRingTileCost = 1024;

struct RingPart {
    const float *x;        // angle of the part's first element (lo)
    void *s;               // outputs of element lo
    void *c;
    int n;                 // elements [lo, lo + n)
    int u0, u1;            // middle [lo + u0, lo + u1), bulk-copied
    int in_off;            // stage index of element lo + u0
    int out_off;           // output-stage index of element lo + u0, -1: stored directly
    int edge0;             // index of the part's first edge within the stage
};

template <class OutT>
constexpr size_t ring_smem_bytes()
{
    return (size_t)kRingStages * kRingCap * 4 + 2 * 2 * (size_t)kRingCap * sizeof(OutT);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;"
                 :: "r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_copy_in(void *dst_smem, const void *src, uint32_t bytes,
                                             uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst_smem)), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ void consumer_sync(int nt)
{
    asm volatile("bar.sync 1, %0;" :: "r"(nt) : "memory");
}

// Metadata of segment `seg` in one producer lane (an empty slot past count).
struct SegMeta {
    const float *x;
    void *s;
    void *c;
    int64_t len, nt;
    int h;
};

template <class OutT>
__device__ __forceinline__ SegMeta load_seg_meta(const sincos_seg *segs, const int64_t *lens,
                                                 int count, int64_t seg)
{
    SegMeta m;
    if (seg < count) {
        const sincos_seg d = segs[seg];
        m.x = d.x;
        m.s = d.s;
        m.c = d.c;
        m.len = lens[seg] > 0 ? lens[seg] : 0;
        m.h = seg_head<OutT, 16>(d);
        m.nt = seg_tiles(m.len, m.h, kBulkChunk);
    } else {
        m.x = nullptr;
        m.s = m.c = nullptr;
        m.len = m.nt = 0;
        m.h = -1;
    }
    return m;
}

// This CTA's share of the batch, as positions (segment, tile of that
// segment): it runs from (seg_a, k_a) up to, not including, (seg_b, k_b).
struct RingRun {
    int64_t seg_a, k_a, seg_b, k_b;
};

// Chunks of blockDim.x segments that ring_run sums at a time, and the chunk
// totals it keeps in shared memory for its second pass.
constexpr int kRunBatch = 8;
constexpr int kRunChunks = 128;

// Work of a segment of length len in the ring schedule: its angles plus
// kRingTileCost per tile, counting ceil(len / T) tiles.  (Its exact tile count
// also depends on the grid start; the schedule only needs a cost that every
// CTA computes the same way from the lengths alone.)
__device__ __forceinline__ int64_t ring_len_cost(int64_t len)
{
    const int64_t ne = len > 0 ? len : 0;
    return ne + kRingTileCost * ((ne + kBulkChunk - 1) / kBulkChunk);
}

// Work of the segments of chunks [c0, c0 + kRunBatch) that belong to this
// thread (segment (c0 + q) * P + tid in slot q); consecutive threads read
// consecutive lengths, so the loads coalesce.
__device__ __forceinline__ void ring_load_costs(const int64_t *lens, int count, int c0,
                                                int64_t *bw)
{
    const int64_t P = blockDim.x;
    int64_t len[kRunBatch];
#pragma unroll
    for (int q = 0; q < kRunBatch; ++q) {
        const int64_t i = (c0 + q) * P + threadIdx.x;
        len[q] = i < count ? lens[i] : 0;
    }
#pragma unroll
    for (int q = 0; q < kRunBatch; ++q) bw[q] = ring_len_cost(len[q]);
}

// Sums over the CTA of v[0 .. kRunBatch), into tot[] (shared, kRunBatch).
__device__ __forceinline__ void cta_sums(const int64_t *v, int64_t (*red)[32], int64_t *tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < kRunBatch; ++q) {
        int64_t x = v[q];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
        if (lane == 0) red[q][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < kRunBatch; ++q) {
            int64_t x = lane < nwarps ? red[q][lane] : 0;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
            if (lane == 0) tot[q] = x;
        }
    }
    __syncthreads();
}

// Locate work position `at` inside chunk c whose work starts at `base`: a CTA
// scan of the chunk's costs; the thread whose segment holds the position
// writes (segment, first tile starting at or after it) to *seg, *k.
template <class OutT>
__device__ __forceinline__ void ring_locate(const sincos_seg *segs, const int64_t *lens,
                                            int count, int c, int64_t base, int64_t at,
                                            int64_t *seg, int64_t *k, int64_t *wa, int64_t *wb)
{
    const int64_t i = (int64_t)c * blockDim.x + threadIdx.x;
    const int64_t len = i < count ? (lens[i] > 0 ? lens[i] : 0) : 0;
    const int64_t w = ring_len_cost(len);
    int64_t incl = w, zero = 0, t1 = 0, t2 = 0;
    cta_scan2(incl, zero, wa, wb, &t1, &t2);
    const int64_t from = base + incl - w;
    if (w > 0 && at >= from && at < from + w) {
        const int h = seg_head<OutT, 16>(segs[i]);
        *seg = i;
        *k = first_tile_from(at - from, h, kBulkChunk, seg_tiles(len, h, kBulkChunk), 1,
                             kRingTileCost);
    }
}

// The CTA computes its own run, with all its threads.  The batch's work W is
// summed over the lengths; CTA b of G then takes the tiles from the first one
// starting at or after work floor(W b / G) to the first one starting at or
// after floor(W (b+1) / G).  CTAs b and b + 1 compute the same boundary, so
// the runs tile the batch.  Lengths are read in chunks of blockDim.x,
// consecutive threads on consecutive segments; the chunk totals stay in shared
// memory (up to kRunChunks chunks, else they are summed again), and only the
// chunks holding the two boundaries are scanned.
template <class OutT>
__device__ __forceinline__ void ring_run(const sincos_seg *segs, const int64_t *lens, int count,
                                         RingRun *run, int64_t *wa, int64_t *wb,
                                         int64_t (*red)[32], int64_t *tot, int64_t *ctot)
{
    const int P = (int)blockDim.x;
    const int nchunks = (count + P - 1) / P;
    int64_t bw[kRunBatch];
    if (threadIdx.x == 0) {
        run->seg_a = run->seg_b = count;
        run->k_a = run->k_b = 0;
    }
    int64_t all = 0;
    for (int c0 = 0; c0 < nchunks; c0 += kRunBatch) {
        ring_load_costs(lens, count, c0, bw);
        cta_sums(bw, red, tot);
#pragma unroll
        for (int q = 0; q < kRunBatch; ++q) {
            if (threadIdx.x == 0 && c0 + q < kRunChunks) ctot[c0 + q] = tot[q];
            all += tot[q];
        }
    }
    __syncthreads();
    const int64_t lo = all * (int64_t)blockIdx.x / gridDim.x;
    const int64_t hi = all * ((int64_t)blockIdx.x + 1) / gridDim.x;
    int64_t base = 0;
    for (int c0 = 0; c0 < nchunks && base <= hi; c0 += kRunBatch) {
        if (nchunks > kRunChunks) {                  // totals not kept: sum this batch again
            ring_load_costs(lens, count, c0, bw);
            cta_sums(bw, red, tot);
        }
        for (int q = 0; q < kRunBatch && c0 + q < nchunks; ++q) {
            const int64_t ct = nchunks > kRunChunks ? tot[q] : ctot[c0 + q];
            if (lo >= base && lo < base + ct)        // uniform over the CTA
                ring_locate<OutT>(segs, lens, count, c0 + q, base, lo, &run->seg_a, &run->k_a,
                                  wa, wb);
            if (hi >= base && hi < base + ct)
                ring_locate<OutT>(segs, lens, count, c0 + q, base, hi, &run->seg_b, &run->k_b,
                                  wa, wb);
            base += ct;
        }
    }
    __syncthreads();
}

template <class T>
__device__ __forceinline__ T *shfl_ptr(T *p, int src)
{
    return (T *)__shfl_sync(0xffffffffu, (unsigned long long)p, src);
}

// First element of tile k of a segment (grid start h; tile 0 starts at 0).
__device__ __forceinline__ int64_t ring_tile_lo(int64_t k, int h)
{
    if (k == 0) return 0;
    return (h > 0 ? h : 0) + k * (int64_t)kBulkChunk;
}

// Producer warp: stream the elements of the CTA's run through the ring.
// The run's tiles of one segment form one element range; ranges are cut into
// parts that fill each stage to kRingCap angles (a range that does not fit is
// split on a 32-angle boundary of its grid), so every stage but the last
// carries a full load however the segments are sized.
template <class OutT, int NT>
__device__ __forceinline__ void ring_producer(const sincos_seg *segs, const int64_t *lens,
                                              int count, const RingRun run, float *xin,
                                              RingPart (*parts)[kRingMaxParts], int *nparts,
                                              int *nedges, int *nmid, int *nout, uint64_t *full,
                                              uint64_t *empty, volatile int *give_up)
{
    constexpr int E = Vec<OutT, 16>::E;
    constexpr int64_t kSplit = 32;                 // split granularity (angles)
    const int lane = threadIdx.x & 31;
    int64_t base = run.seg_a;
    SegMeta w = load_seg_meta<OutT>(segs, lens, count, base + lane);
    int64_t seg = run.seg_a, kt = run.k_a;         // next tile position
    // the current range: elements [pos, rhi) of segment (x, so, co) with grid start h
    const float *x = nullptr;
    OutT *so = nullptr, *co = nullptr;
    int64_t pos = 0, rhi = 0;
    int h = -1;
    bool have = false;
    uint32_t k = 0;
    for (;;) {
        const int st = (int)(k % kRingStages);
        const int slot = (int)(k % kRingSlots);
        // 1. the parts of stage k, into descriptor slot k % kRingSlots
        int n = 0, cap = 0, outc = 0, edges = 0;
        while (n < kRingMaxParts) {
            if (!have) {
                // the next segment with tiles of this run left
                int64_t kend = 0, len = 0, nt = 0;
                bool found = false;
                while (seg < run.seg_b || (seg == run.seg_b && kt < run.k_b)) {
                    while (seg - base >= 32) {
                        base += 32;
                        w = load_seg_meta<OutT>(segs, lens, count, base + lane);
                    }
                    const int c = (int)(seg - base);
                    nt = __shfl_sync(0xffffffffu, w.nt, c);
                    kend = seg == run.seg_b ? run.k_b : nt;
                    if (kt < kend) {
                        x = shfl_ptr(w.x, c);
                        so = shfl_ptr((OutT *)w.s, c);
                        co = shfl_ptr((OutT *)w.c, c);
                        len = __shfl_sync(0xffffffffu, w.len, c);
                        h = __shfl_sync(0xffffffffu, w.h, c);
                        found = true;
                        break;
                    }
                    ++seg;
                    kt = 0;
                }
                if (!found) break;
                pos = ring_tile_lo(kt, h);
                rhi = kend >= nt ? len : ring_tile_lo(kend, h);
                if (rhi > len) rhi = len;
                if (h >= 0 && len <= h) h = -2;                 // no middle at all
                ++seg;                                          // this segment's run is taken
                kt = 0;
                have = true;
            }
            // the part's middle [u0, u1) and end hi
            int64_t u0;
            if (h >= 0) u0 = pos < h ? h : pos;
            else if (h == -1) u0 = pos + (((4u - ((unsigned)((uintptr_t)(x + pos) & 15u) >> 2)) & 3u));
            else u0 = rhi;
            if (u0 > rhi) u0 = rhi;
            const int64_t avail = kRingCap - cap;
            int64_t u1 = u0 + (rhi - u0) / E * E, hi = rhi;
            if (u1 - u0 > avail) {
                const int64_t take = avail / kSplit * kSplit;
                if (take < kSplit) break;                      // stage full
                u1 = u0 + take;
                hi = u1;
            }
            const int need = (int)(u1 - u0);
            const bool grid = h >= 0;
            if (lane == 0) {
                RingPart &p = parts[slot][n];
                p.x = x + pos;
                p.s = so + pos;
                p.c = co + pos;
                p.n = (int)(hi - pos);
                p.u0 = (int)(u0 - pos);
                p.u1 = (int)(u1 - pos);
                p.in_off = cap;
                p.out_off = grid ? outc : -1;
                p.edge0 = edges;
            }
            cap += need;
            if (grid) outc += need;
            edges += (int)((u0 - pos) + (hi - u1));
            ++n;
            pos = hi;
            if (hi == rhi) have = false;
        }
        // 2. wait until every consumer has read stage k - kRingStages
        if (k >= (uint32_t)kRingStages) {
            bool ok = true;
            if (lane == 0) {
                ok = mbar_wait_bounded(smem_addr(&empty[st]), ((k / kRingStages) - 1) & 1);
                if (!ok) {
                    atomicAdd(&g_bulk_wait_timeouts, 1u);
                    *give_up = 1;
                }
            }
            ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
            if (!ok || *give_up) break;
        }
        // 3. start the copies and publish the stage
        if (lane == 0) {
            const uint32_t bar = smem_addr(&full[st]);
            if (cap > 0) mbar_expect_tx(bar, (uint32_t)cap * 4u);
            float *dst = xin + (size_t)st * kRingCap;
            for (int i = 0; i < n; ++i) {
                const RingPart &p = parts[slot][i];
                const int need = p.u1 - p.u0;
                if (need > 0) bulk_copy_in(dst + p.in_off, p.x + p.u0, (uint32_t)need * 4u, bar);
            }
            nparts[slot] = n > 0 ? n : -1;
            nedges[slot] = edges;
            nmid[slot] = cap;
            nout[slot] = outc;
            mbar_arrive(bar);
        }
        __syncwarp();
        ++k;
        if (n == 0) break;
    }
    // Every copy issued must land before the CTA exits: wait (bounded) for the
    // last phase armed on each stage.
    if (lane == 0) {
        for (uint32_t j = k > (uint32_t)kRingStages ? k - kRingStages : 0; j < k; ++j)
            mbar_wait_bounded(smem_addr(&full[j % kRingStages]), (j / kRingStages) & 1);
    }
}

template <class OutT, int RED, int COEF, int NT>
__global__ void __launch_bounds__(NT + 32)
k_batched_ring(const sincos_seg *segs, const int64_t *lens, int count)
{
    constexpr int E = Vec<OutT, 16>::E;
    constexpr int kEdgeRegs = 4;
    extern __shared__ __align__(128) unsigned char smem[];
    float *xin = (float *)smem;                                        // [stages][cap]
    OutT *sout = (OutT *)(xin + kRingStages * kRingCap);                // [2][cap]
    OutT *cout = sout + 2 * kRingCap;                                   // [2][cap]
    __shared__ RingPart parts[kRingSlots][kRingMaxParts];
    __shared__ int nparts[kRingSlots], nedges[kRingSlots], nmid[kRingSlots], nout[kRingSlots];
    __shared__ __align__(8) uint64_t full[kRingStages], empty[kRingStages];
    __shared__ int give_up;
    __shared__ RingRun run;
    __shared__ int64_t wa[32], wb[32];
    __shared__ int64_t red[kRunBatch][32], tot[kRunBatch], ctot[kRunChunks];

    ring_run<OutT>(segs, lens, count, &run, wa, wb, red, tot, ctot);
    const int tid = threadIdx.x;
    if (tid == 0) {
        give_up = 0;
        for (int i = 0; i < kRingStages; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&full[i]))
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                         :: "r"(smem_addr(&empty[i])), "r"(NT) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (tid >= NT) {
        ring_producer<OutT, NT>(segs, lens, count, run, xin, parts, nparts, nedges, nmid, nout,
                                full, empty, &give_up);
        return;
    }

    for (uint32_t k = 0;; ++k) {
        const int st = (int)(k % kRingStages);
        const int slot = (int)(k % kRingSlots);
        if (!mbar_wait_bounded(smem_addr(&full[st]), (k / kRingStages) & 1)) {
            atomicAdd(&g_bulk_wait_timeouts, 1u);
            give_up = 1;
        }
        const int b = (int)(k & 1);
        // The bulk stores that last read output stage b (two stages ago) must
        // be done reading it before it is overwritten.
        if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        consumer_sync(NT);
        if (*(volatile int *)&give_up) break;
        const int n = nparts[slot];
        if (n < 0) break;
        const RingPart *pp = parts[slot];
        const float *xs = xin + (size_t)st * kRingCap;
        OutT *so = sout + (size_t)b * kRingCap;
        OutT *co = cout + (size_t)b * kRingCap;

        // Edges: issue the first loads now, use them after the middles.
        const int ne = nedges[slot];
        float ev[kEdgeRegs];
        int epart[kEdgeRegs], ej[kEdgeRegs];
#pragma unroll
        for (int r = 0; r < kEdgeRegs; ++r) {
            const int g = tid + r * NT;
            epart[r] = -1;
            if (g < ne) {
                int i = 0;
                while (i + 1 < n && pp[i + 1].edge0 <= g) ++i;
                const int q = g - pp[i].edge0;
                const int j = q < pp[i].u0 ? q : pp[i].u1 + (q - pp[i].u0);
                epart[r] = i;
                ej[r] = j;
                ev[r] = __ldg(pp[i].x + j);
            }
        }

        // Middles.  When every middle of the stage is on its segment's grid the
        // output stage mirrors the input stage (same offsets), so the whole
        // stage is one unrolled loop whatever the number of parts.
        const int mid = nmid[slot];
        if (nout[slot] == mid) {
#pragma unroll
            for (int j = 0; j < kRingCap / (NT * E); ++j) {
                const int e = (j * NT + tid) * E;
                if (e < mid) bulk_tile_vec<RED, COEF, OutT>(xs, so, co, e);
            }
        } else {
            for (int i = 0; i < n; ++i) {
                const RingPart p = pp[i];
                const int m = p.u1 - p.u0;
                const float *xi = xs + p.in_off;
                if (p.out_off >= 0) {
                    for (int e = tid * E; e < m; e += NT * E)
                        bulk_tile_vec<RED, COEF, OutT>(xi, so + p.out_off, co + p.out_off, e);
                } else {
                    OutT *sd = (OutT *)p.s + p.u0;
                    OutT *cd = (OutT *)p.c + p.u0;
                    for (int e = tid; e < m; e += NT) {
                        float sv, cv;
                        pair<RED, COEF>(xi[e], sv, cv);
                        store_elem(sd + e, sv);
                        store_elem(cd + e, cv);
                    }
                }
            }
        }

        // This thread is done with the input stage.
        mbar_arrive(smem_addr(&empty[st]));

        // Edges: the pairs of the loaded angles, then any beyond the registers.
#pragma unroll
        for (int r = 0; r < kEdgeRegs; ++r) {
            if (epart[r] >= 0) {
                const RingPart &p = pp[epart[r]];
                float sv, cv;
                pair<RED, COEF>(ev[r], sv, cv);
                store_elem((OutT *)p.s + ej[r], sv);
                store_elem((OutT *)p.c + ej[r], cv);
            }
        }
        for (int g = tid + kEdgeRegs * NT; g < ne; g += NT) {
            int i = 0;
            while (i + 1 < n && pp[i + 1].edge0 <= g) ++i;
            const RingPart &p = pp[i];
            const int q = g - p.edge0;
            const int j = q < p.u0 ? q : p.u1 + (q - p.u0);
            float sv, cv;
            pair<RED, COEF>(p.x[j], sv, cv);
            store_elem((OutT *)p.s + j, sv);
            store_elem((OutT *)p.c + j, cv);
        }

        // Make the output stage visible to the bulk-copy (async) proxy, then
        // one thread stores it and releases the input stage.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        consumer_sync(NT);
        if (tid == 0) {
            for (int i = 0; i < n; ++i) {
                const RingPart &p = pp[i];
                const int m = p.u1 - p.u0;
                if (p.out_off >= 0 && m > 0) {
                    bulk_store((OutT *)p.s + p.u0, so + p.out_off, (uint32_t)(m * sizeof(OutT)));
                    bulk_store((OutT *)p.c + p.u0, co + p.out_off, (uint32_t)(m * sizeof(OutT)));
                }
            }
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Consumer threads of a ring launch for a plan's block size: 128, 256 or 512
// (with the producer warp a CTA must stay within 1024 threads).
static inline int ring_consumers(int block)
{
    return block == 128 ? 128 : block >= 512 ? 512 : 256;
}

template <class OutT, int RED, int COEF>
static const void *ring_kernel_rc(int nt)
{
    switch (nt) {
    case 128: return (const void *)k_batched_ring<OutT, RED, COEF, 128>;
    case 512: return (const void *)k_batched_ring<OutT, RED, COEF, 512>;
    default: return (const void *)k_batched_ring<OutT, RED, COEF, 256>;
    }
}

template <class OutT>
static const void *ring_kernel_t(int red, int coef, int nt)
{
    if (red == RED_PLAIN && coef == COEF_NORMALIZED)
        return ring_kernel_rc<OutT, RED_PLAIN, COEF_NORMALIZED>(nt);
    if (red == RED_COMPENSATED && coef == COEF_NORMALIZED)
        return ring_kernel_rc<OutT, RED_COMPENSATED, COEF_NORMALIZED>(nt);
    if (red == RED_PLAIN && coef == COEF_DAGGER)
        return ring_kernel_rc<OutT, RED_PLAIN, COEF_DAGGER>(nt);
    return ring_kernel_rc<OutT, RED_COMPENSATED, COEF_DAGGER>(nt);
}

// CTAs of a batched tile kernel: all resident ones, at most kMaxBatchedCtas.
static inline int batched_grid(int per_sm, const DeviceInfo &dev)
{
    const int64_t g = (int64_t)per_sm * dev.sms;
    return (int)(g < kMaxBatchedCtas ? g : kMaxBatchedCtas);
}

template <class OutT>
static int launch_batched_ring(const sincos_seg *segs, const int64_t *lens, int count, int red,
                               int coef, int64_t *sched, const sincos_plan &plan,
                               const DeviceInfo &dev, cudaStream_t st)
{
    const int block = ring_consumers(plan.block);
    const void *fn = ring_kernel_t<OutT>(red, coef, block);
    constexpr size_t smem = ring_smem_bytes<OutT>();
    const int per_sm = bulk_resident_ctas(fn, block + 32, smem);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int grid = batched_grid(per_sm, dev);
    (void)sched;                      // the ring kernel schedules itself
    void *args[] = {(void *)&segs, (void *)&lens, (void *)&count};
    const cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((unsigned)(block + 32)),
                                           args, smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "batched ring kernel launch");
    return check_launch("batched ring kernel launch");
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
