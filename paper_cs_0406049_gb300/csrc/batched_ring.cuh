// batched_ring.cuh -- the ring (TMA-staged) batched kernel, the default for
// binary32 outputs: one launch, no scratch (see the section comment below).
#pragma once

#include "batched_common.cuh"

namespace sincos_gb300 {

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
// groups for the two output stages.  Every wait is bounded.  A wait that
// gives up counts a timeout and stops its side; the producer then waits
// (bounded) for every copy it issued before the CTA may exit.
// ---------------------------------------------------------------------------

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

// Stage capacity of the small-stage variant (plans with ctas_per_sm >= 2):
// half the angles per stage, so that two (binary32) or three (16-bit
// outputs) CTAs share an SM, as the single-array kernel's small stages do.
constexpr int kRingSmallCap = kBulkSmallChunk;

template <class OutT, int CAP = kRingCap>
constexpr size_t ring_smem_bytes()
{
    return (size_t)kRingStages * CAP * 4 + 2 * 2 * (size_t)CAP * sizeof(OutT);
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
// ok: the descriptor passes seg_ok (else the producer skips the segment).
struct SegMeta {
    const float *x;
    void *s;
    void *c;
    int64_t len, nt;
    int h;
    bool ok;
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
        m.ok = seg_ok<OutT>(d, m.len);
    } else {
        m.x = nullptr;
        m.s = m.c = nullptr;
        m.len = m.nt = 0;
        m.h = -1;
        m.ok = true;
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
template <class OutT, int CAP>
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
                    // A descriptor that fails seg_ok keeps its place in the
                    // schedule (the prologue reads lengths only) but is not
                    // processed; the CTA that owns its first tile counts it.
                    if (kt < kend && !__shfl_sync(0xffffffffu, (int)w.ok, c)) {
                        if (kt == 0 && lane == 0) atomicAdd(&g_bad_segments, 1u);
                        ++seg;
                        kt = 0;
                        continue;
                    }
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
            const int64_t avail = CAP - cap;
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
            float *dst = xin + (size_t)st * CAP;
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

template <class OutT, int RED, int COEF, int NT, int CAP>
__global__ void __launch_bounds__(NT + 32)
k_batched_ring(const sincos_seg *segs, const int64_t *lens, int count)
{
    constexpr int E = Vec<OutT, 16>::E;
    constexpr int kEdgeRegs = 4;
    extern __shared__ __align__(128) unsigned char smem[];
    float *xin = (float *)smem;                                        // [stages][cap]
    OutT *sout = (OutT *)(xin + kRingStages * CAP);                     // [2][cap]
    OutT *cout = sout + 2 * CAP;                                        // [2][cap]
    __shared__ RingPart parts[kRingSlots][kRingMaxParts];
    __shared__ int nparts[kRingSlots], nedges[kRingSlots], nmid[kRingSlots], nout[kRingSlots];
    __shared__ __align__(8) uint64_t full[kRingStages], empty[kRingStages];
    __shared__ int give_up;
    __shared__ RingRun run;
    __shared__ int64_t wa[32], wb[32];
    __shared__ int64_t red[kRunBatch][32], tot[kRunBatch], ctot[kRunChunks];

    // Programmatic dependent launch (see pdl_release): the descriptors and
    // lengths may come from the previous kernel on the stream, so every
    // global access waits for it.
    pdl_release();
    pdl_acquire();
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
        ring_producer<OutT, CAP>(segs, lens, count, run, xin, parts, nparts, nedges, nmid, nout,
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
        const float *xs = xin + (size_t)st * CAP;
        OutT *so = sout + (size_t)b * CAP;
        OutT *co = cout + (size_t)b * CAP;

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
        // stage is one unrolled loop whatever the number of parts.  Binary32
        // tiles take the packed pair (same bits) with the compensated
        // reduction only: on the 4096-array workload it gave 6153 against
        // 6081 GB/s there, and 6270 against 6301 with the plain reduction.
        constexpr bool kPack = RED == RED_COMPENSATED;
        const int mid = nmid[slot];
        if (nout[slot] == mid) {
#pragma unroll
            for (int j = 0; j < CAP / (NT * E); ++j) {
                const int e = (j * NT + tid) * E;
                if (e < mid) bulk_tile_vec<RED, COEF, OutT, kPack>(xs, so, co, e);
            }
        } else {
            for (int i = 0; i < n; ++i) {
                const RingPart p = pp[i];
                const int m = p.u1 - p.u0;
                const float *xi = xs + p.in_off;
                if (p.out_off >= 0) {
                    for (int e = tid * E; e < m; e += NT * E)
                        bulk_tile_vec<RED, COEF, OutT, kPack>(xi, so + p.out_off, co + p.out_off, e);
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

template <class OutT, int RED, int COEF, int CAP>
static const void *ring_kernel_cap(int nt)
{
    switch (nt) {
    case 128: return (const void *)k_batched_ring<OutT, RED, COEF, 128, CAP>;
    case 512: return (const void *)k_batched_ring<OutT, RED, COEF, 512, CAP>;
    default: return (const void *)k_batched_ring<OutT, RED, COEF, 256, CAP>;
    }
}

template <class OutT, int RED, int COEF>
static const void *ring_kernel_rc(int nt, bool small)
{
    return small ? ring_kernel_cap<OutT, RED, COEF, kRingSmallCap>(nt)
                 : ring_kernel_cap<OutT, RED, COEF, kRingCap>(nt);
}

template <class OutT>
static const void *ring_kernel_t(int red, int coef, int nt, bool small)
{
    if (red == RED_PLAIN && coef == COEF_NORMALIZED)
        return ring_kernel_rc<OutT, RED_PLAIN, COEF_NORMALIZED>(nt, small);
    if (red == RED_COMPENSATED && coef == COEF_NORMALIZED)
        return ring_kernel_rc<OutT, RED_COMPENSATED, COEF_NORMALIZED>(nt, small);
    if (red == RED_PLAIN && coef == COEF_DAGGER)
        return ring_kernel_rc<OutT, RED_PLAIN, COEF_DAGGER>(nt, small);
    return ring_kernel_rc<OutT, RED_COMPENSATED, COEF_DAGGER>(nt, small);
}


template <class OutT>
static int launch_batched_ring(const sincos_seg *segs, const int64_t *lens, int count, int red,
                               int coef, int64_t *sched, const sincos_plan &plan,
                               const DeviceInfo &dev, cudaStream_t st)
{
    const int block = ring_consumers(plan.block);
    // ctas_per_sm >= 2 asks for the small-stage variant, as for the
    // single-array bulk kernel
    const bool small = plan.ctas_per_sm >= 2;
    const void *fn = ring_kernel_t<OutT>(red, coef, block, small);
    const size_t smem = small ? ring_smem_bytes<OutT, kRingSmallCap>() : ring_smem_bytes<OutT>();
    const int per_sm = bulk_resident_ctas(fn, block + 32, smem);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int grid = batched_grid(per_sm, dev);
    (void)sched;                      // the ring kernel schedules itself
    void *args[] = {(void *)&segs, (void *)&lens, (void *)&count};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)(block + 32));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e != cudaSuccess) return cuda_fail(e, "batched ring kernel launch");
    return check_launch("batched ring kernel launch");
}

}  // namespace sincos_gb300
