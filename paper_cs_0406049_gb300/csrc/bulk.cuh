// bulk.cuh -- the forward kernel with TMA bulk-copy staging ("bulk path").
//
// Each CTA owns a two-stage ring of kBulkChunk-angle input tiles in shared
// memory, filled by 1D bulk copies (cp.async.bulk ... mbarrier::complete_tx),
// and a double-buffered pair of output tiles written back by bulk stores
// (cp.async.bulk.global.shared::cta.bulk_group).  The threads only move data
// between shared memory and registers and compute the pairs.  HBM then sees
// 32 KB sequential reads and writes per request, which on GB300 runs within
// about 2 % of the plain copy bandwidth, against ~6 % below it for per-thread
// 16-byte loads and stores.
//
// Chunks are strided over the persistent grid (chunk = blockIdx.x + k *
// gridDim.x).  The angles before the first 128-byte-line-aligned chunk start
// and after the last whole chunk are done with 16-byte vectors and single
// elements after the chunk loop.
//
// Every mbarrier wait is bounded.  A wait that gives up increments a device
// counter (read by sincos_device_wait_timeouts), the CTA stops consuming,
// waits (bounded) for its own copies still in flight, and exits.
#pragma once

#include "core_x2.cuh"
#include "internal.h"

namespace sincos_gb300 {

constexpr int kBulkChunk = 8192;   // angles per stage (32 KB)
constexpr int kBulkStages = 2;
// A bounded wait gives up after this much wall-clock time (%globaltimer), far
// beyond any healthy stage (a 32 KB copy takes microseconds), so a slow but
// healthy copy on a busy GPU cannot trip it.  The clock is read once every
// kBulkWaitClockEvery polls only: a healthy wait ends long before the first
// read, and the polling loop stays as tight as a plain count (reading a clock
// after the first failed poll cost the batched ring kernel 2 % in an A/B).
// The poll count is capped too, far beyond the time limit, so the loop ends
// even if the timer were not to advance.
constexpr unsigned long long kBulkWaitNs = 1000000000ull;   // 1 s
constexpr unsigned kBulkWaitClockEvery = 1024;
constexpr unsigned kBulkWaitPollCap = 1u << 28;

// Per translation unit; each TU that launches bulk kernels reports its own.
static __device__ unsigned int g_bulk_wait_timeouts = 0;

// Chunk of the small-stage variant: 4096 angles, so that two (binary32
// outputs) or three (16-bit outputs) CTAs fit in an SM's shared memory.
constexpr int kBulkSmallChunk = 4096;

template <class OutT, int CH = kBulkChunk>
constexpr size_t bulk_smem_bytes()
{
    return (size_t)kBulkStages * CH * 4 + 4 * (size_t)CH * sizeof(OutT);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One potentially blocking test of the barrier's phase `parity`.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}

// Wait for phase `parity` of the barrier for at most about limit_ns of
// wall-clock time (measured from the first clock read, kBulkWaitClockEvery
// polls in); false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  unsigned long long limit_ns = kBulkWaitNs)
{
    unsigned long long t0 = 0;
    for (unsigned it = 1; it <= kBulkWaitPollCap; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it % kBulkWaitClockEvery == 0) {
            const unsigned long long t = global_ns();
            if (it == kBulkWaitClockEvery) t0 = t;
            else if (t - t0 >= limit_ns) return false;
        }
    }
    return false;
}

// Programmatic dependent launch.  A bulk kernel is launched with
// programmatic stream serialization (launch_bulk_pdl), so it may start while
// the previous kernel on the stream is still draining.  It lets the kernel
// after it start as early (pdl_release at its own start: that kernel cannot
// fit on an SM before this one's CTA there has exited, and it waits in turn),
// and sets up its shared memory and barriers before pdl_acquire, which blocks
// until every earlier kernel on the stream has completed and its memory
// writes are visible.  Before pdl_acquire a kernel only issues L2 prefetches
// of its first input tiles (bulk_prefetch_l2: hints, which deliver nothing to
// the CTA); every load, store and descriptor read comes after it, so the
// results are those of plain stream order.  Without the launch attribute
// both are no-ops.
__device__ __forceinline__ void pdl_release()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void pdl_acquire()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch `kernel` with programmatic stream serialization (see pdl_release).
template <class... KArgs, class... Args>
static cudaError_t launch_bulk_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                   cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes,
                                          uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst_smem)), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Warm L2 with `bytes` of global memory at src (16-byte aligned, a multiple
// of 16 bytes).  A hint: nothing reaches the CTA, and L2 is where the GPU's
// memory is kept coherent, so a line fetched before another kernel's write to
// it is updated by that write.  This lets a kernel start its first reads
// before pdl_acquire without changing what it reads after it.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 :: "l"(dst), "r"(smem_addr(src_smem)), "r"(bytes) : "memory");
}

// Pairs of the E angles at element e of a staged input tile into the staged
// output tiles (16-byte shared-memory accesses).  PACK: two angles per packed
// FP32 instruction where that applies (see below); the batched ring kernel
// uses the scalar form.
template <int RED, int COEF, class OutT, bool PACK = false>
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
    // Packed (the single-array kernel's binary32 tiles): two angles per
    // packed FP32 instruction (core_x2.cuh, the same bits), which shortens
    // the compute phase between stages (+0.4 % plain, +1.1 % compensated at
    // 2^28 with the normalized set; with the dagger set +0.3-1.3 % on the
    // one-CTA plan, +10-14 % on 128-thread CTAs, within 0.5 % on the
    // 512-thread small-stage plan).  For 16-bit outputs the packed form needs
    // more registers than three CTAs of 512 threads can share and loses (6066
    // against 6532 GB/s); the batched ring kernel uses it with the compensated
    // reduction only (+1.2 % there with the normalized set, +6 % with the
    // dagger set; -0.5 % with the plain reduction).
    if constexpr (PACK && sizeof(OutT) == 4) {
#pragma unroll
        for (int i = 0; i < E; i += 2) {
            float2 s2, c2;
            pair_x2<RED, COEF>(make_float2(in[i], in[i + 1]), s2, c2);
            sv[i] = s2.x;
            sv[i + 1] = s2.y;
            cv[i] = c2.x;
            cv[i + 1] = c2.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) pair<RED, COEF>(in[i], sv[i], cv[i]);
    }
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

template <class OutT, int RED, int COEF, int NT, int CH>
__global__ void __launch_bounds__(NT)
k_forward_bulk(const float *x, OutT *s, OutT *c, int64_t n, int64_t head, int64_t nchunks)
{
    constexpr int E = Vec<OutT, 16>::E;                       // pairs per 16-byte output vector
    constexpr int PER_THREAD = CH / (NT * E);         // output vectors per thread per chunk
    static_assert(CH % (NT * E) == 0, "chunk must split evenly over the CTA");
    extern __shared__ __align__(128) unsigned char smem[];
    float *xin = (float *)smem;                                        // [stages][chunk]
    OutT *sout = (OutT *)(xin + kBulkStages * CH);              // [2][chunk]
    OutT *cout = sout + 2 * CH;                                 // [2][chunk]
    __shared__ __align__(8) uint64_t full[kBulkStages];
    __shared__ int64_t issued[kBulkStages];
    __shared__ int give_up;

    pdl_release();
    const float *xg = x + head;
    OutT *sg = s + head;
    OutT *cg = c + head;
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
    // The first stage's angles into L2 while the previous kernel drains.
    // Back-to-back calls on GB300: +1-5 % from 2^23 to 2^26 angles, +0.2 % at
    // 2^28, neutral below; both stages lost up to 6 % at 2^21-2^23.5 angles
    // with L2 flushed between calls.
    if (tid == 0 && blockIdx.x < nchunks)
        bulk_prefetch_l2(xg + blockIdx.x * (int64_t)CH, CH * 4);
    __syncthreads();
    pdl_acquire();
    if (tid == 0) {
        for (int st = 0; st < kBulkStages; ++st) {
            const int64_t ch = blockIdx.x + (int64_t)st * gridDim.x;
            if (ch < nchunks) {
                bulk_load(xin + st * CH, xg + ch * CH, CH * 4,
                          smem_addr(&full[st]));
                issued[st] += 1;
            }
        }
    }

    int64_t k = 0;
    for (;; ++k) {
        const int64_t ch = blockIdx.x + k * gridDim.x;
        if (ch >= nchunks) break;
        const int st = (int)(k % kBulkStages);
        if (!mbar_wait_bounded(smem_addr(&full[st]), (uint32_t)((k / kBulkStages) & 1))) {
            atomicAdd(&g_bulk_wait_timeouts, 1u);
            give_up = 1;
        }
        const int b = (int)(k & 1);
        // The bulk store that last read output buffer b (two chunks ago) must
        // be done reading it before it is overwritten.
        if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncthreads();
        if (give_up) break;
        const float *xi = xin + st * CH;
        OutT *so = sout + b * CH;
        OutT *co = cout + b * CH;
#pragma unroll
        for (int j = 0; j < PER_THREAD; ++j)
            bulk_tile_vec<RED, COEF, OutT, true>(xi, so, co, (j * NT + tid) * E);
        // Make the tile visible to the bulk-copy (async) proxy, then let one
        // thread store it and refill this input stage.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            bulk_store(sg + ch * CH, so, CH * sizeof(OutT));
            bulk_store(cg + ch * CH, co, CH * sizeof(OutT));
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            const int64_t next = blockIdx.x + (k + kBulkStages) * gridDim.x;
            if (next < nchunks) {
                bulk_load(xin + st * CH, xg + next * CH, CH * 4,
                          smem_addr(&full[st]));
                issued[st] += 1;
            }
        }
    }
    if (give_up && tid == 0) {
        // Drain (bounded) the loads still in flight into this CTA's memory.
        for (int st = 0; st < kBulkStages; ++st) {
            const int64_t consumed = k / kBulkStages + ((k % kBulkStages) > st ? 1 : 0);
            for (int64_t j = consumed; j < issued[st]; ++j)
                mbar_wait_bounded(smem_addr(&full[st]), (uint32_t)(j & 1));
        }
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (give_up) return;

    // Angles after the last whole chunk: 16-byte vectors spread over the CTAs,
    // then single elements; the head before the aligned start goes to CTA 0.
    const int64_t rest0 = nchunks * CH;                // relative to head
    const int64_t nrest = (n - head - rest0) / E;
    for (int64_t v = blockIdx.x * (int64_t)NT + tid; v < nrest; v += (int64_t)gridDim.x * NT) {
        float in[E];
        load_vec<OutT, 16, LD_COHERENT>(in, xg + rest0 + v * E);
        compute_store<RED, COEF, OutT, 16>(in, sg + rest0 + v * E, cg + rest0 + v * E);
    }
    if (blockIdx.x == 0) {
        for (int64_t i = tid; i < head; i += NT) scalar_elem<RED, COEF>(x, s, c, i);
        for (int64_t i = head + rest0 + nrest * E + tid; i < n; i += NT)
            scalar_elem<RED, COEF>(x, s, c, i);
    }
}

// Dynamic shared memory opt-in (once per kernel and device) and the resident
// CTAs per SM at that size.
int bulk_resident_ctas(const void *kernel, int block, size_t smem);

template <class OutT, int RED, int COEF, int NT, int CH = kBulkChunk>
static int launch_forward_bulk_nt(const float *x, OutT *s, OutT *c, int64_t n, int64_t head,
                                  const DeviceInfo &dev, cudaStream_t st)
{
    const void *fn = (const void *)k_forward_bulk<OutT, RED, COEF, NT, CH>;
    constexpr size_t smem = bulk_smem_bytes<OutT, CH>();
    const int per_sm = bulk_resident_ctas(fn, NT, smem);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t nchunks = (n - head) / CH;
    int64_t grid = (int64_t)per_sm * dev.sms;
    if (nchunks < grid) grid = nchunks > 0 ? nchunks : 1;
    const cudaError_t e = launch_bulk_pdl(k_forward_bulk<OutT, RED, COEF, NT, CH>,
                                          dim3((unsigned)grid), dim3(NT), smem, st, x, s, c, n,
                                          head, nchunks);
    if (e != cudaSuccess) return cuda_fail(e, "bulk forward kernel launch");
    return check_launch("bulk forward kernel launch");
}

// Reads and clears this translation unit's bulk-wait timeout counter.
static inline unsigned take_bulk_wait_timeouts_here()
{
    unsigned v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_bulk_wait_timeouts, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaMemcpyToSymbol(g_bulk_wait_timeouts, &zero, sizeof zero);
    return v;
}

}  // namespace sincos_gb300
