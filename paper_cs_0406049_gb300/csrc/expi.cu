// expi.cu -- exp(i x) = cos x + i sin x as interleaved complex64: z[2i] = c,
// z[2i+1] = s, for consumers that want phase factors (FFTs, Huygens-type
// sums) in one stream.  The pairs are the method's (core.cuh); only the
// output layout differs from the forward kernels: one 8-byte output stream
// per angle instead of two 4-byte ones, the same 12 bytes per angle.
//
// Register path: 4 angles per 16-byte load, 32 bytes of output per vector
// (one 256-bit evict-first store when z allows, else two 16-byte stores), the
// chunked grid-stride layout of forward.cuh.  Bulk path: 8192-angle chunks through the two-stage TMA ring
// of bulk.cuh; each chunk's 64 KB of output leaves in one bulk store.
#include "bulk.cuh"
#include "core.cuh"
#include "trace.h"
#include "internal.h"

namespace sincos_gb300 {

// Four angles to 32 bytes of (cos, sin) pairs: one 256-bit evict-first store
// when z is 32-byte aligned (W = 32), so every 32-byte sector is written
// whole by one instruction; two 16-byte stores otherwise (W = 16).
template <int RED, int COEF, int W>
__device__ __forceinline__ void expi_vec(const float *in, float *z)
{
    float s0, s1, s2, s3, c0, c1, c2, c3;
    pair<RED, COEF>(in[0], s0, c0);
    pair<RED, COEF>(in[1], s1, c1);
    pair<RED, COEF>(in[2], s2, c2);
    pair<RED, COEF>(in[3], s3, c3);
    const uint32_t w[8] = {__float_as_uint(c0), __float_as_uint(s0), __float_as_uint(c1),
                           __float_as_uint(s1), __float_as_uint(c2), __float_as_uint(s2),
                           __float_as_uint(c3), __float_as_uint(s3)};
    if constexpr (W == 32) {
        store_words<32>(z, w);
    } else {
        store_words<16>(z, w);
        store_words<16>(z + 4, w + 4);
    }
}

template <int RED, int COEF>
__device__ __forceinline__ void expi_elem(const float *x, float *z, int64_t i)
{
    float s, c;
    pair<RED, COEF>(x[i], s, c);
    z[2 * i] = c;
    z[2 * i + 1] = s;
}

template <int RED, int COEF, int UNROLL, int LD, int W>
__global__ void k_expi(const float *x, float *z, int64_t n, int64_t head, int64_t nvec)
{
    const float *xv = x + head;
    float *zv = z + 2 * head;
    const int64_t chunk = (int64_t)blockDim.x * UNROLL;
    const int64_t nfull = nvec / chunk;
    for (int64_t ch = blockIdx.x; ch < nfull; ch += gridDim.x) {
        const int64_t v0 = ch * chunk + threadIdx.x;
        float in[UNROLL][4];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) ld16<LD>(in[u], xv + (v0 + (int64_t)u * blockDim.x) * 4);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            expi_vec<RED, COEF, W>(in[u], zv + (v0 + (int64_t)u * blockDim.x) * 8);
    }
    if (blockIdx.x == (unsigned)(nfull % gridDim.x)) {
        for (int64_t v = nfull * chunk + threadIdx.x; v < nvec; v += blockDim.x) {
            float in[4];
            ld16<LD>(in, xv + v * 4);
            expi_vec<RED, COEF, W>(in, zv + v * 8);
        }
        for (int64_t i = threadIdx.x; i < head; i += blockDim.x) expi_elem<RED, COEF>(x, z, i);
        for (int64_t i = head + nvec * 4 + threadIdx.x; i < n; i += blockDim.x)
            expi_elem<RED, COEF>(x, z, i);
    }
}

template <int RED, int COEF>
__global__ void k_expi_scalar(const float *x, float *z, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        expi_elem<RED, COEF>(x, z, i);
}

template <int RED, int COEF, int NT>
__global__ void __launch_bounds__(NT)
k_expi_bulk(const float *x, float *z, int64_t n, int64_t head, int64_t nchunks)
{
    constexpr int PER_THREAD = kBulkChunk / (NT * 4);
    extern __shared__ __align__(128) unsigned char smem[];
    float *xin = (float *)smem;                              // [stages][chunk]
    float *zout = xin + kBulkStages * kBulkChunk;            // [2][2 * chunk]
    __shared__ __align__(8) uint64_t full[kBulkStages];
    __shared__ int64_t issued[kBulkStages];
    __shared__ int give_up;

    pdl_release();
    const float *xg = x + head;
    float *zg = z + 2 * head;
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
    // The first stage's angles into L2 while the previous kernel drains, as
    // in the single-array forward kernel.
    if (tid == 0 && blockIdx.x < nchunks)
        bulk_prefetch_l2(xg + blockIdx.x * (int64_t)kBulkChunk, kBulkChunk * 4);
    __syncthreads();
    pdl_acquire();                 // no other global access before the previous kernel is done
    if (tid == 0) {
        for (int st = 0; st < kBulkStages; ++st) {
            const int64_t ch = blockIdx.x + (int64_t)st * gridDim.x;
            if (ch < nchunks) {
                bulk_load(xin + st * kBulkChunk, xg + ch * kBulkChunk, kBulkChunk * 4,
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
        if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncthreads();
        if (give_up) break;
        const float *xi = xin + st * kBulkChunk;
        float *zo = zout + b * 2 * kBulkChunk;
#pragma unroll
        for (int j = 0; j < PER_THREAD; ++j) {
            const int e = (j * NT + tid) * 4;
            const float4 v = *reinterpret_cast<const float4 *>(xi + e);
            float s0, s1, s2, s3, c0, c1, c2, c3;
            // The packed pair (same bits) pays with the compensated reduction
            // only: 6425 against 6337 GB/s at 2^26 and 6621 against 6533 at
            // 2^28 (normalized set), 6088 against 6005 and 6213 against 6139
            // (dagger set); with the plain one it measured 0.4 % slower.
            if constexpr (RED == RED_COMPENSATED) {
                float2 sa, ca, sb, cb;
                pair_x2<RED, COEF>(make_float2(v.x, v.y), sa, ca);
                pair_x2<RED, COEF>(make_float2(v.z, v.w), sb, cb);
                s0 = sa.x;
                s1 = sa.y;
                c0 = ca.x;
                c1 = ca.y;
                s2 = sb.x;
                s3 = sb.y;
                c2 = cb.x;
                c3 = cb.y;
            } else {
                pair<RED, COEF>(v.x, s0, c0);
                pair<RED, COEF>(v.y, s1, c1);
                pair<RED, COEF>(v.z, s2, c2);
                pair<RED, COEF>(v.w, s3, c3);
            }
            *reinterpret_cast<float4 *>(zo + 2 * e) = make_float4(c0, s0, c1, s1);
            *reinterpret_cast<float4 *>(zo + 2 * e + 4) = make_float4(c2, s2, c3, s3);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            bulk_store(zg + 2 * ch * kBulkChunk, zo, 2 * kBulkChunk * 4);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            const int64_t next = blockIdx.x + (k + kBulkStages) * gridDim.x;
            if (next < nchunks) {
                bulk_load(xin + st * kBulkChunk, xg + next * kBulkChunk, kBulkChunk * 4,
                          smem_addr(&full[st]));
                issued[st] += 1;
            }
        }
    }
    if (give_up && tid == 0) {
        for (int st = 0; st < kBulkStages; ++st) {
            const int64_t consumed = k / kBulkStages + ((k % kBulkStages) > st ? 1 : 0);
            for (int64_t j = consumed; j < issued[st]; ++j)
                mbar_wait_bounded(smem_addr(&full[st]), (uint32_t)(j & 1));
        }
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (give_up) return;
    const int64_t rest0 = nchunks * kBulkChunk;
    const int64_t nrest = (n - head - rest0) / 4;
    for (int64_t v = blockIdx.x * (int64_t)NT + tid; v < nrest; v += (int64_t)gridDim.x * NT) {
        float in[4];
        ld16<LD_COHERENT>(in, xg + rest0 + v * 4);
        expi_vec<RED, COEF, 16>(in, zg + 2 * (rest0 + v * 4));
    }
    if (blockIdx.x == 0) {
        for (int64_t i = tid; i < head; i += NT) expi_elem<RED, COEF>(x, z, i);
        for (int64_t i = head + rest0 + nrest * 4 + tid; i < n; i += NT)
            expi_elem<RED, COEF>(x, z, i);
    }
}

// Where the vector grid starts: x + h and z + 2h both on a 128-byte line if
// possible, else x + h 16-byte and z + 2h 32-byte aligned (*w = 32), else both
// 16-byte aligned (*w = 16); -1 if none exists.
static int expi_head(const float *x, const float *z, int *w)
{
    const uintptr_t ax = (uintptr_t)x, az = (uintptr_t)z;
    *w = 32;
    if ((ax & 3u) || (az & 7u)) return -1;
    for (int h = 0; h < 32; ++h)
        if (((ax + 4u * h) & 127u) == 0 && ((az + 8u * h) & 127u) == 0) return h;
    for (int h = 0; h < 8; ++h)
        if (((ax + 4u * h) & 15u) == 0 && ((az + 8u * h) & 31u) == 0) return h;
    *w = 16;
    for (int h = 0; h < 4; ++h)
        if (((ax + 4u * h) & 15u) == 0 && ((az + 8u * h) & 15u) == 0) return h;
    return -1;
}

template <int RED, int COEF, int UNROLL, int W>
static int launch_expi_vec(const float *x, float *z, int64_t n, int64_t head,
                           const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    const void *fn = (const void *)k_expi<RED, COEF, UNROLL, LD_NC, W>;
    int per_sm = 0;
    const sincos_plan p = fit_plan(fn, plan, &per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t nvec = (n - head) / 4;
    const int64_t chunks = nvec / ((int64_t)p.block * UNROLL);
    int64_t grid = (int64_t)per_sm * dev.sms;
    if (chunks < grid) grid = chunks > 0 ? chunks : 1;
    k_expi<RED, COEF, UNROLL, LD_NC, W><<<(unsigned)grid, p.block, 0, st>>>(x, z, n, head, nvec);
    return check_launch("expi kernel launch");
}

template <int RED, int COEF, int NT>
static int launch_expi_bulk(const float *x, float *z, int64_t n, int64_t head,
                            const DeviceInfo &dev, cudaStream_t st)
{
    const void *fn = (const void *)k_expi_bulk<RED, COEF, NT>;
    constexpr size_t smem = (size_t)kBulkStages * kBulkChunk * 4 + 2 * 2 * (size_t)kBulkChunk * 4;
    const int per_sm = bulk_resident_ctas(fn, NT, smem);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t nchunks = (n - head) / kBulkChunk;
    int64_t grid = (int64_t)per_sm * dev.sms;
    if (nchunks < grid) grid = nchunks > 0 ? nchunks : 1;
    const cudaError_t e = launch_bulk_pdl(k_expi_bulk<RED, COEF, NT>, dim3((unsigned)grid),
                                          dim3(NT), smem, st, x, z, n, head, nchunks);
    if (e != cudaSuccess) return cuda_fail(e, "exp(ix) bulk kernel launch");
    return check_launch("expi bulk kernel launch");
}

template <int RED, int COEF, int W>
static int launch_expi_w(const float *x, float *z, int64_t n, int64_t head,
                         const sincos_plan &plan, const DeviceInfo &dev, cudaStream_t st)
{
    switch (plan.unroll) {
    case 1:
    case 2: return launch_expi_vec<RED, COEF, 2, W>(x, z, n, head, plan, dev, st);
    case 4: return launch_expi_vec<RED, COEF, 4, W>(x, z, n, head, plan, dev, st);
    default: return launch_expi_vec<RED, COEF, 8, W>(x, z, n, head, plan, dev, st);
    }
}

template <int RED, int COEF>
static int launch_expi_rc(const float *x, float *z, int64_t n, const sincos_plan &plan,
                          const DeviceInfo &dev, cudaStream_t st)
{
    int w = 16;
    const int h = expi_head(x, z, &w);
    if (h < 0) {
        const void *fn = (const void *)k_expi_scalar<RED, COEF>;
        int per_sm = 0;
        const sincos_plan p = fit_plan(fn, plan, &per_sm);
        if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
        int64_t grid = (int64_t)per_sm * dev.sms;
        const int64_t need = (n + p.block - 1) / p.block;
        if (need < grid) grid = need;
        k_expi_scalar<RED, COEF><<<(unsigned)grid, p.block, 0, st>>>(x, z, n);
        return check_launch("expi scalar kernel launch");
    }
    const int64_t head = h < n ? h : n;
    if (plan_vec_bytes(plan) == 0 && n - head >= kBulkChunk)
        return plan.block == 256 ? launch_expi_bulk<RED, COEF, 256>(x, z, n, head, dev, st)
                                 : launch_expi_bulk<RED, COEF, 512>(x, z, n, head, dev, st);
    if (w == 32 && plan_vec_bytes(plan) != 16)
        return launch_expi_w<RED, COEF, 32>(x, z, n, head, plan, dev, st);
    return launch_expi_w<RED, COEF, 16>(x, z, n, head, plan, dev, st);
}

// Launch with an explicit plan (shared by the entry point and the autotuner).
int launch_expi(const float *x, float *z, int64_t n, int red, int coef, const sincos_plan &plan,
                const DeviceInfo &dev, cudaStream_t st)
{
    if (red == RED_PLAIN && coef == COEF_NORMALIZED)
        return launch_expi_rc<RED_PLAIN, COEF_NORMALIZED>(x, z, n, plan, dev, st);
    if (red == RED_COMPENSATED && coef == COEF_NORMALIZED)
        return launch_expi_rc<RED_COMPENSATED, COEF_NORMALIZED>(x, z, n, plan, dev, st);
    if (red == RED_PLAIN && coef == COEF_DAGGER)
        return launch_expi_rc<RED_PLAIN, COEF_DAGGER>(x, z, n, plan, dev, st);
    return launch_expi_rc<RED_COMPENSATED, COEF_DAGGER>(x, z, n, plan, dev, st);
}

unsigned take_timeouts_expi() { return take_bulk_wait_timeouts_here(); }

}  // namespace sincos_gb300

using namespace sincos_gb300;

extern "C" int sincos_expi(const float *x, float *z, int64_t n, int reduction, int coef,
                           sincos_stream_t stream)
{
    SINCOS_TRACE("sincos_expi");
    if (n < 0 || !valid_reduction(reduction) || !valid_coef(coef)) return SINCOS_EINVAL;
    if (n == 0) return SINCOS_OK;
    if (!x || !z) return SINCOS_EINVAL;
    if (!all_float_aligned({x, z})) return SINCOS_EINVAL;
    const uintptr_t x0 = (uintptr_t)x, z0 = (uintptr_t)z;
    if (x0 < z0 + 8u * (uint64_t)n && z0 < x0 + 4u * (uint64_t)n) return SINCOS_EOVERLAP;
    const DeviceInfo *dev = nullptr;
    const int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    const sincos_plan plan = plan_for(*dev, SINCOS_OP_EXPI, SINCOS_F32, n);
    return launch_expi(x, z, n, reduction, coef, plan, *dev, (cudaStream_t)stream);
}
