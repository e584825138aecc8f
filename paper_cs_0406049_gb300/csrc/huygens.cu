// huygens.cu -- Huygens-principle field sum with the method's phase factors
// generated in registers (the application the paper names in its
// conclusions: optical diffraction patterns by Huygens' principle).
//
//   u_i = sum_j a_j exp(i k r_ij) / r_ij,   r_ij = |p_i - q_j|
//
// Each term, in binary32 with explicit roundings:
//   d = p_i - q_j;  r = sqrt_rn(fma(dz, dz, fma(dy, dy, dx*dx)));  w = rcp_rn(r)
//   (s, c) = pair(k*r)                       (core.cuh, normalized set)
//   u_re = fma(w, fma(ar, c, -(ai*s)), u_re);  u_im = fma(w, fma(ar, s, ai*c), u_im)
// summed over j in source order from 0, so the result does not depend on the
// launch configuration.
//
// Schedule.  A thread owns P consecutive observation points and keeps their
// coordinates and sums in registers.  Sources stream through shared memory
// in tiles; inside a tile every thread reads the same source at the same
// time (a broadcast).  Two kernels, chosen by the plan's vec_bytes:
//   16  k_huygens: one instruction per binary32 operation.  About 66
//       instructions per term, bound by instruction issue.
//   32  k_huygens_x2: two consecutive sources per instruction on the packed
//       binary32 pipe (core_x2.cuh); the square root, the reciprocal, rint,
//       the signed steps of the pair and the source-order accumulation stay
//       scalar.  About 47 instructions per term; each packed instruction
//       holds the FMA pipe for two cycles, so that pipe is the bound.
// Pairing points instead of sources halves the warps and loses to latency.
#include "core_rt.cuh"
#include "trace.h"
#include "internal.h"

namespace sincos_gb300 {

constexpr int kHuyTile = 2048;

template <int RED, int P>
__global__ void k_huygens(const float *px, const float *py, const float *pz, int64_t m,
                          const float *qx, const float *qy, const float *qz, const float *ar,
                          const float *ai, int64_t n, float k, float *u)
{
    __shared__ float4 sq[kHuyTile];        // qx, qy, qz, ar
    __shared__ float sai[kHuyTile];        // ai
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * P;
    float x[P], y[P], z[P], ure[P], uim[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int64_t i = i0 + p < m ? i0 + p : m - 1;     // tail threads repeat the last point
        x[p] = px[i];
        y[p] = py[i];
        z[p] = pz[i];
        ure[p] = 0.0f;
        uim[p] = 0.0f;
    }
    for (int64_t j0 = 0; j0 < n; j0 += kHuyTile) {
        const int cnt = (int)(n - j0 < kHuyTile ? n - j0 : kHuyTile);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            sq[t] = make_float4(qx[j0 + t], qy[j0 + t], qz[j0 + t], ar[j0 + t]);
            sai[t] = ai[j0 + t];
        }
        __syncthreads();
#pragma unroll 2
        for (int t = 0; t < cnt; ++t) {
            const float4 q = sq[t];
            const float aim = sai[t];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float dx = __fsub_rn(x[p], q.x);
                const float dy = __fsub_rn(y[p], q.y);
                const float dz = __fsub_rn(z[p], q.z);
                float r, w;
                root_recip(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))), r, w);
                float s, c;
                pair<RED, COEF_NORMALIZED>(__fmul_rn(k, r), s, c);
                const float pr = __fmaf_rn(q.w, c, -__fmul_rn(aim, s));
                const float pi = __fmaf_rn(q.w, s, __fmul_rn(aim, c));
                ure[p] = __fmaf_rn(w, pr, ure[p]);
                uim[p] = __fmaf_rn(w, pi, uim[p]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (i0 + p < m) {
            u[2 * (i0 + p)] = ure[p];
            u[2 * (i0 + p) + 1] = uim[p];
        }
    }
}

constexpr int kHuyTileX2 = 1024;   // sources per tile, even

// P points per thread; the sources are taken two at a time on the packed
// pipe (terms (i, j) and (i, j+1) in one instruction), and each point's sums
// take the two terms in source order with scalar fmas.  Per source pair,
// three 16-byte shared words: (-qx_j, -qx_j+1, -qy_j, -qy_j+1),
// (-qz_j, -qz_j+1, ar_j, ar_j+1), (ai_j, ai_j+1, -ai_j, -ai_j+1).  Per term
// the operations are those of k_huygens: d = p + (-q) = p - q and
// -(ai*s) = (-ai)*s.  An odd last source is done by the scalar term.  With
// one point per thread the kernel is held to 32 registers, so that 2048
// threads (8 CTAs of 256) stay resident on an SM; more points per thread
// need more registers and get no cap.
template <int RED, int P>
__global__ void __launch_bounds__(1024, P == 1 ? 2 : 1) k_huygens_x2(const float *px, const float *py, const float *pz, int64_t m,
                             const float *qx, const float *qy, const float *qz, const float *ar,
                             const float *ai, int64_t n, float k, float *u)
{
    __shared__ float4 src[3 * (kHuyTileX2 / 2)];
    float *srcf = reinterpret_cast<float *>(src);
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * P;
    float2 x[P], y[P], z[P];
    float ure[P], uim[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int64_t i = i0 + p < m ? i0 + p : m - 1;     // tail threads repeat the last point
        x[p] = splat2(px[i]);
        y[p] = splat2(py[i]);
        z[p] = splat2(pz[i]);
        ure[p] = 0.0f;
        uim[p] = 0.0f;
    }
    const float2 k2 = splat2(k);
    for (int64_t j0 = 0; j0 < n; j0 += kHuyTileX2) {
        const int cnt = (int)(n - j0 < kHuyTileX2 ? n - j0 : kHuyTileX2);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            float *f = srcf + 12 * (t >> 1) + (t & 1);
            const float im = ai[j0 + t];
            f[0] = -qx[j0 + t];
            f[2] = -qy[j0 + t];
            f[4] = -qz[j0 + t];
            f[6] = ar[j0 + t];
            f[8] = im;
            f[10] = -im;
        }
        __syncthreads();
        const int npair = cnt >> 1;
#pragma unroll 2
        for (int h = 0; h < npair; ++h) {
            const float4 w0 = src[3 * h], w1 = src[3 * h + 1], w2 = src[3 * h + 2];
            const float2 nqx = make_float2(w0.x, w0.y), nqy = make_float2(w0.z, w0.w);
            const float2 nqz = make_float2(w1.x, w1.y), are = make_float2(w1.z, w1.w);
            const float2 aim = make_float2(w2.x, w2.y), naim = make_float2(w2.z, w2.w);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float2 dx = __fadd2_rn(x[p], nqx);
                const float2 dy = __fadd2_rn(y[p], nqy);
                const float2 dz = __fadd2_rn(z[p], nqz);
                const float2 rr = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                float2 r, w;
                root_recip_x2(rr, r, w);
                float2 sv, cv;
                pair_x2<RED, COEF_NORMALIZED>(__fmul2_rn(k2, r), sv, cv);
                const float2 pr = __ffma2_rn(are, cv, __fmul2_rn(naim, sv));
                const float2 pi = __ffma2_rn(are, sv, __fmul2_rn(aim, cv));
                ure[p] = __fmaf_rn(w.y, pr.y, __fmaf_rn(w.x, pr.x, ure[p]));
                uim[p] = __fmaf_rn(w.y, pi.y, __fmaf_rn(w.x, pi.x, uim[p]));
            }
        }
        if (cnt & 1) {
            const float *f = srcf + 12 * npair;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float dx = __fadd_rn(x[p].x, f[0]);
                const float dy = __fadd_rn(y[p].x, f[2]);
                const float dz = __fadd_rn(z[p].x, f[4]);
                float r, w;
                root_recip(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))), r, w);
                float sv, cv;
                pair<RED, COEF_NORMALIZED>(__fmul_rn(k, r), sv, cv);
                ure[p] = __fmaf_rn(w, __fmaf_rn(f[6], cv, __fmul_rn(f[10], sv)), ure[p]);
                uim[p] = __fmaf_rn(w, __fmaf_rn(f[6], sv, __fmul_rn(f[8], cv)), uim[p]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (i0 + p < m) {
            u[2 * (i0 + p)] = ure[p];
            u[2 * (i0 + p) + 1] = uim[p];
        }
    }
}

template <int RED, int P>
static int launch_huygens_p(const float *px, const float *py, const float *pz, int64_t m,
                            const float *qx, const float *qy, const float *qz, const float *ar,
                            const float *ai, int64_t n, float k, float *u,
                            const sincos_plan &plan, cudaStream_t st)
{
    const bool packed = plan.vec_bytes == 32;
    const void *fn = packed ? (const void *)k_huygens_x2<RED, P> : (const void *)k_huygens<RED, P>;
    int per_sm = 0;
    const sincos_plan p = fit_plan(fn, plan, &per_sm);
    if (per_sm <= 0) return SINCOS_EUNSUPPORTED;
    const int64_t per_cta = (int64_t)p.block * P;
    const int64_t grid = (m + per_cta - 1) / per_cta;
    if (grid > 0x7fffffff) return SINCOS_EUNSUPPORTED;
    if (packed)
        k_huygens_x2<RED, P><<<(unsigned)grid, p.block, 0, st>>>(px, py, pz, m, qx, qy, qz, ar,
                                                                  ai, n, k, u);
    else
        k_huygens<RED, P><<<(unsigned)grid, p.block, 0, st>>>(px, py, pz, m, qx, qy, qz, ar, ai,
                                                               n, k, u);
    return check_launch("huygens kernel launch");
}

template <int RED>
static int launch_huygens_r(const float *px, const float *py, const float *pz, int64_t m,
                            const float *qx, const float *qy, const float *qz, const float *ar,
                            const float *ai, int64_t n, float k, float *u,
                            const sincos_plan &plan, cudaStream_t st)
{
    switch (plan.unroll) {
    case 1: return launch_huygens_p<RED, 1>(px, py, pz, m, qx, qy, qz, ar, ai, n, k, u, plan, st);
    case 2: return launch_huygens_p<RED, 2>(px, py, pz, m, qx, qy, qz, ar, ai, n, k, u, plan, st);
    default: return launch_huygens_p<RED, 4>(px, py, pz, m, qx, qy, qz, ar, ai, n, k, u, plan, st);
    }
}

int launch_huygens(const float *px, const float *py, const float *pz, int64_t m,
                   const float *qx, const float *qy, const float *qz, const float *ar,
                   const float *ai, int64_t n, float k, int red, float *u,
                   const sincos_plan &plan, cudaStream_t st)
{
    if (red == RED_COMPENSATED)
        return launch_huygens_r<RED_COMPENSATED>(px, py, pz, m, qx, qy, qz, ar, ai, n, k, u, plan,
                                                 st);
    return launch_huygens_r<RED_PLAIN>(px, py, pz, m, qx, qy, qz, ar, ai, n, k, u, plan, st);
}

}  // namespace sincos_gb300

using namespace sincos_gb300;

namespace {

// Whether cnt floats at `in` share a byte with the m complex64 outputs at u.
bool overlaps_output(const float *in, int64_t cnt, const float *u, int64_t m)
{
    return ranges_overlap(in, 4u * (size_t)cnt, u, 8u * (size_t)m);
}

int huygens_check(const float *px, const float *py, const float *pz, int64_t m,
                  const float *qx, const float *qy, const float *qz, const float *ar,
                  const float *ai, int64_t n, int reduction, float *u)
{
    if (m < 0 || n < 0 || !valid_reduction(reduction)) return SINCOS_EINVAL;
    if (m == 0) return SINCOS_OK;
    if (!px || !py || !pz || !u) return SINCOS_EINVAL;
    if (n > 0 && (!qx || !qy || !qz || !ar || !ai)) return SINCOS_EINVAL;
    if (!all_float_aligned({px, py, pz, qx, qy, qz, ar, ai, u})) return SINCOS_EINVAL;
    for (const float *p : {px, py, pz})
        if (overlaps_output(p, m, u, m)) return SINCOS_EOVERLAP;
    if (n > 0)
        for (const float *q : {qx, qy, qz, ar, ai})
            if (overlaps_output(q, n, u, m)) return SINCOS_EOVERLAP;
    return 1;   // valid, work to do
}

}  // namespace

extern "C" int sincos_huygens(const float *px, const float *py, const float *pz, int64_t m,
                              const float *qx, const float *qy, const float *qz,
                              const float *ar, const float *ai, int64_t n, float k,
                              int reduction, float *u, sincos_stream_t stream)
{
    SINCOS_TRACE("sincos_huygens");
    int rc = huygens_check(px, py, pz, m, qx, qy, qz, ar, ai, n, reduction, u);
    if (rc != 1) return rc;
    const DeviceInfo *dev = nullptr;
    rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    const sincos_plan plan = plan_for(*dev, SINCOS_OP_HUYGENS, SINCOS_F32, m);
    return launch_huygens(px, py, pz, m, qx, qy, qz, ar, ai, n, k, reduction, u, plan,
                          (cudaStream_t)stream);
}
