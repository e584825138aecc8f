// core.cuh -- per-element arithmetic of the sine-cosine pair method and the
// 16-byte streaming I/O used by every kernel of the library.
//
// Method: M. H. Mendenhall, "A Fast, Vectorizable Algorithm for Producing
// Single-Precision Sine-Cosine Pairs" (cs/0406049), Sec. Methodology, Eq. (1)
// and Fig. 1.  Every operation is an explicitly rounded binary32 intrinsic
// (__fmul_rn, __fmaf_rn, ...), and the library is built with -fmad=false
// -ftz=false, so the compiler neither fuses, reorders nor flushes anything:
// the kernels produce the same bits as a straight IEEE-754 binary32
// evaluation of the same expression tree.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace sincos_gb300 {

enum { RED_PLAIN = 0, RED_COMPENSATED = 1 };
enum { COEF_NORMALIZED = 0, COEF_DAGGER = 1 };

// Quarter-angle series coefficients, each the binary32 rounding of the
// decimal the paper prints (Sec. Methodology).
template <int COEF> struct Series;

// First method ("20031003" normalized set): least-squares sine and cosine.
template <> struct Series<COEF_NORMALIZED> {
    static constexpr float ss1 = (float)1.5707963235;
    static constexpr float ss2 = (float)-0.645963615;
    static constexpr float ss3 = (float)0.0796819754;
    static constexpr float ss4 = (float)-0.0046075748;
    static constexpr float cc1 = (float)-1.2336977925;
    static constexpr float cc2 = (float)0.2536086171;
    static constexpr float cc3 = (float)-0.0204391631;
};

// Second method (dagger set, fit to arctan(s/c)); ss2 as in the displayed
// equation, -0.6466386936.
template <> struct Series<COEF_DAGGER> {
    static constexpr float ss1 = (float)1.5707963268;
    static constexpr float ss2 = (float)-0.6466386936;
    static constexpr float ss3 = (float)0.0679105987;
    static constexpr float ss4 = (float)-0.0011573807;
    static constexpr float cc1 = (float)-1.2341299769;
    static constexpr float cc2 = (float)0.2465220241;
    static constexpr float cc3 = (float)-0.0123926179;
};

// 1/(2 pi) with the paper's decimal pi, rounded once to binary32.
constexpr float kInvTwoPi = (float)(1.0 / (2.0 * 3.1415926536));
// Low part of the two-constant split of 1/(2 pi): binary32 rounding of
// (1/(2 pi) - kInvTwoPi), evaluated in double.
constexpr float kInvTwoPiLo = (float)(1.0 / 6.283185307179586476925286766559 - (double)kInvTwoPi);

// Reduced angle in revolutions, in [-1/2, 1/2].
template <int RED>
__device__ __forceinline__ float reduce(float x)
{
    if (RED == RED_PLAIN) {
        // Sec. Methodology: scale by 1/(2 pi), subtract the nearest integer
        // (rintf: ties to even, as AltiVec vec_round).
        const float x1 = __fmul_rn(x, kInvTwoPi);
        return __fsub_rn(x1, rintf(x1));
    } else {
        // Two-constant split: the fma keeps the low bits of x*Khi - r, the
        // second adds x*Klo, the last subtraction wraps back onto [-1/2, 1/2].
        const float x1 = __fmul_rn(x, kInvTwoPi);
        const float r = rintf(x1);
        float q = __fmaf_rn(x, kInvTwoPi, -r);
        q = __fmaf_rn(x, kInvTwoPiLo, q);
        return __fsub_rn(q, rintf(q));
    }
}

// One sine-cosine pair.
template <int RED, int COEF>
__device__ __forceinline__ void pair(float x, float &s, float &c)
{
    using S = Series<COEF>;
    const float q1 = reduce<RED>(x);
    const float q2 = __fmul_rn(q1, q1);
    // Quarter-angle pair: sin(pi q1 / 2) and cos(pi q1 / 2), Horner in q2.
    const float s1 = __fmul_rn(q1, __fmaf_rn(q2, __fmaf_rn(q2, __fmaf_rn(q2, S::ss4, S::ss3),
                                                            S::ss2), S::ss1));
    const float c1 = __fmaf_rn(q2, __fmaf_rn(q2, __fmaf_rn(q2, S::cc3, S::cc2), S::cc1), 1.0f);
    // Eq. (1), first doubling: c2 = c1^2 - s1^2, s2 = 2 s1 c1.
    const float c2 = __fmaf_rn(-s1, s1, __fmul_rn(c1, c1));
    const float s2 = __fmul_rn(2.0f, __fmul_rn(s1, c1));
    // Drift factor from the half-angle pair (Fig. 1): 2 - c2^2 - s2^2 for the
    // normalized set, the exact reciprocal 1/(s2^2 + c2^2) for the dagger set.
    float fix;
    if (COEF == COEF_DAGGER)
        fix = __frcp_rn(__fmaf_rn(s2, s2, __fmul_rn(c2, c2)));
    else
        fix = __fmaf_rn(-s2, s2, __fmaf_rn(-c2, c2, 2.0f));
    // Eq. (1), second doubling, then the correction.
    const float c3 = __fmaf_rn(-s2, s2, __fmul_rn(c2, c2));
    const float s3 = __fmul_rn(2.0f, __fmul_rn(s2, c2));
    c = __fmul_rn(c3, fix);
    s = __fmul_rn(s3, fix);
}

// ---------------------------------------------------------------------------
// Output element types.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void store_elem(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_elem(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_elem(__half *p, float v) { *p = __float2half_rn(v); }

// Two binary32 values rounded (nearest even) and packed into one 32-bit word,
// the first at the lower address.
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 *, float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack2(__half *, float lo, float hi)
{
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// ---------------------------------------------------------------------------
// Vector global memory access.  A thread moves W = 16 or 32 bytes of output
// per vector (one st.v4 or one 256-bit st.v8), i.e. E = W / sizeof(OutT)
// pairs, reading their 4E bytes of angles with 16- or 32-byte loads.
//   loads   ld.global.nc.L1::no_allocate: every byte is used once, so no L1
//           allocation; the non-coherent path is used only when the kernel
//           does not write the input (LD_COHERENT otherwise).
//   stores  16-byte: st.global.cs (evict-first streaming store);
//           32-byte: st.global.L1::no_allocate.L2::evict_first.v8 -- the
//           256-bit form that sm_100-class GPUs accept with an L2 eviction
//           priority, so the output stream leaves L2 first.
// ---------------------------------------------------------------------------

enum { LD_NC = 0, LD_COHERENT = 1 };

template <int LD>
__device__ __forceinline__ void ld16(float *d, const float *p)
{
    if (LD == LD_NC)
        asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]) : "l"(p));
    else
        asm("ld.global.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]) : "l"(p));
}

template <int LD>
__device__ __forceinline__ void ld32(float *d, const float *p)
{
    if (LD == LD_NC)
        asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]), "=f"(d[4]), "=f"(d[5]),
              "=f"(d[6]), "=f"(d[7]) : "l"(p));
    else
        asm("ld.global.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]), "=f"(d[4]), "=f"(d[5]),
              "=f"(d[6]), "=f"(d[7]) : "l"(p));
}

// NB bytes of binary32 values (16, 32 or 64) into d[0 .. NB/4).
template <int NB, int LD>
__device__ __forceinline__ void load_f32(float *d, const float *p)
{
    if constexpr (NB == 16) {
        ld16<LD>(d, p);
    } else {
#pragma unroll
        for (int k = 0; k < NB / 32; ++k) ld32<LD>(d + 8 * k, p + 8 * k);
    }
}

template <int W>
__device__ __forceinline__ void store_words(void *p, const uint32_t *w)
{
    if constexpr (W == 16)
        asm volatile("st.global.cs.v4.b32 [%0], {%1,%2,%3,%4};"
                     :: "l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]));
    else
        asm volatile("st.global.L1::no_allocate.L2::evict_first.v8.b32 [%0], "
                     "{%1,%2,%3,%4,%5,%6,%7,%8};"
                     :: "l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]),
                        "r"(w[5]), "r"(w[6]), "r"(w[7]));
}

// Pairs per vector for an output type and access width.
template <class OutT, int W>
struct Vec {
    static constexpr int E = W / (int)sizeof(OutT);        // pairs per vector
    static constexpr int IN_BYTES = 4 * E;                 // angle bytes per vector
    static constexpr int IN_ALIGN = IN_BYTES < 32 ? IN_BYTES : 32;
};

template <class OutT, int W, int LD>
__device__ __forceinline__ void load_vec(float *in, const float *x)
{
    load_f32<Vec<OutT, W>::IN_BYTES, LD>(in, x);
}

// The pairs of one vector of angles, stored as one W-byte vector of sines
// and one of cosines.
template <int RED, int COEF, class OutT, int W>
__device__ __forceinline__ void compute_store(const float *in, OutT *s, OutT *c)
{
    constexpr int E = Vec<OutT, W>::E;
    float sv[E], cv[E];
#pragma unroll
    for (int i = 0; i < E; ++i) pair<RED, COEF>(in[i], sv[i], cv[i]);
    uint32_t ws[W / 4], wc[W / 4];
    if constexpr (sizeof(OutT) == 4) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            ws[i] = __float_as_uint(sv[i]);
            wc[i] = __float_as_uint(cv[i]);
        }
    } else {
        OutT *tag = nullptr;
#pragma unroll
        for (int k = 0; k < W / 4; ++k) {
            ws[k] = pack2(tag, sv[2 * k], sv[2 * k + 1]);
            wc[k] = pack2(tag, cv[2 * k], cv[2 * k + 1]);
        }
    }
    store_words<W>(s, ws);
    store_words<W>(c, wc);
}

template <int RED, int COEF, class OutT>
__device__ __forceinline__ void scalar_elem(const float *x, OutT *s, OutT *c, int64_t i)
{
    float sv, cv;
    pair<RED, COEF>(x[i], sv, cv);
    store_elem(s + i, sv);
    store_elem(c + i, cv);
}

// Smallest h in [0, E) such that x + h meets the angle loads' alignment and
// s + h, c + h are W-byte aligned, or -1 if the three pointers admit no
// common vector alignment.
template <class OutT, int W>
__host__ __device__ __forceinline__ int vector_w_head(const void *x, const void *s, const void *c)
{
    using V = Vec<OutT, W>;
    const uintptr_t ax = (uintptr_t)x, as = (uintptr_t)s, ac = (uintptr_t)c;
    for (int h = 0; h < V::E; ++h) {
        if (((ax + 4u * h) % V::IN_ALIGN) == 0 && ((as + sizeof(OutT) * h) % W) == 0 &&
            ((ac + sizeof(OutT) * h) % W) == 0)
            return h;
    }
    return -1;
}

// Smallest h such that x + h, s + h and c + h all start a 128-byte L2 line,
// or -1 if their offsets within a line differ.  Starting the vector grid on
// line boundaries means every warp-wide vector store covers whole lines, so
// no line is written in two halves by different warps at different times.
template <class OutT>
__host__ __device__ __forceinline__ int line_head(const void *x, const void *s, const void *c)
{
    constexpr unsigned osz = sizeof(OutT);
    const unsigned ax = (unsigned)((uintptr_t)x & 127u);
    const unsigned as = (unsigned)((uintptr_t)s & 127u);
    const unsigned ac = (unsigned)((uintptr_t)c & 127u);
    if ((ax & 3u) || (as % osz) || (ac % osz)) return -1;
    const unsigned hs = ((128u - as) & 127u) / osz;
    const unsigned hc = ((128u - ac) & 127u) / osz;
    const unsigned hx = ((128u - ax) & 127u) / 4u;        // h = hx (mod 32)
    if (hs != hc || (hs & 31u) != hx) return -1;
    return (int)hs;
}

// Where the vector grid of an array triple starts: on a 128-byte line if the
// three pointers allow it (h < 128 / sizeof(OutT)), else at the first W-byte
// vector boundary (h < E), else -1 (no common vector alignment).
template <class OutT, int W>
__host__ __device__ __forceinline__ int vector_head(const void *x, const void *s, const void *c)
{
    const int h = line_head<OutT>(x, s, c);
    return h >= 0 ? h : vector_w_head<OutT, W>(x, s, c);
}

}  // namespace sincos_gb300
