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

template <class OutT> struct Out;
template <> struct Out<float> {
    static constexpr int kVec = 4;   // elements per 16-byte output vector
};
template <> struct Out<__nv_bfloat16> {
    static constexpr int kVec = 8;
};
template <> struct Out<__half> {
    static constexpr int kVec = 8;
};

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
// 16-byte global memory access.  Loads bypass L1 allocation (every byte is
// used once); stores are marked evict-first (.cs) so the output stream does
// not push the input out of L2.
// ---------------------------------------------------------------------------

enum { LD_NC = 0, LD_COHERENT = 1 };

template <int LD>
__device__ __forceinline__ float4 ld16(const float *p)
{
    float4 v;
    if (LD == LD_NC)
        asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
            : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    else
        asm("ld.global.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
            : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ void st16(void *p, float a, float b, float c, float d)
{
    asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};"
                 :: "l"(p), "f"(a), "f"(b), "f"(c), "f"(d));
}

__device__ __forceinline__ void st16u(void *p, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.global.cs.v4.b32 [%0], {%1,%2,%3,%4};"
                 :: "l"(p), "r"(a), "r"(b), "r"(c), "r"(d));
}

// ---------------------------------------------------------------------------
// One output vector: Out<OutT>::kVec angles in (one or two 16-byte loads),
// the same number of sines and cosines out (one 16-byte store each).
// ---------------------------------------------------------------------------

template <class OutT> struct InVec;
template <> struct InVec<float> { float4 a; };
template <> struct InVec<__nv_bfloat16> { float4 a, b; };
template <> struct InVec<__half> { float4 a, b; };

template <int LD>
__device__ __forceinline__ void load_vec(InVec<float> &v, const float *x) { v.a = ld16<LD>(x); }
template <int LD>
__device__ __forceinline__ void load_vec(InVec<__nv_bfloat16> &v, const float *x)
{
    v.a = ld16<LD>(x);
    v.b = ld16<LD>(x + 4);
}
template <int LD>
__device__ __forceinline__ void load_vec(InVec<__half> &v, const float *x)
{
    v.a = ld16<LD>(x);
    v.b = ld16<LD>(x + 4);
}

// Compute the pairs of one input vector and store one 16-byte vector of
// sines and one of cosines.
template <int RED, int COEF, class OutT>
__device__ __forceinline__ void compute_store(const InVec<OutT> &v, OutT *s, OutT *c)
{
    if constexpr (Out<OutT>::kVec == 4) {
        float s0, s1, s2, s3, c0, c1, c2, c3;
        pair<RED, COEF>(v.a.x, s0, c0);
        pair<RED, COEF>(v.a.y, s1, c1);
        pair<RED, COEF>(v.a.z, s2, c2);
        pair<RED, COEF>(v.a.w, s3, c3);
        st16(s, s0, s1, s2, s3);
        st16(c, c0, c1, c2, c3);
    } else {
        float sv[8], cv[8];
        pair<RED, COEF>(v.a.x, sv[0], cv[0]);
        pair<RED, COEF>(v.a.y, sv[1], cv[1]);
        pair<RED, COEF>(v.a.z, sv[2], cv[2]);
        pair<RED, COEF>(v.a.w, sv[3], cv[3]);
        pair<RED, COEF>(v.b.x, sv[4], cv[4]);
        pair<RED, COEF>(v.b.y, sv[5], cv[5]);
        pair<RED, COEF>(v.b.z, sv[6], cv[6]);
        pair<RED, COEF>(v.b.w, sv[7], cv[7]);
        OutT *tag = nullptr;
        st16u(s, pack2(tag, sv[0], sv[1]), pack2(tag, sv[2], sv[3]), pack2(tag, sv[4], sv[5]),
              pack2(tag, sv[6], sv[7]));
        st16u(c, pack2(tag, cv[0], cv[1]), pack2(tag, cv[2], cv[3]), pack2(tag, cv[4], cv[5]),
              pack2(tag, cv[6], cv[7]));
    }
}

template <int RED, int COEF, class OutT>
__device__ __forceinline__ void scalar_elem(const float *x, OutT *s, OutT *c, int64_t i)
{
    float sv, cv;
    pair<RED, COEF>(x[i], sv, cv);
    store_elem(s + i, sv);
    store_elem(c + i, cv);
}

// Smallest h in [0, kVec) such that x + h, s + h and c + h are all 16-byte
// aligned, or -1 if the three pointers admit no common vector alignment.
template <class OutT>
__host__ __device__ __forceinline__ int vector_head(const void *x, const void *s, const void *c)
{
    const uintptr_t ax = (uintptr_t)x, as = (uintptr_t)s, ac = (uintptr_t)c;
    for (int h = 0; h < Out<OutT>::kVec; ++h) {
        if (((ax + 4u * h) & 15u) == 0 && ((as + sizeof(OutT) * h) & 15u) == 0 &&
            ((ac + sizeof(OutT) * h) & 15u) == 0)
            return h;
    }
    return -1;
}

}  // namespace sincos_gb300
