// core_x2.cuh -- two sine-cosine pairs at once on Blackwell's packed binary32
// pipe (FFMA2 / FMUL2 / FADD2: one instruction, two correctly rounded
// operations, each component numerically the same as __fmaf_rn, __fmul_rn,
// __fadd_rn).  The result of pair_x2 on (x0, x1) is, bit for bit, the result
// of pair (core.cuh) on x0 and on x1: the expression tree of Sec.
// Methodology, Eq. (1) and Fig. 1 is unchanged; signs are moved only by
// identities that hold exactly in binary32 round-to-nearest-even:
//   a - b           = a + (-b)                  (IEEE 754 defines it so)
//   -rint(v)        = rint(-v)                  (ties to even is symmetric)
//   -(a * b)        = (-a) * b                  (exact, signs of zero too)
//   -fma(a, b, c)   = fma(a, b, -c) with a*b negated   (RN is symmetric;
//                     used only where the exact result cannot be zero, the
//                     one case where the sign of a cancelled sum differs)
// The packed instructions take no negated operands, so the steps whose
// operands carry a sign (the differences of squares and the final products)
// run as scalar instructions, where the sign is free.
// Used by the Huygens kernel (bound by the FMA pipe) and by the bulk
// kernels' binary32 tiles, with either coefficient set (shorter compute phase
// between memory stages).
#pragma once

#include "core.cuh"

namespace sincos_gb300 {

__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

// Reduced angle in revolutions of two angles, as reduce<RED> of each.
template <int RED>
__device__ __forceinline__ float2 reduce_x2(float2 x)
{
    const float2 x1 = __fmul2_rn(x, splat2(kInvTwoPi));
    const float2 nr = make_float2(rintf(-x1.x), rintf(-x1.y));      // -rint(x1)
    if (RED == RED_PLAIN) return __fadd2_rn(x1, nr);                 // x1 - rint(x1)
    float2 q = __ffma2_rn(x, splat2(kInvTwoPi), nr);                 // fma(x, Khi, -r)
    q = __ffma2_rn(x, splat2(kInvTwoPiLo), q);
    return __fadd2_rn(q, make_float2(rintf(-q.x), rintf(-q.y)));    // q - rint(q)
}

// Two pairs, either coefficient set.
template <int RED, int COEF>
__device__ __forceinline__ void pair_x2(float2 x, float2 &s, float2 &c)
{
    using S = Series<COEF>;
    const float2 q1 = reduce_x2<RED>(x);
    const float2 q2 = __fmul2_rn(q1, q1);
    const float2 s1 = __fmul2_rn(
        q1, __ffma2_rn(q2, __ffma2_rn(q2, __ffma2_rn(q2, splat2(S::ss4), splat2(S::ss3)),
                                      splat2(S::ss2)),
                       splat2(S::ss1)));
    const float2 c1 = __ffma2_rn(
        q2, __ffma2_rn(q2, __ffma2_rn(q2, splat2(S::cc3), splat2(S::cc2)), splat2(S::cc1)),
        splat2(1.0f));
    // Eq. (1), first doubling: c2 = fma(-s1, s1, c1*c1), s2 = 2 (s1 c1).  The
    // fmas with a negated operand stay scalar, where the sign is an operand
    // modifier: packed, it would take a multiply by -1 on the same pipe.
    const float2 c1c1 = __fmul2_rn(c1, c1);
    const float2 c2 = make_float2(__fmaf_rn(-s1.x, s1.x, c1c1.x), __fmaf_rn(-s1.y, s1.y, c1c1.y));
    const float2 s2 = __fmul2_rn(splat2(2.0f), __fmul2_rn(s1, c1));
    const float2 c2c2 = __fmul2_rn(c2, c2);
    if constexpr (COEF == COEF_DAGGER) {
        // Drift factor 1/fma(s2, s2, c2^2): the sum on the packed pipe, the
        // IEEE reciprocals scalar; then the second doubling and the
        // correction, the products with fix packed (no sign to move).
        const float2 d = __ffma2_rn(s2, s2, c2c2);
        const float2 fix = make_float2(__frcp_rn(d.x), __frcp_rn(d.y));
        const float2 c3 =
            make_float2(__fmaf_rn(-s2.x, s2.x, c2c2.x), __fmaf_rn(-s2.y, s2.y, c2c2.y));
        const float2 s3 = __fmul2_rn(splat2(2.0f), __fmul2_rn(s2, c2));
        c = __fmul2_rn(c3, fix);
        s = __fmul2_rn(s3, fix);
    } else {
        // Drift factor fma(-s2, s2, fma(-c2, c2, 2)), computed as its
        // negation nfix = fma(s2, s2, fma(c2, c2, -2)); neither fma can cancel
        // to zero, since c2^2 and s2^2 are at most about 1.
        const float2 nfix = __ffma2_rn(s2, s2, __ffma2_rn(c2, c2, splat2(-2.0f)));
        // Eq. (1), second doubling, then the correction (times -nfix = fix).
        const float2 c3 =
            make_float2(__fmaf_rn(-s2.x, s2.x, c2c2.x), __fmaf_rn(-s2.y, s2.y, c2c2.y));
        const float2 s3 = __fmul2_rn(splat2(2.0f), __fmul2_rn(s2, c2));
        c = make_float2(__fmul_rn(c3.x, -nfix.x), __fmul_rn(c3.y, -nfix.y));
        s = make_float2(__fmul_rn(s3.x, -nfix.x), __fmul_rn(s3.y, -nfix.y));
    }
}

}  // namespace sincos_gb300
