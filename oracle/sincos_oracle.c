/*
 * sincos_oracle.c -- CPU oracle for the branch-free single-precision
 * sine-cosine pair method of M. H. Mendenhall, "A Fast, Vectorizable
 * Algorithm for Producing Single-Precision Sine-Cosine Pairs" (cs/0406049).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, constant or helper with the CUDA library.
 *
 * Arithmetic: IEEE-754 binary32 throughout, as the paper defines the method
 * (Section "Methodology").  Every place where the paper's Fig. 1 uses a fused
 * AltiVec multiply-add (vec_madd / vec_nmsub) with a non-zero addend, this
 * file uses fmaf(); where the addend is +0.0 it uses a plain rounded multiply
 * (the only difference is the sign of an exact zero).  The file must be
 * compiled with -ffp-contract=off and without -ffast-math so that the C
 * compiler neither fuses nor reorders any of these operations.
 *
 * Parity status: every function here is pinned by the CPU tests against
 * values the paper prints, closed forms, invariants or an FP64 brute force
 * (see the test files that import this oracle).  No function is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------------ */
/* Constants.                                                                */
/* ------------------------------------------------------------------------ */

/* Scale factor 1/(2*pi) as the paper writes it in Fig. 1 (the decimal value
 * 3.1415926536 for pi), rounded once to binary32. */
#define ORC_K ((float)(1.0 / (2.0 * 3.1415926536)))

/* Normalized ("20031003") coefficient set, Section "Methodology", first
 * method: sin(pi*q/2) ~ q*(ss1 + ss2 q^2 + ss3 q^4 + ss4 q^6) and
 * cos(pi*q/2) ~ 1 + cc1 q^2 + cc2 q^4 + cc3 q^6, each rounded to binary32. */
static const float NORM_SS1 = (float)1.5707963235;
static const float NORM_SS2 = (float)-0.645963615;
static const float NORM_SS3 = (float)0.0796819754;
static const float NORM_SS4 = (float)-0.0046075748;
static const float NORM_CC1 = (float)-1.2336977925;
static const float NORM_CC2 = (float)0.2536086171;
static const float NORM_CC3 = (float)-0.0204391631;

/* Un-normalized "dagger" coefficient set, Section "Methodology", second
 * method (fit to arctan(s/c)).  ss2 is taken from the displayed equation
 * (-0.6466386936); the figure prints -0.6466386396, a digit transposition
 * whose reading is recorded in the design notes. */
static const float DAG_SS1 = (float)1.5707963268;
static const float DAG_SS2 = (float)-0.6466386936;
static const float DAG_SS3 = (float)0.0679105987;
static const float DAG_SS4 = (float)-0.0011573807;
static const float DAG_CC1 = (float)-1.2341299769;
static const float DAG_CC2 = (float)0.2465220241;
static const float DAG_CC3 = (float)-0.0123926179;

enum { ORC_RED_PLAIN = 0, ORC_RED_COMPENSATED = 1 };
enum { ORC_COEF_NORMALIZED = 0, ORC_COEF_DAGGER = 1 };

/* ------------------------------------------------------------------------ */
/* Range reduction, Section "Methodology": scale by 1/(2 pi) and reduce onto  */
/* [-1/2, 1/2] by rounding and subtraction.                                  */
/* ------------------------------------------------------------------------ */

/* Plain reduction (the paper's): x1 = x*K; q1 = x1 - round(x1).  Rounding is
 * to nearest with ties to even, which is what AltiVec vec_round does and what
 * rintf() does in the default rounding mode. */
static float reduce_plain(float x)
{
    float x1 = x * ORC_K;
    float r = rintf(x1);
    return x1 - r;
}

/* Compensated reduction (not in the paper; an accuracy extension for large
 * |x|).  1/(2 pi) is split as Khi + Klo with Khi = K and Klo the binary32
 * rounding of (1/(2 pi) - Khi) computed in double with the C library's pi.
 *   r  = round(x*Khi)
 *   q  = fma(x, Khi, -r)        -- x*Khi - r with one rounding
 *   q  = fma(x, Klo, q)         -- add the low part of the product
 *   q1 = q - round(q)           -- wrap back onto [-1/2, 1/2]
 * The last wrap is a no-op for |x| up to about 1e6 and keeps the result a
 * finite unit pair for every finite x beyond. */
static float reduce_compensated(float x)
{
    const double two_pi = 6.283185307179586476925286766559;
    const float khi = ORC_K;
    const float klo = (float)(1.0 / two_pi - (double)khi);
    float x1 = x * khi;
    float r = rintf(x1);
    float q = fmaf(x, khi, -r);
    q = fmaf(x, klo, q);
    return q - rintf(q);
}

/* ------------------------------------------------------------------------ */
/* One sine-cosine pair, Section "Methodology" and Fig. 1.                   */
/* ------------------------------------------------------------------------ */

static void orc_pair(float x, int reduction, int coef, float *s_out, float *c_out)
{
    float ss1, ss2, ss3, ss4, cc1, cc2, cc3;
    if (coef == ORC_COEF_DAGGER) {
        ss1 = DAG_SS1; ss2 = DAG_SS2; ss3 = DAG_SS3; ss4 = DAG_SS4;
        cc1 = DAG_CC1; cc2 = DAG_CC2; cc3 = DAG_CC3;
    } else {
        ss1 = NORM_SS1; ss2 = NORM_SS2; ss3 = NORM_SS3; ss4 = NORM_SS4;
        cc1 = NORM_CC1; cc2 = NORM_CC2; cc3 = NORM_CC3;
    }

    /* Reduced angle q1 in revolutions and its square. */
    float q1 = (reduction == ORC_RED_COMPENSATED) ? reduce_compensated(x)
                                                  : reduce_plain(x);
    float q2 = q1 * q1;

    /* Quarter-angle pair: s1 ~ sin(pi q1 / 2), c1 ~ cos(pi q1 / 2), each a
     * Horner evaluation in q2 of the series printed in the paper. */
    float s1 = q1 * fmaf(q2, fmaf(q2, fmaf(q2, ss4, ss3), ss2), ss1);
    float c1 = fmaf(q2, fmaf(q2, fmaf(q2, cc3, cc2), cc1), 1.0f);

    /* First angle doubling, Eq. (1): c' = c^2 - s^2, s' = 2 s c. */
    float c2 = fmaf(-s1, s1, c1 * c1);
    float s2 = 2.0f * (s1 * c1);

    /* Amplitude correction factor, taken from the half-angle pair (s2, c2)
     * as in Fig. 1.  Normalized set: if (s2, c2) has magnitude squared 1+e,
     * the next doubling has magnitude 1+e as well, so multiplying by
     * 2 - s2^2 - c2^2 = 1 - e removes the drift to first order.  Dagger set:
     * the magnitude error is not small, so the exact reciprocal
     * 1/(s2^2 + c2^2) of the final pair's magnitude is used instead. */
    float fixmag;
    if (coef == ORC_COEF_DAGGER) {
        float mag2 = fmaf(s2, s2, c2 * c2);
        fixmag = 1.0f / mag2;
    } else {
        fixmag = fmaf(-s2, s2, fmaf(-c2, c2, 2.0f));
    }

    /* Second angle doubling, Eq. (1), reaching the full angle 2*pi*q1. */
    float c3 = fmaf(-s2, s2, c2 * c2);
    float s3 = 2.0f * (s2 * c2);

    /* Apply the correction to the final pair. */
    *c_out = c3 * fixmag;
    *s_out = s3 * fixmag;
}

/* ------------------------------------------------------------------------ */
/* Output rounding to 16-bit formats, written out bit by bit.                */
/* Round to nearest, ties to even, from binary32.                            */
/* ------------------------------------------------------------------------ */

uint16_t oracle_f32_to_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    if ((u & 0x7fffffffu) > 0x7f800000u)          /* NaN: keep it a quiet NaN */
        return (uint16_t)((u >> 16) | 0x0040u);
    uint32_t keep_lsb = (u >> 16) & 1u;            /* ties go to the even result */
    u += 0x7fffu + keep_lsb;
    return (uint16_t)(u >> 16);
}

uint16_t oracle_f32_to_f16(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    uint16_t sign = (uint16_t)((u >> 16) & 0x8000u);
    uint32_t a = u & 0x7fffffffu;

    if (a > 0x7f800000u)                           /* NaN */
        return (uint16_t)(sign | 0x7e00u);
    if (a >= 0x477ff000u)                          /* >= 65520 rounds to infinity */
        return (uint16_t)(sign | 0x7c00u);
    if (a >= 0x38800000u) {                        /* result is a normal half */
        uint32_t e = (a >> 23) - 127u + 15u;       /* 1 .. 30 */
        uint32_t mant = a & 0x7fffffu;
        uint32_t h = (e << 10) | (mant >> 13);
        uint32_t rem = mant & 0x1fffu;
        if (rem > 0x1000u || (rem == 0x1000u && (h & 1u)))
            h += 1u;                               /* a carry may bump the exponent */
        return (uint16_t)(sign | h);
    }
    /* Result is a subnormal half (unit 2^-24) or zero. */
    uint32_t e = a >> 23;
    if (e == 0u)                                   /* binary32 subnormals are < 2^-126 */
        return sign;
    uint32_t m = (a & 0x7fffffu) | 0x800000u;      /* value = m * 2^(e-150) */
    uint32_t shift = 126u - e;                     /* value / 2^-24 = m >> shift */
    if (shift > 24u)                               /* below half of 2^-24 */
        return sign;
    uint32_t h = m >> shift;
    uint32_t rem = m & ((1u << shift) - 1u);
    uint32_t halfway = 1u << (shift - 1u);
    if (rem > halfway || (rem == halfway && (h & 1u)))
        h += 1u;
    return (uint16_t)(sign | h);
}

/* ------------------------------------------------------------------------ */
/* Exported array entry points.                                              */
/* ------------------------------------------------------------------------ */

/* Forward, binary32 outputs: s[i], c[i] for i < n. */
void oracle_sincos_f32(const float *x, float *s, float *c, int64_t n,
                       int reduction, int coef)
{
    for (int64_t i = 0; i < n; ++i)
        orc_pair(x[i], reduction, coef, &s[i], &c[i]);
}

/* Forward with 16-bit outputs: the binary32 result rounded to bf16
 * (out16 = 1) or fp16 (out16 = 2), stored as raw 16-bit patterns. */
void oracle_sincos_16(const float *x, uint16_t *s, uint16_t *c, int64_t n,
                      int reduction, int coef, int out16)
{
    for (int64_t i = 0; i < n; ++i) {
        float sf, cf;
        orc_pair(x[i], reduction, coef, &sf, &cf);
        if (out16 == 1) {
            s[i] = oracle_f32_to_bf16(sf);
            c[i] = oracle_f32_to_bf16(cf);
        } else {
            s[i] = oracle_f32_to_f16(sf);
            c[i] = oracle_f32_to_f16(cf);
        }
    }
}

/* Array form of the two roundings above: kind 1 = bf16, kind 2 = fp16. */
void oracle_round_16(const float *v, uint16_t *out, int64_t n, int kind)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = (kind == 1) ? oracle_f32_to_bf16(v[i]) : oracle_f32_to_f16(v[i]);
}

/* Backward of (s, c) = (sin x, cos x):  d/dx [gs*sin x + gc*cos x]
 * = gs*cos x - gc*sin x, evaluated on the forward's own outputs:
 *   gx = fma(gs, c, -(gc*s)).
 * A null gs or gc stands for an all-zero gradient:
 *   gs == NULL  ->  gx = -(gc*s)
 *   gc == NULL  ->  gx = gs*c
 *   both NULL   ->  gx = +0. */
void oracle_sincos_backward(const float *gs, const float *gc, const float *s,
                            const float *c, float *gx, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        if (gs && gc)
            gx[i] = fmaf(gs[i], c[i], -(gc[i] * s[i]));
        else if (gc)
            gx[i] = -(gc[i] * s[i]);
        else if (gs)
            gx[i] = gs[i] * c[i];
        else
            gx[i] = 0.0f;
    }
}

/* ------------------------------------------------------------------------ */
/* Huygens-principle field sum (Sec. Conclusions: the method's application  */
/* to optical diffraction), with the phase factor of every source-point     */
/* pair produced by the method.  For observation point i and sources j:     */
/*   dx = px_i - qx_j, dy, dz likewise                                       */
/*   r  = sqrt(fma(dz, dz, fma(dy, dy, dx*dx)))      (correctly rounded)     */
/*   w  = 1 / r                                      (correctly rounded)     */
/*   (s, c) = the method's pair of theta = k * r     (given reduction)       */
/*   pr = fma(ar_j, c, -(ai_j * s)),  pi = fma(ar_j, s, ai_j * c)            */
/*   u_re = fma(w, pr, u_re),  u_im = fma(w, pi, u_im)                       */
/* summed over j = 0, 1, ..., n-1 in that order from u = 0, in binary32.     */
/* Result: u[2i] = u_re, u[2i+1] = u_im, i.e. sum_j a_j exp(i k r_ij) / r_ij.*/
/* ------------------------------------------------------------------------ */

void oracle_huygens(const float *px, const float *py, const float *pz, int64_t m,
                    const float *qx, const float *qy, const float *qz, const float *ar,
                    const float *ai, int64_t n, float k, int reduction, float *u)
{
    for (int64_t i = 0; i < m; ++i) {
        float ure = 0.0f, uim = 0.0f;
        for (int64_t j = 0; j < n; ++j) {
            float dx = px[i] - qx[j];
            float dy = py[i] - qy[j];
            float dz = pz[i] - qz[j];
            float r = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            float w = 1.0f / r;
            float s, c;
            orc_pair(k * r, reduction, ORC_COEF_NORMALIZED, &s, &c);
            float pr = fmaf(ar[j], c, -(ai[j] * s));
            float pi = fmaf(ar[j], s, ai[j] * c);
            ure = fmaf(w, pr, ure);
            uim = fmaf(w, pi, uim);
        }
        u[2 * i] = ure;
        u[2 * i + 1] = uim;
    }
}

/* ------------------------------------------------------------------------ */
/* Threaded driver, used only to time the oracle as a CPU baseline: a static */
/* contiguous split of [0, n) over nthreads POSIX threads.                   */
/* ------------------------------------------------------------------------ */

struct orc_job {
    const float *x;
    float *s, *c;
    int64_t lo, hi;
    int reduction, coef;
};

static void *orc_worker(void *arg)
{
    struct orc_job *j = (struct orc_job *)arg;
    oracle_sincos_f32(j->x + j->lo, j->s + j->lo, j->c + j->lo, j->hi - j->lo,
                      j->reduction, j->coef);
    return 0;
}

int oracle_sincos_f32_mt(const float *x, float *s, float *c, int64_t n,
                         int reduction, int coef, int nthreads)
{
    enum { MAXT = 512 };
    if (nthreads < 1) nthreads = 1;
    if (nthreads > MAXT) nthreads = MAXT;
    pthread_t tid[MAXT];
    int joined[MAXT];
    struct orc_job job[MAXT];
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        job[t].x = x; job[t].s = s; job[t].c = c;
        job[t].lo = n * t / nthreads;
        job[t].hi = n * (t + 1) / nthreads;
        job[t].reduction = reduction; job[t].coef = coef;
        joined[t] = pthread_create(&tid[t], 0, orc_worker, &job[t]) == 0;
        if (joined[t])
            ++started;
        else
            orc_worker(&job[t]);     /* could not spawn: run inline */
    }
    for (int t = 0; t < nthreads; ++t)
        if (joined[t]) pthread_join(tid[t], 0);
    return started;
}
