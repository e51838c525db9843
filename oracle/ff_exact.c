/*
 * ff_exact.c -- exact references for the oracle's self-checks and for the
 * accuracy measurements of the float-float operators.
 *
 * TEST INFRASTRUCTURE ONLY (see ff_oracle.c).  No code here is shared with
 * the CUDA library.
 *
 * Two independent exact tools:
 *   1. A superaccumulator: a signed fixed-point integer wide enough to hold
 *      any sum of binary64 numbers exactly (bits 2^-1152 .. 2^1151), kept as
 *      32-bit digits in 64-bit signed limbs so additions never carry until
 *      an explicit normalisation.  Every product of two binary32 numbers is
 *      exact in binary64, so sums of float-float products (four binary32
 *      partial products each) are accumulated exactly, then rounded once.
 *   2. IEEE binary128 arithmetic (GCC _Float128, 113-bit significand) for
 *      quotients and square roots, which have no finite exact sum form; its
 *      relative error (2^-113) is far below the 2^-44 being measured.
 *
 * The paper measured errors against MPFR (Section 6.1); MPFR is not part of
 * this tool set, so these two stand in for it.
 */
#define _GNU_SOURCE
#define __STDC_WANT_IEC_60559_TYPES_EXT__
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#if defined(__FAST_MATH__)
#error "the oracle must not be compiled with -ffast-math"
#endif

#if defined(__LDBL_MANT_DIG__) && (__LDBL_MANT_DIG__ == 113)
typedef long double q128;
#define Q_SQRT sqrtl
#else
typedef _Float128 q128;
#define Q_SQRT sqrtf128
#endif

/* ------------------------------------------------------------------------ */
/* Superaccumulator                                                          */
/* ------------------------------------------------------------------------ */

#define SA_LOW (-1152)      /* weight of bit 0 of limb 0 is 2^SA_LOW        */
#define SA_NLIMB 72         /* 72 * 32 = 2304 bits: 2^-1152 .. 2^1151        */
#define SA_RENORM (1u << 28)

typedef struct {
    int64_t limb[SA_NLIMB];
    uint32_t pending;       /* additions since the last normalisation        */
    int lo, hi;             /* range of limbs touched since clearing          */
} sacc;

static void sa_clear(sacc *a)
{
    memset(a->limb, 0, sizeof(a->limb));
    a->pending = 0;
    a->lo = SA_NLIMB;
    a->hi = -1;
}

/* Carry-propagate so that limbs 0..N-2 lie in [0, 2^32) and the top limb
 * holds the sign. */
static void sa_normalize(sacc *a)
{
    if (a->hi < 0) {
        a->pending = 0;
        return;
    }
    int top = SA_NLIMB - 1;
    for (int k = a->lo; k < top; ++k) {
        int64_t c = a->limb[k] >> 32; /* arithmetic shift = floor division */
        a->limb[k] -= c * ((int64_t)1 << 32);
        a->limb[k + 1] += c;
        if (k + 1 > a->hi)
            a->hi = k + 1;
    }
    a->pending = 0;
}

static void sa_add_double(sacc *a, double d)
{
    if (d == 0.0)
        return;
    int e;
    double m = frexp(fabs(d), &e);         /* |d| = m 2^e, m in [0.5, 1)   */
    uint64_t mant = (uint64_t)ldexp(m, 53); /* exact: 53-bit integer       */
    int lsb = e - 53;                        /* |d| = mant * 2^lsb          */
    int p = lsb - SA_LOW;                    /* >= 0 for every double       */
    int k = p >> 5, sh = p & 31;
    unsigned __int128 v = (unsigned __int128)mant << sh; /* < 2^85           */
    int64_t d0 = (int64_t)(uint32_t)v;
    int64_t d1 = (int64_t)(uint32_t)(v >> 32);
    int64_t d2 = (int64_t)(uint32_t)(v >> 64);
    if (d < 0) {
        a->limb[k] -= d0;
        a->limb[k + 1] -= d1;
        a->limb[k + 2] -= d2;
    } else {
        a->limb[k] += d0;
        a->limb[k + 1] += d1;
        a->limb[k + 2] += d2;
    }
    if (k < a->lo)
        a->lo = k;
    if (k + 2 > a->hi)
        a->hi = k + 2;
    if (++a->pending >= SA_RENORM)
        sa_normalize(a);
}

/* Round the accumulated value to a binary floating-point number with `prec`
 * significand bits and least exponent `emin_lsb` (weight of the lowest
 * representable bit), round-to-nearest-even.  Returns the sign (-1, 0, +1),
 * the integer significand and the weight exponent of its lowest bit. */
static int sa_round(const sacc *src, int prec, int emin_lsb,
                    unsigned __int128 *mant_out, int *exp_out)
{
    sacc a = *src;
    sa_normalize(&a);
    int sign = 0;
    int top = -1;
    for (int k = SA_NLIMB - 1; k >= 0; --k)
        if (a.limb[k] != 0) {
            top = k;
            break;
        }
    if (top < 0) {
        *mant_out = 0;
        *exp_out = 0;
        return 0;
    }
    sign = (a.limb[SA_NLIMB - 1] < 0) ? -1 : 1;
    if (sign < 0) {
        for (int k = 0; k < SA_NLIMB; ++k)
            a.limb[k] = -a.limb[k];
        a.lo = 0;
        a.hi = SA_NLIMB - 1;
        sa_normalize(&a);
    }
    top = -1;
    for (int k = SA_NLIMB - 1; k >= 0; --k)
        if (a.limb[k] != 0) {
            top = k;
            break;
        }
    /* absolute bit index (from bit 0 of limb 0) of the leading one */
    uint64_t tl = (uint64_t)a.limb[top];
    int msb = 63;
    while (!((tl >> msb) & 1u))
        --msb;
    int P = top * 32 + msb;
    int lsb_idx = P - prec + 1;                   /* lowest kept bit index   */
    int min_idx = emin_lsb - SA_LOW;
    if (lsb_idx < min_idx)
        lsb_idx = min_idx;                        /* subnormal range         */
    /* gather kept bits [lsb_idx, P] */
    unsigned __int128 M = 0;
    for (int b = P; b >= lsb_idx; --b) {
        int idx = b;
        uint64_t bit = (idx < 0) ? 0 : (((uint64_t)a.limb[idx >> 5] >> (idx & 31)) & 1u);
        M = (M << 1) | bit;
    }
    int round_bit = 0, sticky = 0;
    int rb = lsb_idx - 1;
    if (rb >= 0) {
        round_bit = (int)(((uint64_t)a.limb[rb >> 5] >> (rb & 31)) & 1u);
        for (int b = rb - 1; b >= 0 && !sticky; --b) {
            if ((b & 31) == 31 && a.limb[b >> 5] == 0) {
                b -= 31;
                continue;
            }
            if (((uint64_t)a.limb[b >> 5] >> (b & 31)) & 1u)
                sticky = 1;
        }
    }
    if (round_bit && (sticky || (M & 1)))
        M += 1;
    *mant_out = M;
    *exp_out = lsb_idx + SA_LOW;
    return sign;
}

static q128 q_pow2(int e)
{
    q128 r = 1;
    const q128 two64 = (q128)18446744073709551616.0;
    while (e >= 64) {
        r *= two64;
        e -= 64;
    }
    while (e <= -64) {
        r /= two64;
        e += 64;
    }
    while (e > 0) {
        r *= 2;
        --e;
    }
    while (e < 0) {
        r /= 2;
        ++e;
    }
    return r;
}

static q128 sa_to_q128(const sacc *a)
{
    unsigned __int128 M;
    int e;
    int s = sa_round(a, 113, -16494, &M, &e);
    if (s == 0)
        return 0;
    q128 v = (q128)M * q_pow2(e); /* M < 2^114: exact; scaling exact      */
    return s < 0 ? -v : v;
}

static double sa_to_double(const sacc *a)
{
    unsigned __int128 M;
    int e;
    int s = sa_round(a, 53, -1074, &M, &e);
    if (s == 0)
        return 0.0;
    double v = ldexp((double)(uint64_t)M, e);
    return s < 0 ? -v : v;
}

/* ------------------------------------------------------------------------ */
/* Entry points                                                              */
/* ------------------------------------------------------------------------ */

/* Correctly rounded (RN) binary64 sum of n doubles. */
double exact_sum_f64(const double *v, size_t n)
{
    sacc a;
    sa_clear(&a);
    for (size_t i = 0; i < n; ++i)
        sa_add_double(&a, v[i]);
    return sa_to_double(&a);
}

/* The same sum rounded to binary128, returned as an unevaluated pair
 * (hi, lo) of doubles with hi = RN64(s) and lo = RN64(s - hi). */
void exact_sum_f64_q(const double *v, size_t n, double *out2)
{
    sacc a;
    sa_clear(&a);
    for (size_t i = 0; i < n; ++i)
        sa_add_double(&a, v[i]);
    q128 s = sa_to_q128(&a);
    double hi = (double)s;
    out2[0] = hi;
    out2[1] = (double)(s - (q128)hi);
}

/* Count of i where a_i + b_i != c_i + d_i exactly (all binary32).  Used for
 * the exactness of Add12 (a + b = s + r) and of Split (a + 0 = hi + lo). */
size_t exact_count_sum2_mismatch(const float *ab, const float *cd, size_t n)
{
    size_t bad = 0;
    sacc a;
    for (size_t i = 0; i < n; ++i) {
        sa_clear(&a);
        sa_add_double(&a, (double)ab[2 * i]);
        sa_add_double(&a, (double)ab[2 * i + 1]);
        sa_add_double(&a, -(double)cd[2 * i]);
        sa_add_double(&a, -(double)cd[2 * i + 1]);
        sa_normalize(&a);
        int nz = 0;
        for (int k = 0; k < SA_NLIMB; ++k)
            if (a.limb[k]) {
                nz = 1;
                break;
            }
        bad += (size_t)nz;
    }
    return bad;
}

/* Count of i where a_i * b_i != x_i + y_i exactly (Mul12 exactness). */
size_t exact_count_prod_mismatch(const float *ab, const float *xy, size_t n)
{
    size_t bad = 0;
    sacc a;
    for (size_t i = 0; i < n; ++i) {
        sa_clear(&a);
        sa_add_double(&a, (double)ab[2 * i] * (double)ab[2 * i + 1]); /* exact */
        sa_add_double(&a, -(double)xy[2 * i]);
        sa_add_double(&a, -(double)xy[2 * i + 1]);
        sa_normalize(&a);
        int nz = 0;
        for (int k = 0; k < SA_NLIMB; ++k)
            if (a.limb[k]) {
                nz = 1;
                break;
            }
        bad += (size_t)nz;
    }
    return bad;
}

/* Add22 bound (Add22 theorem): for each i writes three doubles
 *   out[3i]   = |delta|, delta = (rh + rl) - ((ah + al) + (bh + bl)) exactly,
 *   out[3i+1] = 2^-24 |al + bl|,
 *   out[3i+2] = 2^-44 |ah + al + bh + bl|,
 * each rounded once to binary64 from its exact value. */
void exact_add22_bound(const float *a, const float *b, const float *r, double *out, size_t n)
{
    sacc s;
    for (size_t i = 0; i < n; ++i) {
        double ah = a[2 * i], al = a[2 * i + 1], bh = b[2 * i], bl = b[2 * i + 1];
        sa_clear(&s);
        sa_add_double(&s, (double)r[2 * i]);
        sa_add_double(&s, (double)r[2 * i + 1]);
        sa_add_double(&s, -ah);
        sa_add_double(&s, -al);
        sa_add_double(&s, -bh);
        sa_add_double(&s, -bl);
        out[3 * i] = fabs(sa_to_double(&s));
        sa_clear(&s);
        sa_add_double(&s, al);
        sa_add_double(&s, bl);
        out[3 * i + 1] = ldexp(fabs(sa_to_double(&s)), -24);
        sa_clear(&s);
        sa_add_double(&s, ah);
        sa_add_double(&s, al);
        sa_add_double(&s, bh);
        sa_add_double(&s, bl);
        out[3 * i + 2] = ldexp(fabs(sa_to_double(&s)), -44);
    }
}

/* Relative error of a float-float result against the exact value of the
 * operation, in binary128, rounded to binary64.
 *   op 0: (ah+al) + (bh+bl)      op 1: (ah+al) * (bh+bl)
 *   op 2: (ah+al) / (bh+bl)      op 3: sqrt(ah+al)        (b ignored)
 * Sums and products are formed exactly with the superaccumulator (every
 * partial product of two binary32 numbers is exact in binary64) and rounded
 * once to binary128; quotient and square root are one binary128 operation on
 * exactly represented operands.  A zero exact value gives |error| instead of
 * the relative error. */
void exact_relerr_ff(int op, const float *a, const float *b, const float *r,
                     double *rel, size_t n)
{
    sacc s;
    for (size_t i = 0; i < n; ++i) {
        double ah = a[2 * i], al = a[2 * i + 1];
        double bh = b ? b[2 * i] : 0.0, bl = b ? b[2 * i + 1] : 0.0;
        q128 ex;
        if (op == 0 || op == 1) {
            sa_clear(&s);
            if (op == 0) {
                sa_add_double(&s, ah);
                sa_add_double(&s, al);
                sa_add_double(&s, bh);
                sa_add_double(&s, bl);
            } else {
                sa_add_double(&s, ah * bh);
                sa_add_double(&s, ah * bl);
                sa_add_double(&s, al * bh);
                sa_add_double(&s, al * bl);
            }
            ex = sa_to_q128(&s);
        } else {
            q128 qa = (q128)ah + (q128)al; /* exact for normalised pairs */
            if (op == 2) {
                q128 qb = (q128)bh + (q128)bl;
                ex = qa / qb;
            } else {
                ex = Q_SQRT(qa);
            }
        }
        q128 res = (q128)r[2 * i] + (q128)r[2 * i + 1];
        q128 err = res - ex;
        if (ex != 0)
            err = err / ex;
        double e = (double)err;
        rel[i] = fabs(e);
    }
}

/* Exact reference of a float-float dot product (or sum when y is NULL):
 *   out[0], out[1]: S = sum_i x_i y_i rounded to binary128, as (hi, lo)
 *                   doubles;
 *   out[2]:         A = sum_i |x_i y_i| (RN binary64);
 *   out[3]:         E = (rh + rl) - S exactly, RN binary64, where (rh, rl)
 *                   = res[0], res[1] is the result under test (res may be
 *                   NULL, then out[3] = 0).
 * x_i y_i = (xh + xl)(yh + yl) is accumulated as its four exact binary64
 * partial products. */
void exact_dot_ff(const float *x, const float *y, size_t n, const float *res, double *out)
{
    static sacc s, sabs; /* large: keep off the stack; not reentrant */
    sa_clear(&s);
    sa_clear(&sabs);
    for (size_t i = 0; i < n; ++i) {
        double xh = x[2 * i], xl = x[2 * i + 1];
        if (y) {
            double yh = y[2 * i], yl = y[2 * i + 1];
            double p0 = xh * yh, p1 = xh * yl, p2 = xl * yh, p3 = xl * yl;
            sa_add_double(&s, p0);
            sa_add_double(&s, p1);
            sa_add_double(&s, p2);
            sa_add_double(&s, p3);
            /* |x_i y_i| = sign(x_i y_i) * x_i y_i; the sign of a normalised
             * pair is the sign of its high part */
            double sg = ((xh < 0) != (yh < 0)) ? -1.0 : 1.0;
            if (xh == 0 || yh == 0) {
                /* fall back to the exact sign of the (tiny) product */
                sacc t;
                sa_clear(&t);
                sa_add_double(&t, p0);
                sa_add_double(&t, p1);
                sa_add_double(&t, p2);
                sa_add_double(&t, p3);
                double tv = sa_to_double(&t);
                sg = (tv < 0) ? -1.0 : 1.0;
            }
            sa_add_double(&sabs, sg * p0);
            sa_add_double(&sabs, sg * p1);
            sa_add_double(&sabs, sg * p2);
            sa_add_double(&sabs, sg * p3);
        } else {
            sa_add_double(&s, xh);
            sa_add_double(&s, xl);
            double sg = (xh < 0) ? -1.0 : 1.0;
            sa_add_double(&sabs, sg * xh);
            sa_add_double(&sabs, sg * xl);
        }
    }
    q128 S = sa_to_q128(&s);
    double hi = (double)S;
    out[0] = hi;
    out[1] = (double)(S - (q128)hi);
    out[2] = sa_to_double(&sabs);
    if (res) {
        sa_add_double(&s, -(double)res[0]);
        sa_add_double(&s, -(double)res[1]);
        out[3] = -sa_to_double(&s);
    } else {
        out[3] = 0.0;
    }
}

/* Exact reference of a binary32 dot product (or sum when y is NULL), with
 * the same outputs as exact_dot_ff: S as a binary128 (hi, lo) double pair,
 * A = sum |x_i y_i|, E = (res[0] + res[1]) - S.  Every x_i y_i is exact in
 * binary64. */
void exact_dot_f32(const float *x, const float *y, size_t n, const float *res, double *out)
{
    static sacc s, sabs;
    sa_clear(&s);
    sa_clear(&sabs);
    for (size_t i = 0; i < n; ++i) {
        double p = y ? (double)x[i] * (double)y[i] : (double)x[i];
        sa_add_double(&s, p);
        sa_add_double(&sabs, fabs(p));
    }
    q128 S = sa_to_q128(&s);
    double hi = (double)S;
    out[0] = hi;
    out[1] = (double)(S - (q128)hi);
    out[2] = sa_to_double(&sabs);
    if (res) {
        sa_add_double(&s, -(double)res[0]);
        sa_add_double(&s, -(double)res[1]);
        out[3] = -sa_to_double(&s);
    } else {
        out[3] = 0.0;
    }
}
