/*
 * ff_oracle.c -- plain, slow, obviously-correct CPU restatement of the
 * float-float arithmetic of Da Graca & Defour, "Implementation of
 * float-float operators on graphics hardware" (arXiv cs/0603115), in IEEE
 * binary32 with round-to-nearest-even.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, helper or constant with
 * the CUDA library; the two meet only through the seeded input generators.
 *
 * Every binary32 operation below is a plain C `float` operation.  The file
 * is compiled with -ffp-contract=off and without -ffast-math, so each
 * `x * y + z` is two roundings, never a fused multiply-add; the only FMA is
 * the explicit fmaf() of the FMA form of Mul12.  Subnormals are kept (the
 * default floating-point environment has no flush-to-zero).
 *
 * Notation follows Section 4.1 of the paper: (+),(-),(x),(/) are the rounded
 * binary32 operations; a float-float value is the unevaluated sum hi + lo
 * of two binary32 numbers, stored as the pair (hi, lo) (Section 4, "Proposed
 * format").  Arrays of float-float values are packed pairs: x[2i] = hi_i,
 * x[2i+1] = lo_i.
 *
 * Readings of the paper where it is silent or garbled (all listed in the
 * design notes of the repository):
 *   - Split uses the splitting point s = 12 (constant 2^12 + 1 = 4097), the
 *     only choice in [p/2, p-1] for p = 24 that keeps every partial product
 *     of Mul12 exact.
 *   - Mul22's last step is Add12(t1, t3): the printed Add12(t1, t2) leaves t3
 *     unused and cannot meet the stated 2^-44 bound whenever al or bl matter.
 *   - Add22 keeps the paper's Add12 (not Fast2Sum) as its last step, and its
 *     tie |ah| == |bh| takes the first branch (the test is ">=").
 *   - Div22 and Sqrt22 are not in the paper; they follow Dekker's div2 and
 *     sqrt2 (Dekker 1971, the paper's reference for Split and Mul12) with the
 *     paper's Add12 as the final renormalisation.
 *   - Reductions (sum, dot), AXPY, GEMV, GEMM and the dot backward are not
 *     in the paper either; they are the plain left-to-right Add22 accumulation of
 *     the paper's operators (the compensated algorithms Section 7 names as
 *     future work).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#if defined(__FAST_MATH__)
#error "the oracle must not be compiled with -ffast-math"
#endif

/* ------------------------------------------------------------------------ */
/* Error-free transformations, Section 4.1                                   */
/* ------------------------------------------------------------------------ */

/* Add12 theorem (Knuth): s = a (+) b and r = (a + b) - s exactly, branch
 * free, in the three-line order the paper gives. */
static void add12(float a, float b, float *s_out, float *r_out)
{
    float s = a + b;
    float v = s - a;
    float r = (a - (s - v)) + (b - v);
    *s_out = s;
    *r_out = r;
}

/* Split theorem (Dekker), s = 12: a = a_hi + a_lo with a_hi on 12 bits and
 * a_lo on 12 bits (11 bits plus the sign). */
static void split(float a, float *a_hi, float *a_lo)
{
    const float two_s_plus_1 = 4097.0f; /* 2^12 (+) 1, exact */
    float c = two_s_plus_1 * a;
    float a_big = c - a;
    float hi = c - a_big;
    float lo = a - hi;
    *a_hi = hi;
    *a_lo = lo;
}

/* Mul12 theorem (Dekker): x = a (x) b and y = a*b - x exactly, through two
 * Splits and four exact partial products. */
static void mul12_dekker(float a, float b, float *x_out, float *y_out)
{
    float a_hi, a_lo, b_hi, b_lo;
    float x = a * b;
    split(a, &a_hi, &a_lo);
    split(b, &b_hi, &b_lo);
    float err1 = x - (a_hi * b_hi);
    float err2 = err1 - (a_lo * b_hi);
    float err3 = err2 - (a_hi * b_lo);
    float y = (a_lo * b_lo) - err3;
    *x_out = x;
    *y_out = y;
}

/* Mul12 in its fused form: the same pair (RN(ab), ab - RN(ab)), with the
 * error read off one correctly rounded fused multiply-add. */
static void mul12_fma(float a, float b, float *x_out, float *y_out)
{
    float x = a * b;
    float y = fmaf(a, b, -x);
    *x_out = x;
    *y_out = y;
}

/* ------------------------------------------------------------------------ */
/* Float-float operators                                                     */
/* ------------------------------------------------------------------------ */

/* Add22 theorem: the paper's one-branch float-float addition. */
static void add22(float ah, float al, float bh, float bl, float *rh, float *rl)
{
    float r = ah + bh;
    float s;
    if (fabsf(ah) >= fabsf(bh))
        s = (((ah - r) + bh) + bl) + al;
    else
        s = (((bh - r) + ah) + al) + bl;
    add12(r, s, rh, rl);
}

/* Mul22 theorem, with Mul12 in its fused form (bitwise equal to the Dekker
 * form wherever neither under- nor overflows; see mul22_dekker). */
static void mul22(float ah, float al, float bh, float bl, float *rh, float *rl)
{
    float t1, t2;
    mul12_fma(ah, bh, &t1, &t2);
    float t3 = ((ah * bl) + (al * bh)) + t2;
    add12(t1, t3, rh, rl);
}

/* Mul22 with the paper's own Dekker Mul12 (cross-check only). */
static void mul22_dekker(float ah, float al, float bh, float bl, float *rh, float *rl)
{
    float t1, t2;
    mul12_dekker(ah, bh, &t1, &t2);
    float t3 = ((ah * bl) + (al * bh)) + t2;
    add12(t1, t3, rh, rl);
}

/* Div22: Dekker's div2.  ch approximates the quotient, the exact product
 * ch * bh gives the remainder of the high parts, and the low parts enter a
 * first-order correction cl; Add12 renormalises. */
static void div22(float ah, float al, float bh, float bl, float *rh, float *rl)
{
    float ch = ah / bh;
    float uh, ul;
    mul12_fma(ch, bh, &uh, &ul);
    float cl = ((((ah - uh) - ul) + al) - (ch * bl)) / bh;
    add12(ch, cl, rh, rl);
}

/* Sqrt22: Dekker's sqrt2.  c = sqrt(ah); the exact square c*c gives the
 * remainder, halved and divided by c for the correction term.  Zero returns
 * (ah, 0) (keeping -0), a negative high part returns (NaN, NaN). */
static void sqrt22(float ah, float al, float *rh, float *rl)
{
    if (ah == 0.0f) {
        *rh = ah;
        *rl = 0.0f;
        return;
    }
    if (ah < 0.0f) {
        *rh = NAN;
        *rl = NAN;
        return;
    }
    float c = sqrtf(ah);
    float u, uu;
    mul12_fma(c, c, &u, &uu);
    float cc = ((((ah - u) - uu) + al) * 0.5f) / c;
    add12(c, cc, rh, rl);
}

/* Fast2Sum (Dekker): s = a (+) b, t = (a + b) - s exactly when the exponent
 * of a is at least that of b. */
static void fast2sum(float a, float b, float *s_out, float *t_out)
{
    float s = a + b;
    float z = s - a;
    float t = b - z;
    *s_out = s;
    *t_out = t;
}

/* Weight gradient of Y = A X: dA = dY X^T, dA[r, j] = acc over c = 0 .. k-1
 * of Add22(acc, Mul22(dY[r, c], X[j, c])).  dY: m x k column-major (lddy),
 * X: n x k column-major (ldx), dA: m x n row-major (ldda). */
void orc_gemv_dA(const float *dY, int64_t m, int64_t lddy, const float *X, int64_t n, int64_t ldx,
                 int64_t k, float *dA, int64_t ldda)
{
    for (int64_t r = 0; r < m; ++r) {
        for (int64_t j = 0; j < n; ++j) {
            float h = 0.0f, l = 0.0f;
            for (int64_t c = 0; c < k; ++c) {
                const float *dy = &dY[2 * (c * lddy + r)];
                const float *xv = &X[2 * (c * ldx + j)];
                float ph, pl;
                mul22(dy[0], dy[1], xv[0], xv[1], &ph, &pl);
                add22(h, l, ph, pl, &h, &l);
            }
            dA[2 * (r * ldda + j)] = h;
            dA[2 * (r * ldda + j) + 1] = l;
        }
    }
}

/* Float-float matrix product C = op(A) op(B) (a GEMV with many right-hand
 * sides; not in the paper), all matrices row-major:
 *   C[i, j] = acc over p = 0 .. kk-1 of Add22(acc, Mul22(op(A)[i, p], op(B)[p, j])),
 * acc starting at (0, 0), p in increasing order.  op(A)[i, p] is A[i, p]
 * (A is m x kk, leading dimension lda) or, when transa, A[p, i] (A is kk x m);
 * op(B)[p, j] is B[p, j] (kk x n, ldb) or, when transb, B[j, p] (n x kk). */
void orc_gemm(int transa, int transb, int64_t m, int64_t n, int64_t kk,
              const float *A, int64_t lda, const float *B, int64_t ldb, float *C, int64_t ldc)
{
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            float h = 0.0f, l = 0.0f;
            for (int64_t p = 0; p < kk; ++p) {
                const float *a = transa ? &A[2 * (p * lda + i)] : &A[2 * (i * lda + p)];
                const float *b = transb ? &B[2 * (j * ldb + p)] : &B[2 * (p * ldb + j)];
                float ph, pl;
                mul22(a[0], a[1], b[0], b[1], &ph, &pl);
                add22(h, l, ph, pl, &h, &l);
            }
            C[2 * (i * ldc + j)] = h;
            C[2 * (i * ldc + j) + 1] = l;
        }
    }
}

/* Accurate float-float addition (the paper's open problem of Add22's
 * cancellation error, Sections 6.1 and 7): Algorithm 6 ("AccurateDWPlusDW")
 * of Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
 * building blocks of double-word arithmetic" (ACM TOMS 2017):
 *   (sh, sl) = TwoSum(xh, yh); (th, tl) = TwoSum(xl, yl); c = sl + th;
 *   (vh, vl) = Fast2Sum(sh, c); w = tl + vl; (zh, zl) = Fast2Sum(vh, w).
 * Relative error <= 3u^2 / (1 - 4u), u = 2^-24, with no cancellation term.
 * TwoSum is the paper's Add12. */
static void add22_accurate(float xh, float xl, float yh, float yl, float *zh, float *zl)
{
    float sh, sl, th, tl, vh, vl;
    add12(xh, yh, &sh, &sl);
    add12(xl, yl, &th, &tl);
    float c = sl + th;
    fast2sum(sh, c, &vh, &vl);
    float w = tl + vl;
    fast2sum(vh, w, zh, zl);
}

/* ------------------------------------------------------------------------ */
/* Array entry points (called from the test harness through ctypes)          */
/* ------------------------------------------------------------------------ */

void orc_add12(const float *ab, float *se, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        add12(ab[2 * i], ab[2 * i + 1], &se[2 * i], &se[2 * i + 1]);
}

void orc_split(const float *a, float *hl, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        split(a[i], &hl[2 * i], &hl[2 * i + 1]);
}

void orc_mul12_dekker(const float *ab, float *xy, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        mul12_dekker(ab[2 * i], ab[2 * i + 1], &xy[2 * i], &xy[2 * i + 1]);
}

void orc_mul12(const float *ab, float *xy, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        mul12_fma(ab[2 * i], ab[2 * i + 1], &xy[2 * i], &xy[2 * i + 1]);
}

void orc_add22(const float *a, const float *b, float *r, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        add22(a[2 * i], a[2 * i + 1], b[2 * i], b[2 * i + 1], &r[2 * i], &r[2 * i + 1]);
}

void orc_mul22(const float *a, const float *b, float *r, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        mul22(a[2 * i], a[2 * i + 1], b[2 * i], b[2 * i + 1], &r[2 * i], &r[2 * i + 1]);
}

void orc_mul22_dekker(const float *a, const float *b, float *r, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        mul22_dekker(a[2 * i], a[2 * i + 1], b[2 * i], b[2 * i + 1], &r[2 * i], &r[2 * i + 1]);
}

void orc_div22(const float *a, const float *b, float *r, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        div22(a[2 * i], a[2 * i + 1], b[2 * i], b[2 * i + 1], &r[2 * i], &r[2 * i + 1]);
}

void orc_sqrt22(const float *a, float *r, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        sqrt22(a[2 * i], a[2 * i + 1], &r[2 * i], &r[2 * i + 1]);
}

/* Sum: acc = (0,0), then acc = Add22(acc, x_i) for i = 0 .. n-1 in order. */
void orc_sum(const float *x, size_t n, float *out)
{
    float h = 0.0f, l = 0.0f;
    for (size_t i = 0; i < n; ++i)
        add22(h, l, x[2 * i], x[2 * i + 1], &h, &l);
    out[0] = h;
    out[1] = l;
}

/* Dot: acc = (0,0), then acc = Add22(acc, Mul22(x_i, y_i)) in order. */
void orc_dot(const float *x, const float *y, size_t n, float *out)
{
    float h = 0.0f, l = 0.0f;
    for (size_t i = 0; i < n; ++i) {
        float ph, pl;
        mul22(x[2 * i], x[2 * i + 1], y[2 * i], y[2 * i + 1], &ph, &pl);
        add22(h, l, ph, pl, &h, &l);
    }
    out[0] = h;
    out[1] = l;
}

/* Adjoint of the dot product d = sum_i x_i y_i: dx_i = Mul22(dout, y_i),
 * dy_i = Mul22(dout, x_i).  dout is one float-float value. */
void orc_dot_backward(const float *dout, const float *x, const float *y,
                      float *dx, float *dy, size_t n)
{
    for (size_t i = 0; i < n; ++i) {
        mul22(dout[0], dout[1], y[2 * i], y[2 * i + 1], &dx[2 * i], &dx[2 * i + 1]);
        mul22(dout[0], dout[1], x[2 * i], x[2 * i + 1], &dy[2 * i], &dy[2 * i + 1]);
    }
}

/* AXPY: z_i = Add22(Mul22(alpha, x_i), y_i).  alpha is one float-float. */
void orc_axpy(const float *alpha, const float *x, const float *y, float *z, size_t n)
{
    for (size_t i = 0; i < n; ++i) {
        float ph, pl;
        mul22(alpha[0], alpha[1], x[2 * i], x[2 * i + 1], &ph, &pl);
        add22(ph, pl, y[2 * i], y[2 * i + 1], &z[2 * i], &z[2 * i + 1]);
    }
}

/* GEMV Y = A X: A is m x n row-major float-float with row stride lda (in
 * float-float elements), X is n x k column-major with column stride ldx, Y is
 * m x k column-major with column stride ldy.
 * Y[r, c] = acc over j = 0 .. n-1 of Add22(acc, Mul22(A[r, j], X[j, c])). */
void orc_gemv(const float *A, int64_t m, int64_t n, int64_t lda,
              const float *X, int64_t ldx, int64_t k, float *Y, int64_t ldy)
{
    for (int64_t c = 0; c < k; ++c) {
        for (int64_t r = 0; r < m; ++r) {
            float h = 0.0f, l = 0.0f;
            for (int64_t j = 0; j < n; ++j) {
                const float *a = &A[2 * (r * lda + j)];
                const float *xv = &X[2 * (c * ldx + j)];
                float ph, pl;
                mul22(a[0], a[1], xv[0], xv[1], &ph, &pl);
                add22(h, l, ph, pl, &h, &l);
            }
            Y[2 * (c * ldy + r)] = h;
            Y[2 * (c * ldy + r) + 1] = l;
        }
    }
}

/* Adjoint GEMV dX = A^T dY: dX[j, c] = acc over r = 0 .. m-1 of
 * Add22(acc, Mul22(A[r, j], dY[r, c])).  dY is m x k column-major (lddy),
 * dX is n x k column-major (lddx). */
void orc_gemv_t(const float *A, int64_t m, int64_t n, int64_t lda,
                const float *dY, int64_t lddy, int64_t k, float *dX, int64_t lddx)
{
    for (int64_t c = 0; c < k; ++c) {
        for (int64_t j = 0; j < n; ++j) {
            float h = 0.0f, l = 0.0f;
            for (int64_t r = 0; r < m; ++r) {
                const float *a = &A[2 * (r * lda + j)];
                const float *dy = &dY[2 * (c * lddy + r)];
                float ph, pl;
                mul22(a[0], a[1], dy[0], dy[1], &ph, &pl);
                add22(h, l, ph, pl, &h, &l);
            }
            dX[2 * (c * lddx + j)] = h;
            dX[2 * (c * lddx + j) + 1] = l;
        }
    }
}

void orc_add22_accurate(const float *a, const float *b, float *r, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        add22_accurate(a[2 * i], a[2 * i + 1], b[2 * i], b[2 * i + 1], &r[2 * i], &r[2 * i + 1]);
}

/* Compensated summation and dot product of binary32 vectors (the
 * compensated algorithms Section 7 names as future work): Ogita, Rump and
 * Oishi, "Accurate
 * sum and dot product" (SIAM J. Sci. Comput. 2005), Sum2 and Dot2, in their
 * left-to-right order, with the paper's Add12 as TwoSum and the fused Mul12
 * as TwoProduct.  The result is returned unrounded as the float-float value
 * Add12(p, s) (equal to p + s exactly).
 *   Sum2: p = x_0, s = 0; for i >= 1: (p, q) = TwoSum(p, x_i); s = s + q.
 *   Dot2: (p, s) = TwoProduct(x_0, y_0); for i >= 1: (h, r) =
 *         TwoProduct(x_i, y_i); (p, q) = TwoSum(p, h); s = s + (q + r). */
void orc_sum2(const float *x, size_t n, float *out)
{
    float p = 0.0f, s = 0.0f;
    if (n > 0)
        p = x[0];
    for (size_t i = 1; i < n; ++i) {
        float q;
        add12(p, x[i], &p, &q);
        s = s + q;
    }
    add12(p, s, &out[0], &out[1]);
}

void orc_dot2(const float *x, const float *y, size_t n, float *out)
{
    float p = 0.0f, s = 0.0f;
    if (n > 0)
        mul12_fma(x[0], y[0], &p, &s);
    for (size_t i = 1; i < n; ++i) {
        float h, r, q;
        mul12_fma(x[i], y[i], &h, &r);
        add12(p, h, &p, &q);
        s = s + (q + r);
    }
    add12(p, s, &out[0], &out[1]);
}

/* Plain binary32 operations, the normalisation baseline of the paper's
 * timing tables (Section 6: times relative to 4096 single additions). */
void orc_fp32_add(const float *a, const float *b, float *out, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        out[i] = a[i] + b[i];
}

void orc_fp32_mul(const float *a, const float *b, float *out, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        out[i] = a[i] * b[i];
}

/* Multiply-and-add as two roundings (the file is built without contraction). */
void orc_fp32_mad(const float *a, const float *b, const float *c, float *out, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        out[i] = a[i] * b[i] + c[i];
}

/* Contraction canary: returns a*b + c as written.  With contraction off it is
 * RN(RN(a*b) + c); a test compares it with a fused result to prove the build
 * did not fuse it. */
float orc_canary_mul_add(float a, float b, float c)
{
    return a * b + c;
}
