// ff_core.cuh -- device-side error-free transformations and float-float
// operators (Da Graca & Defour, Section 4.1), written with explicit
// round-to-nearest binary32 intrinsics so that the compiler can neither
// contract a multiply and an add into an FMA nor reassociate anything.  The
// only fused multiply-add is the explicit one of Mul12.
//
// A float-float value is a float2 {x = hi, y = lo}: the unevaluated sum
// hi + lo (the format of Section 4).
#pragma once
#include <cuda_runtime.h>

namespace ffk {

// Add12 theorem (Knuth): s = a (+) b, r = (a + b) - s exactly; branch free.
__device__ __forceinline__ float2 add12(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    const float r = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return make_float2(s, r);
}

// Mul12 theorem: p = a (x) b, e = a*b - p exactly.  The paper derives the
// error with Dekker's Split; one correctly rounded FMA gives the same pair
// (the pair is unique wherever neither part under- or overflows).
__device__ __forceinline__ float2 mul12(float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return make_float2(p, e);
}

// Add22 theorem.  The paper's one test |ah| >= |bh| chooses which high part
// is subtracted from r first; here it selects operands instead of branching
// (the paper prefers extra work to tests on GPUs, Section 4), so that
//   s = (((P (-) r) (+) Q) (+) L1) (+) L2
// is, operation for operation, the paper's line for the taken branch.
__device__ __forceinline__ float2 add22(float2 a, float2 b)
{
    const float r = __fadd_rn(a.x, b.x);
    const bool c = fabsf(a.x) >= fabsf(b.x);
    const float P = c ? a.x : b.x;
    const float Q = c ? b.x : a.x;
    const float L1 = c ? b.y : a.y;
    const float L2 = c ? a.y : b.y;
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(__fsub_rn(P, r), Q), L1), L2);
    return add12(r, s);
}

// Mul22 theorem: (t1, t2) = Mul12(ah, bh); t3 = ((ah bl) + (al bh)) + t2;
// result Add12(t1, t3).  al * bl is dropped, as in the paper.
__device__ __forceinline__ float2 mul22(float2 a, float2 b)
{
    const float2 t = mul12(a.x, b.x);
    const float t3 = __fadd_rn(__fadd_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)), t.y);
    return add12(t.x, t3);
}

// Div22: Dekker's div2 with the paper's Add12 as the final renormalisation.
//   ch = ah / bh; (uh, ul) = Mul12(ch, bh);
//   cl = ((((ah - uh) - ul) + al) - ch bl) / bh;  result Add12(ch, cl)
__device__ __forceinline__ float2 div22(float2 a, float2 b)
{
    const float ch = __fdiv_rn(a.x, b.x);
    const float2 u = mul12(ch, b.x);
    const float num = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(a.x, u.x), u.y), a.y),
                                __fmul_rn(ch, b.y));
    const float cl = __fdiv_rn(num, b.x);
    return add12(ch, cl);
}

// Sqrt22: Dekker's sqrt2 with the paper's Add12 as the final step.
//   c = sqrt(ah); (u, uu) = Mul12(c, c);
//   cc = ((((ah - u) - uu) + al) * 0.5) / c;  result Add12(c, cc)
// ah == 0 returns (ah, 0) (keeping the sign of zero).  A negative ah makes
// every step NaN, so the result is (NaN, NaN) without a test.
__device__ __forceinline__ float2 sqrt22(float2 a)
{
    const float c = __fsqrt_rn(a.x);
    const float2 u = mul12(c, c);
    const float rem = __fadd_rn(__fsub_rn(__fsub_rn(a.x, u.x), u.y), a.y);
    const float cc = __fdiv_rn(__fmul_rn(rem, 0.5f), c);
    const float2 r = add12(c, cc);
    const bool z = (a.x == 0.0f);
    return make_float2(z ? a.x : r.x, z ? 0.0f : r.y);
}

// Fast2Sum (Dekker): s = a (+) b, t = (a + b) - s exactly when the exponent
// of a is at least that of b.
__device__ __forceinline__ float2 fast2sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    return make_float2(s, __fsub_rn(b, z));
}

// Accurate float-float addition (Joldes, Muller and Popescu 2017,
// Algorithm 6): the two TwoSums of the high and the low parts, then two
// Fast2Sum renormalisations.  Relative error <= 3u^2 / (1 - 4u) (u = 2^-24)
// even under cancellation, where Add22 only bounds the error by 2^-24 |al + bl|.
__device__ __forceinline__ float2 add22_accurate(float2 x, float2 y)
{
    const float2 s = add12(x.x, y.x);
    const float2 t = add12(x.y, y.y);
    const float c = __fadd_rn(s.y, t.x);
    const float2 v = fast2sum(s.x, c);
    const float w = __fadd_rn(t.y, v.y);
    return fast2sum(v.x, w);
}

}  // namespace ffk
