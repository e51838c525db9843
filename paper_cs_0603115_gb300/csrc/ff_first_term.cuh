// ff_first_term.cuh -- the first accumulation step of a float-float sum that
// starts from (0, 0), as the weight gradient forms it: every output element
// is Add22((0, 0), term_0), then Add22 of the later terms.  (The GEMM kernel
// keeps the plain Add22 for its first term: peeling it off the slice loop
// measured 0.3-1% slower, its loop being tuned for instruction fetch.)
#pragma once
#include <cuda_runtime.h>

#include "ff_core.cuh"

namespace ffk {

// Add22((+0, +0), t) bit for bit, with two additions instead of the full
// sequence when t is a finite pair whose sum rounds to its high part (every
// Mul22 result is one: it ends with Add12).  For such t the Add22 theorem's
// steps reduce to r = th (+) 0, s = tl (+) 0 and Add12(r, s) = (r, s):
// th - r = +0 (the tie branch when th = +-0, which forces tl = +-0), the zero
// operand's low part adds nothing, and Add12 of a pair whose sum rounds to its
// first part returns the pair.  "(+) 0" does what the full sequence does to a
// negative zero (it becomes +0).  Any other t (infinite, NaN, not normalised)
// takes the full sequence.  The test is voted over the warp so that the
// branch never diverges; every lane of the warp must be present.
__device__ __forceinline__ bool from_zero_fast(float2 t)
{
    return fabsf(t.x) <= 3.40282347e38f && __fadd_rn(t.x, t.y) == t.x;
}

__device__ __forceinline__ float2 add22_from_zero(float2 t, bool warp_fast)
{
    if (warp_fast) return make_float2(__fadd_rn(t.x, 0.0f), __fadd_rn(t.y, 0.0f));
    return add22(make_float2(0.0f, 0.0f), t);
}

}  // namespace ffk
