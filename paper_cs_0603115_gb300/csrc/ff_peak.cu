// ff_peak.cu -- FMA throughput probe: the FP32 and FP64 arithmetic peaks of
// the device, measured by a kernel of this library rather than taken from a
// data sheet.  They are the denominators of the FP32-issue-bound rooflines
// (GEMV with several right-hand sides, GEMM) and the yardstick of the FP64
// baselines.
//
// Every thread runs eight independent chains x <- fma(x, a, b) for `iters`
// rounds (sixteen rounds per loop trip, so that the loop's own instructions
// take under 3% of the issue slots) and writes the sum of its chains, so
// nothing can be removed as dead code; a and b are kernel arguments, so
// nothing can be folded.  With a = b = 1 every chain counts exactly:
// x_final = x_0 + iters.
#include "ff_host.cuh"

namespace {

__device__ __forceinline__ float fma_rn(float x, float a, float b) { return __fmaf_rn(x, a, b); }
__device__ __forceinline__ double fma_rn(double x, double a, double b) { return __fma_rn(x, a, b); }

template <typename T>
__global__ void fma_peak_kernel(T a, T b, int64_t iters, T* __restrict__ out)
{
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = static_cast<T>(c);
    int64_t it = 0;
    for (; it + 16 <= iters; it += 16) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fma_rn(x[c], a, b);
    }
    for (; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = fma_rn(x[c], a, b);
    T s = x[0];
#pragma unroll
    for (int c = 1; c < 8; ++c) s += x[c];
    out[static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

ff_status ff_fma_peak(int f64, int64_t iters, int blocks, int threads, void* out, cudaStream_t s)
{
    if ((f64 != 0 && f64 != 1) || iters < 0 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0)
        return FF_ERR_INVALID_ARG;
    if (out == nullptr || !ffh::aligned(out, 8)) return FF_ERR_INVALID_ARG;
    if (f64)
        fma_peak_kernel<double><<<blocks, threads, 0, s>>>(1.0, 1.0, iters, static_cast<double*>(out));
    else
        fma_peak_kernel<float><<<blocks, threads, 0, s>>>(1.0f, 1.0f, iters, static_cast<float*>(out));
    return ffh::check_launch();
}

}  // extern "C"
