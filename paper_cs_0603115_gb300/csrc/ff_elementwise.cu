// ff_elementwise.cu -- the streaming elementwise entry points: the
// error-free transformations (Section 4.1), the float-float operators, AXPY,
// the dot-product adjoint, and the native binary64 / binary32 baselines.
// Every op is a small functor applied by the shared streaming kernel.
#include <cmath>

#include "ff_core.cuh"
#include "ff_host.cuh"
#include "ff_stream.cuh"

namespace {

struct OpAdd12 {
    __device__ void operator()(const float2 (&x)[1], float2 (&y)[1]) const { y[0] = ffk::add12(x[0].x, x[0].y); }
};
struct OpMul12 {
    __device__ void operator()(const float2 (&x)[1], float2 (&y)[1]) const { y[0] = ffk::mul12(x[0].x, x[0].y); }
};
struct OpAdd22 {
    __device__ void operator()(const float2 (&x)[2], float2 (&y)[1]) const { y[0] = ffk::add22(x[0], x[1]); }
};
struct OpAdd22Acc {
    __device__ void operator()(const float2 (&x)[2], float2 (&y)[1]) const { y[0] = ffk::add22_accurate(x[0], x[1]); }
};
struct OpMul22 {
    __device__ void operator()(const float2 (&x)[2], float2 (&y)[1]) const { y[0] = ffk::mul22(x[0], x[1]); }
};
struct OpDiv22 {
    __device__ void operator()(const float2 (&x)[2], float2 (&y)[1]) const { y[0] = ffk::div22(x[0], x[1]); }
};
struct OpSqrt22 {
    __device__ void operator()(const float2 (&x)[1], float2 (&y)[1]) const { y[0] = ffk::sqrt22(x[0]); }
};
struct OpAxpy {
    float2 alpha;
    __device__ void operator()(const float2 (&x)[2], float2 (&y)[1]) const
    {
        y[0] = ffk::add22(ffk::mul22(alpha, x[0]), x[1]);
    }
};
// dx = Mul22(dout, y), dy = Mul22(dout, x); dout is read once per element
// from device memory (an L1/L2 broadcast).
struct OpDotBwd {
    const float2* dout;
    __device__ void operator()(const float2 (&x)[2], float2 (&y)[2]) const
    {
        const float2 d = __ldg(dout);
        y[0] = ffk::mul22(d, x[1]);
        y[1] = ffk::mul22(d, x[0]);
    }
};

struct OpF64Add {
    __device__ void operator()(const double (&x)[2], double (&y)[1]) const { y[0] = __dadd_rn(x[0], x[1]); }
};
struct OpF64Mul {
    __device__ void operator()(const double (&x)[2], double (&y)[1]) const { y[0] = __dmul_rn(x[0], x[1]); }
};
struct OpF64Div {
    __device__ void operator()(const double (&x)[2], double (&y)[1]) const { y[0] = __ddiv_rn(x[0], x[1]); }
};
struct OpF64Sqrt {
    __device__ void operator()(const double (&x)[1], double (&y)[1]) const { y[0] = __dsqrt_rn(x[0]); }
};
struct OpF32Add {
    __device__ void operator()(const float (&x)[2], float (&y)[1]) const { y[0] = __fadd_rn(x[0], x[1]); }
};
struct OpF32Mul {
    __device__ void operator()(const float (&x)[2], float (&y)[1]) const { y[0] = __fmul_rn(x[0], x[1]); }
};
struct OpF32Mad {
    __device__ void operator()(const float (&x)[3], float (&y)[1]) const
    {
        y[0] = __fadd_rn(__fmul_rn(x[0], x[1]), x[2]);
    }
};

template <typename T, class Op>
ff_status run1(const T* a, T* out, size_t n, cudaStream_t s, Op op = Op())
{
    if (!ffh::ok_ptr(a, n) || !ffh::ok_ptr(out, n)) return FF_ERR_INVALID_ARG;
    if (!ffh::aligned(a, sizeof(T)) || !ffh::aligned(out, sizeof(T))) return FF_ERR_INVALID_ARG;
    ffst::Args<T, 1, 1> args{{a}, {out}, n, 0};
    return ffst::launch(args, op, s);
}

template <typename T, class Op>
ff_status run2(const T* a, const T* b, T* out, size_t n, cudaStream_t s, Op op = Op())
{
    if (!ffh::ok_ptr(a, n) || !ffh::ok_ptr(b, n) || !ffh::ok_ptr(out, n)) return FF_ERR_INVALID_ARG;
    if (!ffh::aligned(a, sizeof(T)) || !ffh::aligned(b, sizeof(T)) || !ffh::aligned(out, sizeof(T)))
        return FF_ERR_INVALID_ARG;
    ffst::Args<T, 2, 1> args{{a, b}, {out}, n, 0};
    return ffst::launch(args, op, s);
}

// binary32 arrays need only 4-byte alignment
inline bool ok_f32(const float* p, size_t n) { return n == 0 || (p != nullptr && ffh::aligned(p, 4)); }

}  // namespace

extern "C" {

ff_status ff_add12(const ff2* ab, ff2* se, size_t n, cudaStream_t s)
{
    return run1<float2, OpAdd12>(reinterpret_cast<const float2*>(ab), reinterpret_cast<float2*>(se), n, s);
}

ff_status ff_mul12(const ff2* ab, ff2* pe, size_t n, cudaStream_t s)
{
    return run1<float2, OpMul12>(reinterpret_cast<const float2*>(ab), reinterpret_cast<float2*>(pe), n, s);
}

ff_status ff_add(const ff2* a, const ff2* b, ff2* out, size_t n, cudaStream_t s)
{
    return run2<float2, OpAdd22>(reinterpret_cast<const float2*>(a), reinterpret_cast<const float2*>(b),
                                 reinterpret_cast<float2*>(out), n, s);
}

ff_status ff_add_accurate(const ff2* a, const ff2* b, ff2* out, size_t n, cudaStream_t s)
{
    return run2<float2, OpAdd22Acc>(reinterpret_cast<const float2*>(a), reinterpret_cast<const float2*>(b),
                                    reinterpret_cast<float2*>(out), n, s);
}

ff_status ff_mul(const ff2* a, const ff2* b, ff2* out, size_t n, cudaStream_t s)
{
    return run2<float2, OpMul22>(reinterpret_cast<const float2*>(a), reinterpret_cast<const float2*>(b),
                                 reinterpret_cast<float2*>(out), n, s);
}

ff_status ff_div(const ff2* a, const ff2* b, ff2* out, size_t n, cudaStream_t s)
{
    return run2<float2, OpDiv22>(reinterpret_cast<const float2*>(a), reinterpret_cast<const float2*>(b),
                                 reinterpret_cast<float2*>(out), n, s);
}

ff_status ff_sqrt(const ff2* a, ff2* out, size_t n, cudaStream_t s)
{
    return run1<float2, OpSqrt22>(reinterpret_cast<const float2*>(a), reinterpret_cast<float2*>(out), n, s);
}

ff_status ff_axpy(ff2 alpha, const ff2* x, const ff2* y, ff2* z, size_t n, cudaStream_t s)
{
    OpAxpy op{make_float2(alpha.hi, alpha.lo)};
    return run2<float2, OpAxpy>(reinterpret_cast<const float2*>(x), reinterpret_cast<const float2*>(y),
                                reinterpret_cast<float2*>(z), n, s, op);
}

ff_status ff_dot_backward(const ff2* dout_dev, const ff2* x, const ff2* y, ff2* dx, ff2* dy, size_t n,
                          cudaStream_t s)
{
    if (!ffh::ok_ptr(x, n) || !ffh::ok_ptr(y, n) || !ffh::ok_ptr(dx, n) || !ffh::ok_ptr(dy, n))
        return FF_ERR_INVALID_ARG;
    if (n == 0) return FF_OK;
    if (!ffh::ok_ptr(dout_dev, 1)) return FF_ERR_INVALID_ARG;
    OpDotBwd op{reinterpret_cast<const float2*>(dout_dev)};
    ffst::Args<float2, 2, 2> args{{reinterpret_cast<const float2*>(x), reinterpret_cast<const float2*>(y)},
                                 {reinterpret_cast<float2*>(dx), reinterpret_cast<float2*>(dy)}, n, 0};
    return ffst::launch(args, op, s);
}

ff_status ff_f64_add(const double* a, const double* b, double* out, size_t n, cudaStream_t s)
{
    return run2<double, OpF64Add>(a, b, out, n, s);
}
ff_status ff_f64_mul(const double* a, const double* b, double* out, size_t n, cudaStream_t s)
{
    return run2<double, OpF64Mul>(a, b, out, n, s);
}
ff_status ff_f64_div(const double* a, const double* b, double* out, size_t n, cudaStream_t s)
{
    return run2<double, OpF64Div>(a, b, out, n, s);
}
ff_status ff_f64_sqrt(const double* a, double* out, size_t n, cudaStream_t s)
{
    return run1<double, OpF64Sqrt>(a, out, n, s);
}

ff_status ff_f32_add(const float* a, const float* b, float* out, size_t n, cudaStream_t s)
{
    if (!ok_f32(a, n) || !ok_f32(b, n) || !ok_f32(out, n)) return FF_ERR_INVALID_ARG;
    ffst::Args<float, 2, 1> args{{a, b}, {out}, n, 0};
    return ffst::launch(args, OpF32Add(), s);
}
ff_status ff_f32_mul(const float* a, const float* b, float* out, size_t n, cudaStream_t s)
{
    if (!ok_f32(a, n) || !ok_f32(b, n) || !ok_f32(out, n)) return FF_ERR_INVALID_ARG;
    ffst::Args<float, 2, 1> args{{a, b}, {out}, n, 0};
    return ffst::launch(args, OpF32Mul(), s);
}
ff_status ff_f32_mad(const float* a, const float* b, const float* c, float* out, size_t n, cudaStream_t s)
{
    if (!ok_f32(a, n) || !ok_f32(b, n) || !ok_f32(c, n) || !ok_f32(out, n)) return FF_ERR_INVALID_ARG;
    ffst::Args<float, 3, 1> args{{a, b, c}, {out}, n, 0};
    return ffst::launch(args, OpF32Mad(), s);
}

}  // extern "C"
