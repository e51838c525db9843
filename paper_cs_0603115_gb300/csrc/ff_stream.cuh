// ff_stream.cuh -- one grid-stride streaming kernel for every elementwise op.
//
// Each op reads NIN arrays and writes NOUT arrays of the same element type T
// (float2 for float-float values and packed operand pairs, double or float
// for the native baselines).  The body moves 16-byte vectors (two float2,
// two double, four float) with evict-first streaming loads and stores: every
// byte is touched once, so nothing is worth keeping in L1/L2.  Each thread
// issues U vector loads per input before computing.
//
// Residency: a GB300 sustains the highest read+write DRAM throughput on these
// kernels with a moderate number of loads in flight per SM, not with every
// SM full: measured on 2^28 values with the pipelined sweep below (U = 2),
// the two-input operators reach ~7.0 TB/s with 3 blocks of 256 per SM
// against ~6.6 TB/s at full occupancy, the one-input operators ~6.8 TB/s
// with 4.  The launcher caps the grid at SMs x blocks_per_sm(NIN).
//
// Alignment: device arrays are only required to be aligned to sizeof(T).
// If all arrays share the same offset modulo 16 bytes, a scalar head of
// `head` elements brings them to a 16-byte boundary and the remainder that
// does not fill a vector is a scalar tail; otherwise the whole range runs on
// scalar accesses (still coalesced).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ff_host.cuh"

namespace ffst {

constexpr int kBlock = 256;

template <typename T> struct Vec;
template <> struct Vec<float2> { using V = float4; static constexpr int E = 2; };
template <> struct Vec<double> { using V = double2; static constexpr int E = 2; };
template <> struct Vec<float>  { using V = float4; static constexpr int E = 4; };

template <typename T, int NIN, int NOUT>
struct Args {
    const T* in[NIN];
    T* out[NOUT];
    size_t n;      // elements
    int head;      // scalar elements before the first 16-byte boundary
};

// Split a 16-byte vector into its E values and join them back.  Explicit
// component moves, not a union: with a union the compiler scheduled the
// Add22 kernel measurably worse (about 6.2 instead of 7.1 TB/s on 2^28
// values at the same launch shape), the other operators were unaffected.
__device__ __forceinline__ void unpack(const float4& v, float2 (&e)[2])
{
    e[0] = make_float2(v.x, v.y);
    e[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ float4 pack(const float2 (&e)[2]) { return make_float4(e[0].x, e[0].y, e[1].x, e[1].y); }
__device__ __forceinline__ void unpack(const double2& v, double (&e)[2])
{
    e[0] = v.x;
    e[1] = v.y;
}
__device__ __forceinline__ double2 pack(const double (&e)[2]) { return make_double2(e[0], e[1]); }
__device__ __forceinline__ void unpack(const float4& v, float (&e)[4])
{
    e[0] = v.x;
    e[1] = v.y;
    e[2] = v.z;
    e[3] = v.w;
}
__device__ __forceinline__ float4 pack(const float (&e)[4]) { return make_float4(e[0], e[1], e[2], e[3]); }

template <typename T, int NIN, int NOUT, class Op>
__device__ __forceinline__ void scalar_at(const Args<T, NIN, NOUT>& a, const Op& op, size_t i)
{
    T x[NIN];
    T y[NOUT];
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = a.in[k][i];
    op(x, y);
#pragma unroll
    for (int k = 0; k < NOUT; ++k) a.out[k][i] = y[k];
}

// Apply the op to the E values of one vector per input and store one vector
// per output at vector index j.
template <typename T, int NIN, int NOUT, class Op>
__device__ __forceinline__ void apply_vec(const Op& op, const typename Vec<T>::V (&x)[NIN],
                                          typename Vec<T>::V* const (&out)[NOUT], size_t j)
{
    constexpr int E = Vec<T>::E;
    T xe[NIN][E];
#pragma unroll
    for (int k = 0; k < NIN; ++k) unpack(x[k], xe[k]);
    T ye[NOUT][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        T xs[NIN];
        T ys[NOUT];
#pragma unroll
        for (int k = 0; k < NIN; ++k) xs[k] = xe[k][e];
        op(xs, ys);
#pragma unroll
        for (int k = 0; k < NOUT; ++k) ye[k][e] = ys[k];
    }
#pragma unroll
    for (int k = 0; k < NOUT; ++k) __stcs(out[k] + j, pack(ye[k]));
}

// Vector path: elements [0, head) and the tail are scalar; the body is
// processed as 16-byte vectors, U per input per thread per sweep.  The sweep
// is software-pipelined: the loads of sweep s + 1 are issued before the
// values of sweep s are computed and stored, so each thread keeps loads in
// flight while it computes.  (The scalar head and tail come after the sweep:
// placed before it, they made the compiler schedule the Add22 loop worse.)
template <typename T, int NIN, int NOUT, class Op, int U>
__global__ void __launch_bounds__(kBlock) stream_vec(Args<T, NIN, NOUT> a, Op op)
{
    using V = typename Vec<T>::V;
    constexpr int E = Vec<T>::E;
    const size_t tid = static_cast<size_t>(blockIdx.x) * kBlock + threadIdx.x;
    const size_t nthr = static_cast<size_t>(gridDim.x) * kBlock;
    const size_t head = static_cast<size_t>(a.head);
    const size_t nv = (a.n - head) / E;            // full vectors
    const size_t tail0 = head + nv * E;            // first tail element

    const V* in[NIN];
    V* out[NOUT];
#pragma unroll
    for (int k = 0; k < NIN; ++k) in[k] = reinterpret_cast<const V*>(a.in[k] + head);
#pragma unroll
    for (int k = 0; k < NOUT; ++k) out[k] = reinterpret_cast<V*>(a.out[k] + head);

    size_t i = tid;
    bool full = i + (U - 1) * nthr < nv;
    V cur[U][NIN];
    if (full) {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < NIN; ++k) cur[u][k] = __ldcs(in[k] + i + u * nthr);
    }
    while (full) {
        const size_t nx = i + U * nthr;
        const bool nfull = nx + (U - 1) * nthr < nv;
        V nxt[U][NIN];
        if (nfull) {
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int k = 0; k < NIN; ++k) nxt[u][k] = __ldcs(in[k] + nx + u * nthr);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) apply_vec<T, NIN, NOUT>(op, cur[u], out, i + u * nthr);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < NIN; ++k) cur[u][k] = nxt[u][k];
        i = nx;
        full = nfull;
    }
    for (; i < nv; i += nthr) {
        V x[NIN];
#pragma unroll
        for (int k = 0; k < NIN; ++k) x[k] = __ldcs(in[k] + i);
        apply_vec<T, NIN, NOUT>(op, x, out, i);
    }

    if (tid < head) scalar_at(a, op, tid);
    if (tid < a.n - tail0) scalar_at(a, op, tail0 + tid);
}

// Scalar path for arrays whose offsets modulo 16 bytes differ.
template <typename T, int NIN, int NOUT, class Op, int U>
__global__ void __launch_bounds__(kBlock) stream_scalar(Args<T, NIN, NOUT> a, Op op)
{
    const size_t tid = static_cast<size_t>(blockIdx.x) * kBlock + threadIdx.x;
    const size_t nthr = static_cast<size_t>(gridDim.x) * kBlock;
    size_t i = tid;
    for (; i + (U - 1) * nthr < a.n; i += U * nthr) {
        T x[U][NIN];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < NIN; ++k) x[u][k] = a.in[k][i + u * nthr];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            T y[NOUT];
            op(x[u], y);
#pragma unroll
            for (int k = 0; k < NOUT; ++k) a.out[k][i + u * nthr] = y[k];
        }
    }
    for (; i < a.n; i += nthr) scalar_at(a, op, i);
}

// Resident 256-thread blocks per SM by number of input arrays (see above).
constexpr int blocks_per_sm(int nin) { return nin == 1 ? 4 : nin == 2 ? 3 : 2; }

// Host launcher: validates nothing (the caller did), picks the path and the
// grid, launches on `s`.
template <typename T, int NIN, int NOUT, class Op, int U = 2>
ff_status launch(Args<T, NIN, NOUT> a, Op op, cudaStream_t s)
{
    if (a.n == 0) return FF_OK;
    ffh::DeviceInfo di;
    ff_status st = ffh::device_info(&di);
    if (st != FF_OK) return st;
    constexpr int E = Vec<T>::E;
    // offset of each array modulo 16 bytes, in elements
    uintptr_t phase = reinterpret_cast<uintptr_t>(a.in[0]) & 15u;
    bool same = true;
    for (int k = 1; k < NIN; ++k) same &= ((reinterpret_cast<uintptr_t>(a.in[k]) & 15u) == phase);
    for (int k = 0; k < NOUT; ++k) same &= ((reinterpret_cast<uintptr_t>(a.out[k]) & 15u) == phase);
    if (same && (phase % sizeof(T)) == 0) {
        size_t head = phase ? (16u - phase) / sizeof(T) : 0;
        if (head > a.n) head = a.n;
        a.head = static_cast<int>(head);
        const void* kern = reinterpret_cast<const void*>(&stream_vec<T, NIN, NOUT, Op, U>);
        int occ = ffh::occupancy(kern, kBlock);
        if (occ > blocks_per_sm(NIN)) occ = blocks_per_sm(NIN);
        const size_t nv = (a.n - head) / E;
        unsigned grid = ffh::grid_for(nv > 0 ? nv : 1, static_cast<size_t>(kBlock) * U, di.sm_count, occ);
        stream_vec<T, NIN, NOUT, Op, U><<<grid, kBlock, 0, s>>>(a, op);
    } else {
        a.head = 0;
        const void* kern = reinterpret_cast<const void*>(&stream_scalar<T, NIN, NOUT, Op, U>);
        int occ = ffh::occupancy(kern, kBlock);
        if (occ > 2 * blocks_per_sm(NIN)) occ = 2 * blocks_per_sm(NIN);
        unsigned grid = ffh::grid_for(a.n, static_cast<size_t>(kBlock) * U, di.sm_count, occ);
        stream_scalar<T, NIN, NOUT, Op, U><<<grid, kBlock, 0, s>>>(a, op);
    }
    return ffh::check_launch();
}

}  // namespace ffst
