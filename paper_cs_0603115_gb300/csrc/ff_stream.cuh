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
// kernels with about 40-50 KB of loads in flight per SM, not with every SM
// full: measured on 2^28 values, Add22 reaches ~7.0 TB/s with U = 2 and 3
// blocks of 256 per SM against ~6.6 TB/s at full occupancy, and the
// one-input kernels ~6.6 TB/s with U = 2 and 5 blocks per SM.  The launcher
// therefore caps the grid at SMs x kBlocksPerSm[NIN].
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

template <typename T>
union Pack {
    typename Vec<T>::V v;
    T e[Vec<T>::E];
};

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

// Vector path: elements [0, head) and the tail are scalar; the body is
// processed as 16-byte vectors, U per input per thread per sweep.
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

    if (tid < head) scalar_at(a, op, tid);
    if (tid < a.n - tail0) scalar_at(a, op, tail0 + tid);

    const V* in[NIN];
    V* out[NOUT];
#pragma unroll
    for (int k = 0; k < NIN; ++k) in[k] = reinterpret_cast<const V*>(a.in[k] + head);
#pragma unroll
    for (int k = 0; k < NOUT; ++k) out[k] = reinterpret_cast<V*>(a.out[k] + head);

    size_t i = tid;
    for (; i + (U - 1) * nthr < nv; i += U * nthr) {
        Pack<T> x[U][NIN];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < NIN; ++k) x[u][k].v = __ldcs(in[k] + i + u * nthr);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            Pack<T> y[NOUT];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                T xs[NIN];
                T ys[NOUT];
#pragma unroll
                for (int k = 0; k < NIN; ++k) xs[k] = x[u][k].e[e];
                op(xs, ys);
#pragma unroll
                for (int k = 0; k < NOUT; ++k) y[k].e[e] = ys[k];
            }
#pragma unroll
            for (int k = 0; k < NOUT; ++k) __stcs(out[k] + i + u * nthr, y[k].v);
        }
    }
    for (; i < nv; i += nthr) {
        Pack<T> x[NIN];
#pragma unroll
        for (int k = 0; k < NIN; ++k) x[k].v = __ldcs(in[k] + i);
        Pack<T> y[NOUT];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            T xs[NIN];
            T ys[NOUT];
#pragma unroll
            for (int k = 0; k < NIN; ++k) xs[k] = x[k].e[e];
            op(xs, ys);
#pragma unroll
            for (int k = 0; k < NOUT; ++k) y[k].e[e] = ys[k];
        }
#pragma unroll
        for (int k = 0; k < NOUT; ++k) __stcs(out[k] + i, y[k].v);
    }
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
constexpr int blocks_per_sm(int nin) { return nin == 1 ? 5 : nin == 2 ? 3 : 2; }

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
