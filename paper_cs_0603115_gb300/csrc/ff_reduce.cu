// ff_reduce.cu -- deterministic compensated reductions: the float-float sum
// and dot product (Add22 accumulation of the paper's operators, the
// compensated algorithms Section 7 names as future work) and a binary64 dot
// baseline.
//
// One launch per reduction.  Order of combination (fixed for a given n,
// device and build, hence bit-reproducible):
//   1. thread t of T = grid x 256 threads starts from zero and accumulates,
//      left to right, the head elements before the first 16-byte boundary
//      (thread 0 only; none when the arrays are 16-byte aligned), then the
//      16-byte chunks t, t + T, t + 2T, ... (E = 2 float-float or binary64
//      values, 4 binary32 values; the values of chunk c in increasing
//      order), then the tail elements after the last whole chunk (thread 0
//      only).  Arrays whose offsets modulo 16 bytes differ take one element
//      per step instead: elements t, t + T, t + 2T, ...;
//   2. each warp combines lanes with a shuffle-down tree
//      (v_l = combine(v_l, v_{l+off}), off = 16, 8, 4, 2, 1);
//   3. lane 0 of each warp stores its value; warp 0 combines the 8 warp
//      values with the same tree (off = 4, 2, 1);
//   4. every block stores its value in the workspace; the last block to
//      arrive (atomic ticket) accumulates the block values b, b + 256, ... per
//      thread, from zero, and reduces them with steps 2-3, then sets the
//      ticket back to zero (the caller zeroes a workspace once, before its
//      first use, so a call is a single launch).
// No block ever waits for another.
#include <mutex>

#include "ff_core.cuh"
#include "ff_host.cuh"

namespace {

constexpr int kRBlock = 256;
constexpr int kRWarps = kRBlock / 32;
// Resident 256-thread blocks per SM at most: a read-only stream reaches a
// higher DRAM rate with moderate residency than with every SM full (ff_sum
// at 2^26 / 2^28: 0.97 / 1.02 of the measured copy rate with 8 blocks,
// 0.995 / 1.06 with 6; ff_dot is held at 6 by its registers either way).
constexpr int kRMaxBlocksPerSm = 6;
constexpr size_t kPartialsOffset = 256;  // ticket at offset 0, partials at 256

struct FFSum {
    using T = float2;
    using Acc = float2;
    static constexpr bool kDot = false;
    __device__ static Acc finalize(Acc a) { return a; }
    __device__ static Acc zero() { return make_float2(0.0f, 0.0f); }
    __device__ static Acc step(Acc acc, T x, T) { return ffk::add22(acc, x); }
    __device__ static Acc combine(Acc a, Acc b) { return ffk::add22(a, b); }
    __device__ static Acc shfl_down(Acc v, int off)
    {
        return make_float2(__shfl_down_sync(0xffffffffu, v.x, off), __shfl_down_sync(0xffffffffu, v.y, off));
    }
};

struct FFDot : FFSum {
    static constexpr bool kDot = true;
    __device__ static Acc step(Acc acc, T x, T y) { return ffk::add22(acc, ffk::mul22(x, y)); }
};

struct F64Dot {
    using T = double;
    using Acc = double;
    static constexpr bool kDot = true;
    __device__ static Acc finalize(Acc a) { return a; }
    __device__ static Acc zero() { return 0.0; }
    __device__ static Acc step(Acc acc, T x, T y) { return __fma_rn(x, y, acc); }
    __device__ static Acc combine(Acc a, Acc b) { return __dadd_rn(a, b); }
    __device__ static Acc shfl_down(Acc v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }
};

// Compensated Sum2 / Dot2 of binary32 vectors (Ogita, Rump and Oishi 2005)
// with the accumulator (p, s): p the running sum, s the running sum of the
// exact errors.  Step: (h, r) = TwoProduct(x, y); (p, q) = TwoSum(p, h);
// s = s + (q + r) (Sum2: h = x, r = 0).  Two accumulators combine as
// (p, q) = TwoSum(a.p, b.p); s = a.s + (b.s + q).  The result is the
// float-float Add12(p, s), equal to p + s exactly.
struct F32Sum2 {
    using T = float;
    using Acc = float2;  // (p, s)
    static constexpr bool kDot = false;
    __device__ static Acc zero() { return make_float2(0.0f, 0.0f); }
    __device__ static Acc step(Acc a, T x, T)
    {
        const float2 pq = ffk::add12(a.x, x);
        return make_float2(pq.x, __fadd_rn(a.y, pq.y));
    }
    __device__ static Acc combine(Acc a, Acc b)
    {
        const float2 pq = ffk::add12(a.x, b.x);
        return make_float2(pq.x, __fadd_rn(a.y, __fadd_rn(b.y, pq.y)));
    }
    __device__ static Acc finalize(Acc a) { return ffk::add12(a.x, a.y); }
    __device__ static Acc shfl_down(Acc v, int off)
    {
        return make_float2(__shfl_down_sync(0xffffffffu, v.x, off), __shfl_down_sync(0xffffffffu, v.y, off));
    }
};

struct F32Dot2 : F32Sum2 {
    static constexpr bool kDot = true;
    __device__ static Acc step(Acc a, T x, T y)
    {
        const float2 hr = ffk::mul12(x, y);
        const float2 pq = ffk::add12(a.x, hr.x);
        return make_float2(pq.x, __fadd_rn(a.y, __fadd_rn(pq.y, hr.y)));
    }
};

template <typename T> struct V16;
template <> struct V16<float2> { using V = float4; static constexpr int E = 2; };
template <> struct V16<double> { using V = double2; static constexpr int E = 2; };
template <> struct V16<float> { using V = float4; static constexpr int E = 4; };

// Explicit split of a 16-byte vector into its values (see ff_stream.cuh on
// why not a union).
__device__ __forceinline__ void split_vec(const float4& v, float2 (&e)[2])
{
    e[0] = make_float2(v.x, v.y);
    e[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void split_vec(const double2& v, double (&e)[2])
{
    e[0] = v.x;
    e[1] = v.y;
}
__device__ __forceinline__ void split_vec(const float4& v, float (&e)[4])
{
    e[0] = v.x;
    e[1] = v.y;
    e[2] = v.z;
    e[3] = v.w;
}

// Steps 2-3: the block's combined value ends in thread 0.
template <class P>
__device__ __forceinline__ typename P::Acc block_reduce(typename P::Acc v, typename P::Acc* sm)
{
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = P::combine(v, P::shfl_down(v, off));
    if (lane == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (lane < kRWarps) ? sm[lane] : P::zero();
#pragma unroll
        for (int off = kRWarps / 2; off > 0; off >>= 1) v = P::combine(v, P::shfl_down(v, off));
    }
    __syncthreads();
    return v;
}

template <class P, int U>
__global__ void __launch_bounds__(kRBlock)
reduce_kernel(const typename P::T* x, const typename P::T* y, size_t n, int head, typename P::Acc* out,
              typename P::Acc* partials, unsigned* ticket)
{
    using T = typename P::T;
    using Acc = typename P::Acc;
    using V = typename V16<T>::V;
    __shared__ Acc sm[kRWarps];
    __shared__ bool is_last;

    constexpr int E = V16<T>::E;
    const size_t tid = static_cast<size_t>(blockIdx.x) * kRBlock + threadIdx.x;
    const size_t nthr = static_cast<size_t>(gridDim.x) * kRBlock;
    const size_t h = static_cast<size_t>(head);
    const size_t nv = (n - h) / E;

    Acc acc = P::zero();
    if (tid == 0)
        for (size_t j = 0; j < h; ++j) acc = P::step(acc, x[j], P::kDot ? y[j] : T());

    const V* xv = reinterpret_cast<const V*>(x + h);
    const V* yv = reinterpret_cast<const V*>((P::kDot ? y : x) + h);
    size_t i = tid;
    for (; i + (U - 1) * nthr < nv; i += U * nthr) {
        V xs[U], ys[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xs[u] = __ldcs(xv + i + u * nthr);
            if (P::kDot) ys[u] = __ldcs(yv + i + u * nthr);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            T xe[E], ye[E];
            split_vec(xs[u], xe);
            if (P::kDot) split_vec(ys[u], ye);
#pragma unroll
            for (int e = 0; e < E; ++e) acc = P::step(acc, xe[e], P::kDot ? ye[e] : T());
        }
    }
    for (; i < nv; i += nthr) {
        V xs, ys;
        xs = __ldcs(xv + i);
        if (P::kDot) ys = __ldcs(yv + i);
        T xe[E], ye[E];
        split_vec(xs, xe);
        if (P::kDot) split_vec(ys, ye);
#pragma unroll
        for (int e = 0; e < E; ++e) acc = P::step(acc, xe[e], P::kDot ? ye[e] : T());
    }
    if (tid == 0)
        for (size_t j = h + nv * E; j < n; ++j) acc = P::step(acc, x[j], P::kDot ? y[j] : T());

    acc = block_reduce<P>(acc, sm);
    if (gridDim.x == 1) {
        if (threadIdx.x == 0) *out = P::finalize(acc);
        return;
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = acc;
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    Acc a2 = P::zero();
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kRBlock) a2 = P::combine(a2, __ldcg(partials + b));
    a2 = block_reduce<P>(a2, sm);
    if (threadIdx.x == 0) {
        *out = P::finalize(a2);
        *ticket = 0u;
    }
}

// Unaligned operands (offsets modulo 16 differ): scalar loads, same tree.
template <class P>
__global__ void __launch_bounds__(kRBlock)
reduce_scalar_kernel(const typename P::T* x, const typename P::T* y, size_t n, typename P::Acc* out,
                     typename P::Acc* partials, unsigned* ticket)
{
    using T = typename P::T;
    using Acc = typename P::Acc;
    __shared__ Acc sm[kRWarps];
    __shared__ bool is_last;
    const size_t tid = static_cast<size_t>(blockIdx.x) * kRBlock + threadIdx.x;
    const size_t nthr = static_cast<size_t>(gridDim.x) * kRBlock;
    Acc acc = P::zero();
    for (size_t i = tid; i < n; i += nthr) acc = P::step(acc, x[i], P::kDot ? y[i] : T());
    acc = block_reduce<P>(acc, sm);
    if (gridDim.x == 1) {
        if (threadIdx.x == 0) *out = P::finalize(acc);
        return;
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = acc;
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    Acc a2 = P::zero();
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kRBlock) a2 = P::combine(a2, __ldcg(partials + b));
    a2 = block_reduce<P>(a2, sm);
    if (threadIdx.x == 0) {
        *out = P::finalize(a2);
        *ticket = 0u;
    }
}

constexpr int kU = 4;

size_t max_blocks(const ffh::DeviceInfo& di) { return static_cast<size_t>(di.sm_count) * kRMaxBlocksPerSm; }

size_t workspace_bytes(const ffh::DeviceInfo& di) { return kPartialsOffset + max_blocks(di) * 8; }

struct Shape {
    unsigned grid;
    int head;
    bool vec;
};

template <class P>
Shape shape_for(const typename P::T* x, const typename P::T* y, size_t n, const ffh::DeviceInfo& di)
{
    using T = typename P::T;
    const uintptr_t px = reinterpret_cast<uintptr_t>(x) & 15u;
    const uintptr_t py = P::kDot ? (reinterpret_cast<uintptr_t>(y) & 15u) : px;
    Shape sh{};
    sh.vec = (px == py) && (px % sizeof(T) == 0);
    const size_t cap = max_blocks(di);
    if (sh.vec) {
        constexpr int E = V16<T>::E;
        sh.head = px != 0 ? static_cast<int>((16u - px) / sizeof(T)) : 0;
        if (static_cast<size_t>(sh.head) > n) sh.head = static_cast<int>(n);
        const void* kern = reinterpret_cast<const void*>(&reduce_kernel<P, kU>);
        int occ = ffh::occupancy(kern, kRBlock);
        if (occ > kRMaxBlocksPerSm) occ = kRMaxBlocksPerSm;
        const size_t nv = n > static_cast<size_t>(sh.head) ? (n - sh.head) / E : 0;
        sh.grid = ffh::grid_for(nv, static_cast<size_t>(kRBlock) * kU, di.sm_count, occ);
    } else {
        sh.head = 0;
        const void* kern = reinterpret_cast<const void*>(&reduce_scalar_kernel<P>);
        int occ = ffh::occupancy(kern, kRBlock);
        if (occ > kRMaxBlocksPerSm) occ = kRMaxBlocksPerSm;
        sh.grid = ffh::grid_for(n, static_cast<size_t>(kRBlock) * kU, di.sm_count, occ);
    }
    if (sh.grid > cap) sh.grid = static_cast<unsigned>(cap);
    return sh;
}

template <class P>
ff_status run_reduce(const typename P::T* x, const typename P::T* y, size_t n, typename P::Acc* out, void* ws,
                     size_t ws_bytes, cudaStream_t s)
{
    using T = typename P::T;
    auto ok_in = [n](const void* p) { return n == 0 || (p != nullptr && ffh::aligned(p, sizeof(T))); };
    if (!ok_in(x) || (P::kDot && !ok_in(y))) return FF_ERR_INVALID_ARG;
    if (!ffh::ok_ptr(out, 1)) return FF_ERR_INVALID_ARG;
    ffh::DeviceInfo di;
    ff_status st = ffh::device_info(&di);
    if (st != FF_OK) return st;
    if (ws == nullptr || ws_bytes < workspace_bytes(di) || !ffh::aligned(ws, 16)) return FF_ERR_WORKSPACE;

    unsigned* ticket = static_cast<unsigned*>(ws);
    auto* partials = reinterpret_cast<typename P::Acc*>(static_cast<char*>(ws) + kPartialsOffset);
    const Shape sh = shape_for<P>(x, y, n, di);
    // No clearing launch: the ticket is zero on entry (the workspace contract)
    // and the last block resets it to zero before the kernel ends.
    if (sh.vec)
        reduce_kernel<P, kU><<<sh.grid, kRBlock, 0, s>>>(x, y, n, sh.head, out, partials, ticket);
    else
        reduce_scalar_kernel<P><<<sh.grid, kRBlock, 0, s>>>(x, y, n, out, partials, ticket);
    return ffh::check_launch();
}

}  // namespace

extern "C" {

size_t ff_reduce_workspace_bytes(size_t n)
{
    (void)n;
    ffh::DeviceInfo di;
    if (ffh::device_info(&di) != FF_OK) return kPartialsOffset + 1024 * 8 * 8;
    return workspace_bytes(di);
}

ff_status ff_reduce_launch_shape(const ff2* x, const ff2* y, size_t n, unsigned* grid, int* head, int* vector)
{
    if (!grid || !head || !vector) return FF_ERR_INVALID_ARG;
    ffh::DeviceInfo di;
    ff_status st = ffh::device_info(&di);
    if (st != FF_OK) return st;
    Shape sh = y ? shape_for<FFDot>(reinterpret_cast<const float2*>(x), reinterpret_cast<const float2*>(y), n, di)
                 : shape_for<FFSum>(reinterpret_cast<const float2*>(x), nullptr, n, di);
    *grid = sh.grid;
    *head = sh.head;
    *vector = sh.vec ? 1 : 0;
    return FF_OK;
}

ff_status ff_sum(const ff2* x, size_t n, ff2* out_dev, void* ws, size_t ws_bytes, cudaStream_t s)
{
    return run_reduce<FFSum>(reinterpret_cast<const float2*>(x), nullptr, n, reinterpret_cast<float2*>(out_dev), ws,
                             ws_bytes, s);
}

ff_status ff_dot(const ff2* x, const ff2* y, size_t n, ff2* out_dev, void* ws, size_t ws_bytes, cudaStream_t s)
{
    return run_reduce<FFDot>(reinterpret_cast<const float2*>(x), reinterpret_cast<const float2*>(y), n,
                             reinterpret_cast<float2*>(out_dev), ws, ws_bytes, s);
}

ff_status ff_sum2(const float* x, size_t n, ff2* out_dev, void* ws, size_t ws_bytes, cudaStream_t s)
{
    if (!(n == 0 || (x != nullptr && ffh::aligned(x, 4)))) return FF_ERR_INVALID_ARG;
    return run_reduce<F32Sum2>(x, nullptr, n, reinterpret_cast<float2*>(out_dev), ws, ws_bytes, s);
}

ff_status ff_dot2(const float* x, const float* y, size_t n, ff2* out_dev, void* ws, size_t ws_bytes,
                  cudaStream_t s)
{
    if (!(n == 0 || (x != nullptr && y != nullptr && ffh::aligned(x, 4) && ffh::aligned(y, 4))))
        return FF_ERR_INVALID_ARG;
    return run_reduce<F32Dot2>(x, y, n, reinterpret_cast<float2*>(out_dev), ws, ws_bytes, s);
}

ff_status ff_reduce2_launch_shape(const float* x, const float* y, size_t n, unsigned* grid, int* head, int* vector)
{
    if (!grid || !head || !vector) return FF_ERR_INVALID_ARG;
    ffh::DeviceInfo di;
    ff_status st = ffh::device_info(&di);
    if (st != FF_OK) return st;
    Shape sh = y ? shape_for<F32Dot2>(x, y, n, di) : shape_for<F32Sum2>(x, nullptr, n, di);
    *grid = sh.grid;
    *head = sh.head;
    *vector = sh.vec ? 1 : 0;
    return FF_OK;
}

ff_status ff_f64_dot(const double* x, const double* y, size_t n, double* out_dev, void* ws, size_t ws_bytes,
                     cudaStream_t s)
{
    return run_reduce<F64Dot>(x, y, n, out_dev, ws, ws_bytes, s);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ff_dot_noalloc: ff_dot for callers that may not allocate device memory.
// Its scratch (the arrival ticket and the per-block partial sums) lives in
// one fixed array in this file instead of a caller-provided workspace.
// ---------------------------------------------------------------------------
namespace {
constexpr unsigned kNoAllocMaxBlocks = 2048;
constexpr size_t kNoAllocScratchBytes = kPartialsOffset + kNoAllocMaxBlocks * sizeof(float2);
}  // namespace

// One copy per device that loads the library, kept until the process exits.
static __device__ __align__(256) unsigned char g_dot_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
ff_status noalloc_scratch(int dev, void** out)
{
    constexpr int kMaxDev = 64;
    static void* addr[kMaxDev] = {};
    static std::mutex mu;
    if (dev < 0 || dev >= kMaxDev) return FF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (addr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dot_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return ffh::cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        addr[dev] = p;
    }
    *out = addr[dev];
    return FF_OK;
}

}  // namespace

extern "C" ff_status ff_dot_noalloc(const ff2* x_, const ff2* y_, size_t n, ff2* out_, cudaStream_t s)
{
    auto* x = reinterpret_cast<const float2*>(x_);
    auto* y = reinterpret_cast<const float2*>(y_);
    auto* out = reinterpret_cast<float2*>(out_);
    if (!ffh::ok_ptr(x, n) || !ffh::ok_ptr(y, n) || !ffh::ok_ptr(out, 1)) return FF_ERR_INVALID_ARG;
    ffh::DeviceInfo di;
    ff_status st = ffh::device_info(&di);
    if (st != FF_OK) return st;
    const Shape sh = shape_for<FFDot>(x, y, n, di);
    if (sh.grid > kNoAllocMaxBlocks) return FF_ERR_WORKSPACE;  // more partial sums than the array holds
    void* scratch = nullptr;
    st = noalloc_scratch(di.device, &scratch);
    if (st != FF_OK) return st;
    unsigned* ticket = static_cast<unsigned*>(scratch);
    auto* partials = reinterpret_cast<float2*>(static_cast<char*>(scratch) + kPartialsOffset);
    if (sh.grid > 1) {
        // the previous call left its contents; the ticket must start at zero
        st = ffh::cuda_status(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
        if (st != FF_OK) return st;
    }
    if (sh.vec)
        reduce_kernel<FFDot, kU><<<sh.grid, kRBlock, 0, s>>>(x, y, n, sh.head, out, partials, ticket);
    else
        reduce_scalar_kernel<FFDot><<<sh.grid, kRBlock, 0, s>>>(x, y, n, out, partials, ticket);
    return ffh::check_launch();
}
