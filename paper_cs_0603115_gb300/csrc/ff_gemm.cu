// ff_gemm.cu -- float-float matrix product C = op(A) op(B), each term a Mul22
// and each accumulation an Add22 (the paper's operators, Section 4.1).
//
// Every output accumulates its terms in increasing order of the inner index,
// starting from (0, 0), one thread per output: the result does not depend on
// the launch shape and equals the plain triple loop bit for bit.
//
// The work is FP32-instruction bound (about 28 instructions per term, 8
// bytes of A and B read from L2 per 64 terms), so the kernel is shaped for
// issue rate: a 256-thread block computes a 64 x 64 tile of C, each thread a
// 4 x 4 sub-tile (16 independent Add22 chains).  The A and B panels of the
// current K slice (16 values deep) sit in shared memory, double buffered; the
// next slice is loaded into registers while the current one is computed.
// Two blocks per SM (121 registers a thread) keep 16 warps resident.
// Global loads are coalesced for each operand layout (row-major or
// transposed); the shared-memory tiles are k-major with one padding value per
// row so that the transposing stores do not serialise on one bank.
#include "ff_core.cuh"
#include "ff_host.cuh"

namespace {

constexpr int kBM = 64;              // rows of C per block
constexpr int kBN = 64;              // columns of C per block
constexpr int kBK = 16;              // inner-index depth of one shared slice
constexpr int kThreads = 256;        // 16 x 16 threads, 4 x 4 outputs each
constexpr int kLdS = kBM + 1;        // shared row length (kBM == kBN)
constexpr int kLoads = kBM * kBK / kThreads;  // values of one operand slice per thread

static_assert(kBM == kBN, "one shared row length serves both operands");
static_assert(kLoads == 4, "load mappings below assume four values per thread");

struct Dims {
    int64_t m, n, k, lda, ldb, ldc;
    int64_t tiles_n, tiles;
};

// Slice `p0` of op(A) into registers: op(A)[i0 + r, p0 + c] for the 64 x 16
// slice.  Row-major A (TA = false) is contiguous along the inner index: a
// thread reads column c = t & 15 of rows (t >> 4) + 16 s.  Transposed A is
// contiguous along i: a thread reads row i = t & 63 of inner indices
// (t >> 6) + 4 s.  Out-of-range values read as (0, 0); they are never used
// for a stored output nor for a term beyond k.
template <bool TA>
__device__ __forceinline__ void load_a(const float2* __restrict__ A, const Dims& d, int64_t i0, int64_t p0,
                                       float2 (&v)[kLoads])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int s = 0; s < kLoads; ++s) {
        int64_t i, p;
        if (!TA) {
            i = i0 + (t >> 4) + 16 * s;
            p = p0 + (t & 15);
        } else {
            i = i0 + (t & 63);
            p = p0 + (t >> 6) + 4 * s;
        }
        const bool in = (i < d.m) && (p < d.k);
        v[s] = in ? __ldg(TA ? A + p * d.lda + i : A + i * d.lda + p) : make_float2(0.0f, 0.0f);
    }
}

template <bool TA>
__device__ __forceinline__ void store_a(float2 (*As)[kLdS], const float2 (&v)[kLoads])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int s = 0; s < kLoads; ++s) {
        if (!TA)
            As[t & 15][(t >> 4) + 16 * s] = v[s];
        else
            As[(t >> 6) + 4 * s][t & 63] = v[s];
    }
}

// Slice `p0` of op(B): op(B)[p0 + r, j0 + c], 16 x 64.  Row-major B
// (TB = false) is contiguous along j; transposed B along the inner index.
template <bool TB>
__device__ __forceinline__ void load_b(const float2* __restrict__ B, const Dims& d, int64_t j0, int64_t p0,
                                       float2 (&v)[kLoads])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int s = 0; s < kLoads; ++s) {
        int64_t j, p;
        if (!TB) {
            j = j0 + (t & 63);
            p = p0 + (t >> 6) + 4 * s;
        } else {
            j = j0 + (t >> 4) + 16 * s;
            p = p0 + (t & 15);
        }
        const bool in = (j < d.n) && (p < d.k);
        v[s] = in ? __ldg(TB ? B + j * d.ldb + p : B + p * d.ldb + j) : make_float2(0.0f, 0.0f);
    }
}

template <bool TB>
__device__ __forceinline__ void store_b(float2 (*Bs)[kLdS], const float2 (&v)[kLoads])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int s = 0; s < kLoads; ++s) {
        if (!TB)
            Bs[(t >> 6) + 4 * s][t & 63] = v[s];
        else
            Bs[t & 15][(t >> 4) + 16 * s] = v[s];
    }
}

// One inner index of the slice: 16 terms, one per accumulator.
__device__ __forceinline__ void step(const float2 (*As)[kLdS], const float2 (*Bs)[kLdS], int kk, int ty, int tx,
                                     float2 (&acc)[4][4])
{
    float2 a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
    for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = ffk::add22(acc[r][c], ffk::mul22(a[r], b[c]));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(kThreads, 2)
gemm_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C, Dims d)
{
    __shared__ float2 As[2][kBK][kLdS];
    __shared__ float2 Bs[2][kBK][kLdS];
    const int tx = threadIdx.x & 15;
    const int ty = threadIdx.x >> 4;
    const int64_t nslices = (d.k + kBK - 1) / kBK;

    for (int64_t tile = blockIdx.x; tile < d.tiles; tile += gridDim.x) {
        const int64_t i0 = (tile / d.tiles_n) * kBM;
        const int64_t j0 = (tile % d.tiles_n) * kBN;
        float2 acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.0f, 0.0f);

        float2 va[kLoads], vb[kLoads];
        if (nslices > 0) {
            load_a<TA>(A, d, i0, 0, va);
            load_b<TB>(B, d, j0, 0, vb);
            store_a<TA>(As[0], va);
            store_b<TB>(Bs[0], vb);
        }
        __syncthreads();
        for (int64_t sl = 0; sl < nslices; ++sl) {
            const int cur = static_cast<int>(sl & 1);
            const bool more = sl + 1 < nslices;
            if (more) {
                load_a<TA>(A, d, i0, (sl + 1) * kBK, va);
                load_b<TB>(B, d, j0, (sl + 1) * kBK, vb);
            }
            const int64_t rem = d.k - sl * kBK;
            if (rem >= kBK) {
                // Unrolled by two, not sixteen: one inner index is ~460
                // instructions, and the fully unrolled slice (~7,300) overflows
                // the instruction cache (measured: 0.74 -> 0.88 of FP32 issue).
#pragma unroll 2
                for (int kk = 0; kk < kBK; ++kk) step(As[cur], Bs[cur], kk, ty, tx, acc);
            } else {
                for (int kk = 0; kk < static_cast<int>(rem); ++kk) step(As[cur], Bs[cur], kk, ty, tx, acc);
            }
            if (more) {
                store_a<TA>(As[cur ^ 1], va);
                store_b<TB>(Bs[cur ^ 1], vb);
            }
            __syncthreads();
        }

#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t i = i0 + ty + 16 * r;
            if (i >= d.m) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t j = j0 + tx + 16 * c;
                if (j < d.n) C[i * d.ldc + j] = acc[r][c];
            }
        }
    }
}

template <bool TA, bool TB>
ff_status launch(const float2* A, const float2* B, float2* C, const Dims& d, cudaStream_t s)
{
    // one block per tile up to the 1-D grid limit; blocks loop over the rest
    const int64_t cap = 0x7fffffffLL;
    const unsigned grid = static_cast<unsigned>(d.tiles < cap ? d.tiles : cap);
    gemm_kernel<TA, TB><<<grid, kThreads, 0, s>>>(A, B, C, d);
    return ffh::check_launch();
}

}  // namespace

extern "C" {

ff_status ff_gemm(int transa, int transb, int64_t m, int64_t n, int64_t k, const ff2* A_, int64_t lda,
                  const ff2* B_, int64_t ldb, ff2* C_, int64_t ldc, cudaStream_t s)
{
    if (m < 0 || n < 0 || k < 0) return FF_ERR_INVALID_ARG;
    if ((transa != 0 && transa != 1) || (transb != 0 && transb != 1)) return FF_ERR_INVALID_ARG;
    const int64_t a_cols = transa ? m : k;  // row length of A as stored
    const int64_t b_cols = transb ? k : n;
    if (lda < (a_cols > 1 ? a_cols : 1) || ldb < (b_cols > 1 ? b_cols : 1) || ldc < (n > 1 ? n : 1))
        return FF_ERR_INVALID_ARG;
    if (m == 0 || n == 0) return FF_OK;  // nothing to write, no pointer read
    const size_t an = static_cast<size_t>(m) * static_cast<size_t>(k);
    const size_t bn = static_cast<size_t>(k) * static_cast<size_t>(n);
    const size_t cn = static_cast<size_t>(m) * static_cast<size_t>(n);
    if (!ffh::ok_ptr(A_, an) || !ffh::ok_ptr(B_, bn) || !ffh::ok_ptr(C_, cn)) return FF_ERR_INVALID_ARG;
    Dims d;
    d.m = m; d.n = n; d.k = k; d.lda = lda; d.ldb = ldb; d.ldc = ldc;
    d.tiles_n = (n + kBN - 1) / kBN;
    d.tiles = ((m + kBM - 1) / kBM) * d.tiles_n;
    auto* A = reinterpret_cast<const float2*>(A_);
    auto* B = reinterpret_cast<const float2*>(B_);
    auto* C = reinterpret_cast<float2*>(C_);
    if (!transa && !transb) return launch<false, false>(A, B, C, d, s);
    if (transa && !transb) return launch<true, false>(A, B, C, d, s);
    if (!transa && transb) return launch<false, true>(A, B, C, d, s);
    return launch<true, true>(A, B, C, d, s);
}

}  // extern "C"
