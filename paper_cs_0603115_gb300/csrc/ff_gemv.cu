// ff_gemv.cu -- float-float GEMV Y = A X, its adjoint dX = A^T dY and the
// weight gradient dA = dY X^T, each term a Mul22 and each accumulation an
// Add22 (the paper's operators), plus a binary64 GEMV baseline with the same
// layouts.
//
// Layouts: A is m x n row-major (row stride lda); X, dX are n x k and Y, dY
// are m x k, all column-major (column strides ldx, lddx, ldy, lddy).
//
// ff_gemv: one warp per row, 8 rows per 256-thread block.  Lane l walks the
// row in two-column steps (j = 2l + 64t, 16-byte loads of A and of each
// column of X) and keeps KT float-float accumulators, one per right-hand
// side of the current column tile; k > KT is processed as successive tiles.
// The 32 lane accumulators are combined by a shuffle-down Add22 tree.
//
// ff_gemv_t: one thread per pair of adjacent columns of A (coalesced
// 16-byte loads along rows), one block row per row block of A.  Each thread
// accumulates its rows in order; the row blocks' partial sums go to the
// workspace and a second kernel adds them in row-block order.
//
// ff_gemv_dA: one thread per pair of adjacent columns of dA, the block's
// rows walked in pairs with dY staged in shared memory; every element adds
// its k terms in order from (0, 0), in one pass up to twelve right-hand
// sides and two above, or through the GEMM kernel for larger k.
#include "ff_core.cuh"
#include "ff_first_term.cuh"
#include "ff_host.cuh"

namespace {

constexpr int kGBlock = 256;
constexpr int kGWarps = kGBlock / 32;
constexpr int kMaxK = 64;
// Widest tile for which the forward kernel keeps four chunks per lane in flight.
constexpr int kGemvFourChunksMaxK = 7;

__device__ __forceinline__ float2 shfl_down2(float2 v, int off)
{
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, off), __shfl_down_sync(0xffffffffu, v.y, off));
}

// ---------------------------------------------------------------------------
// Y = A X
// ---------------------------------------------------------------------------
// Resident blocks per SM that the 16-byte forward kernel of a KT-wide tile
// is compiled for (0: the compiler's own choice).  Four for three to seven
// right-hand sides (32768^2: +0.3-1.4%); for two, a budget for 6 or 8
// blocks measured 4% and 14% slower than the compiler's own 48 registers.
constexpr int gemv_min_blocks(int kt, bool vec) { return vec && kt >= 3 && kt <= 7 ? 4 : 0; }

template <int KT, bool VEC>
__global__ void __launch_bounds__(kGBlock, gemv_min_blocks(KT, VEC))
gemv_kernel(const float2* __restrict__ A, int64_t m, int64_t n, int64_t lda, const float2* __restrict__ X,
            int64_t ldx, float2* __restrict__ Y, int64_t ldy)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * kGWarps + (threadIdx.x >> 5);
    if (r >= m) return;
    const float2* Ar = A + r * lda;
    float2 acc[KT];
#pragma unroll
    for (int c = 0; c < KT; ++c) acc[c] = make_float2(0.0f, 0.0f);

    if (VEC) {
        // two columns per lane per step; n even, A rows and X columns 16-byte aligned
        const float4* Ar4 = reinterpret_cast<const float4*>(Ar);
        const int64_t n2 = n >> 1;
        int64_t t = lane;
        // four chunks in flight per lane for narrow tiles (each lane still takes
        // its chunks t, t + 32, t + 64, ... in order): 32768^2, k = 2 / 3 /
        // 4-7 0.87 / 0.89 / 0.91-0.92 -> 0.89 / 0.92 / 0.93 of the FP32
        // roofline; at k = 1, where the stream is HBM-bound, it measured
        // slower (1.03 -> 0.94)
        if constexpr (KT >= 2 && KT <= kGemvFourChunksMaxK) {
            for (; t + 96 < n2; t += 128) {
                const float4 a0 = __ldcs(Ar4 + t), a1 = __ldcs(Ar4 + t + 32);
                const float4 a2 = __ldcs(Ar4 + t + 64), a3 = __ldcs(Ar4 + t + 96);
#pragma unroll
                for (int c = 0; c < KT; ++c) {
                    const float4* Xc = reinterpret_cast<const float4*>(X + c * ldx);
                    const float4 x0 = __ldg(Xc + t), x1 = __ldg(Xc + t + 32);
                    const float4 x2 = __ldg(Xc + t + 64), x3 = __ldg(Xc + t + 96);
                    acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a0.x, a0.y), make_float2(x0.x, x0.y)));
                    acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a0.z, a0.w), make_float2(x0.z, x0.w)));
                    acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a1.x, a1.y), make_float2(x1.x, x1.y)));
                    acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a1.z, a1.w), make_float2(x1.z, x1.w)));
                    acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a2.x, a2.y), make_float2(x2.x, x2.y)));
                    acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a2.z, a2.w), make_float2(x2.z, x2.w)));
                    acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a3.x, a3.y), make_float2(x3.x, x3.y)));
                    acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a3.z, a3.w), make_float2(x3.z, x3.w)));
                }
            }
        }
        for (; t + 32 < n2; t += 64) {
            const float4 a0 = __ldcs(Ar4 + t);
            const float4 a1 = __ldcs(Ar4 + t + 32);
#pragma unroll
            for (int c = 0; c < KT; ++c) {
                const float4* Xc = reinterpret_cast<const float4*>(X + c * ldx);
                const float4 x0 = __ldg(Xc + t);
                const float4 x1 = __ldg(Xc + t + 32);
                acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a0.x, a0.y), make_float2(x0.x, x0.y)));
                acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a0.z, a0.w), make_float2(x0.z, x0.w)));
                acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a1.x, a1.y), make_float2(x1.x, x1.y)));
                acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a1.z, a1.w), make_float2(x1.z, x1.w)));
            }
        }
        for (; t < n2; t += 32) {
            const float4 a0 = __ldcs(Ar4 + t);
#pragma unroll
            for (int c = 0; c < KT; ++c) {
                const float4 x0 = __ldg(reinterpret_cast<const float4*>(X + c * ldx) + t);
                acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a0.x, a0.y), make_float2(x0.x, x0.y)));
                acc[c] = ffk::add22(acc[c], ffk::mul22(make_float2(a0.z, a0.w), make_float2(x0.z, x0.w)));
            }
        }
    } else {
        for (int64_t j = lane; j < n; j += 32) {
            const float2 a = Ar[j];
#pragma unroll
            for (int c = 0; c < KT; ++c) acc[c] = ffk::add22(acc[c], ffk::mul22(a, __ldg(X + c * ldx + j)));
        }
    }
#pragma unroll
    for (int c = 0; c < KT; ++c) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[c] = ffk::add22(acc[c], shfl_down2(acc[c], off));
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < KT; ++c) Y[c * ldy + r] = acc[c];
    }
}

template <int KT>
ff_status launch_gemv_tile(const float2* A, int64_t m, int64_t n, int64_t lda, const float2* X, int64_t ldx,
                           float2* Y, int64_t ldy, bool vec, cudaStream_t s)
{
    const unsigned grid = static_cast<unsigned>((m + kGWarps - 1) / kGWarps);
    if (vec)
        gemv_kernel<KT, true><<<grid, kGBlock, 0, s>>>(A, m, n, lda, X, ldx, Y, ldy);
    else
        gemv_kernel<KT, false><<<grid, kGBlock, 0, s>>>(A, m, n, lda, X, ldx, Y, ldy);
    return ffh::check_launch();
}

// Tile width for the float-float kernels: up to seven right-hand sides in
// one pass (one read of A: below eight the kernels are issue-bound only
// once all k share the pass), else passes of eight.  Each pass of eight is
// bound by FP32 issue several times over its read of A, so re-reading A per
// pass costs nothing, and the eight-wide kernels issue better than sixteen-
// wide ones (32768^2, k = 16-64: forward 0.93 -> 0.94, adjoint 0.90 -> 0.93
// of the FP32 roofline).  Nine to eleven remaining right-hand sides are split
// in two near halves rather than eight and a one- to three-wide pass that
// would be bound by its read of A.  The FP64 baseline uses powers of two.
// `k` is the number of right-hand sides not yet done.
inline int tile_for(int64_t k)
{
    return k >= 12 ? 8 : (k > 8 ? static_cast<int>((k + 1) / 2) : static_cast<int>(k));
}
inline int f64_tile_for(int64_t k) { return k >= 16 ? 16 : k >= 8 ? 8 : k >= 4 ? 4 : k >= 2 ? 2 : 1; }

// ---------------------------------------------------------------------------
// dX = A^T dY
// ---------------------------------------------------------------------------
// Rows of A each thread of the adjoint loads before using them (the tiles
// are at most eight wide): the fewer terms a row gives, the more rows must
// be in flight to cover the HBM latency.
constexpr int kTRows(int kt) { return kt <= 2 ? 8 : 4; }

// Resident blocks per SM the register allocation must leave room for: with
// this many warps the narrow tiles (bound by FP32 issue, with a row load
// ahead of few terms) hide their load latency; left to itself the compiler
// chose fewer registers and scheduled the row loads later (k = 2-7 at 32768^2:
// 0.83-0.92 of the FP32 roofline without, 0.88-0.93 with).
constexpr int gemv_t_min_blocks(int kt, bool vec)
{
    return vec ? (kt <= 2 ? 5 : (kt <= 3 ? 4 : (kt <= 8 ? 3 : 2))) : (kt <= 8 ? 4 : 3);
}

// Partial sums: ws[(rb * k + c) * n + j] for row block rb.
template <int KT, bool VEC>
__global__ void __launch_bounds__(kGBlock, gemv_t_min_blocks(KT, VEC))
gemv_t_kernel(const float2* __restrict__ A, int64_t m, int64_t n, int64_t lda, const float2* __restrict__ dY,
              int64_t lddy, int64_t rows_per_block, float2* __restrict__ out, int64_t out_ld, int64_t out_rb_stride)
{
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rows_per_block;
    int64_t r1 = r0 + rows_per_block;
    if (r1 > m) r1 = m;
    float2* o = out + static_cast<int64_t>(blockIdx.y) * out_rb_stride;
    if (VEC) {
        const int64_t jp = static_cast<int64_t>(blockIdx.x) * kGBlock + threadIdx.x;  // column pair
        if (2 * jp >= n) return;
        float2 acc0[KT], acc1[KT];
#pragma unroll
        for (int c = 0; c < KT; ++c) {
            acc0[c] = make_float2(0.0f, 0.0f);
            acc1[c] = make_float2(0.0f, 0.0f);
        }
        int64_t r = r0;
        {
            // kTRows(KT) rows loaded ahead of use: a tile of at most eight
            // right-hand sides has too few terms per row to hide the HBM
            // latency of the next row's load (the loops below take the
            // remaining rows)
            constexpr int R = kTRows(KT);
            for (; r + R - 1 < r1; r += R) {
                float4 a[R];
#pragma unroll
                for (int q = 0; q < R; ++q) a[q] = __ldcs(reinterpret_cast<const float4*>(A + (r + q) * lda) + jp);
#pragma unroll
                for (int c = 0; c < KT; ++c) {
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const float2 d = __ldg(dY + c * lddy + r + q);
                        acc0[c] = ffk::add22(acc0[c], ffk::mul22(make_float2(a[q].x, a[q].y), d));
                        acc1[c] = ffk::add22(acc1[c], ffk::mul22(make_float2(a[q].z, a[q].w), d));
                    }
                }
            }
        }
        for (; r + 1 < r1; r += 2) {
            const float4 a0 = __ldcs(reinterpret_cast<const float4*>(A + r * lda) + jp);
            const float4 a1 = __ldcs(reinterpret_cast<const float4*>(A + (r + 1) * lda) + jp);
#pragma unroll
            for (int c = 0; c < KT; ++c) {
                const float2 d0 = __ldg(dY + c * lddy + r);
                const float2 d1 = __ldg(dY + c * lddy + r + 1);
                acc0[c] = ffk::add22(acc0[c], ffk::mul22(make_float2(a0.x, a0.y), d0));
                acc1[c] = ffk::add22(acc1[c], ffk::mul22(make_float2(a0.z, a0.w), d0));
                acc0[c] = ffk::add22(acc0[c], ffk::mul22(make_float2(a1.x, a1.y), d1));
                acc1[c] = ffk::add22(acc1[c], ffk::mul22(make_float2(a1.z, a1.w), d1));
            }
        }
        for (; r < r1; ++r) {
            const float4 a0 = __ldcs(reinterpret_cast<const float4*>(A + r * lda) + jp);
#pragma unroll
            for (int c = 0; c < KT; ++c) {
                const float2 d0 = __ldg(dY + c * lddy + r);
                acc0[c] = ffk::add22(acc0[c], ffk::mul22(make_float2(a0.x, a0.y), d0));
                acc1[c] = ffk::add22(acc1[c], ffk::mul22(make_float2(a0.z, a0.w), d0));
            }
        }
#pragma unroll
        for (int c = 0; c < KT; ++c) {
            o[c * out_ld + 2 * jp] = acc0[c];
            o[c * out_ld + 2 * jp + 1] = acc1[c];
        }
    } else {
        const int64_t j = static_cast<int64_t>(blockIdx.x) * kGBlock + threadIdx.x;
        if (j >= n) return;
        float2 acc[KT];
#pragma unroll
        for (int c = 0; c < KT; ++c) acc[c] = make_float2(0.0f, 0.0f);
        for (int64_t r = r0; r < r1; ++r) {
            const float2 a = A[r * lda + j];
#pragma unroll
            for (int c = 0; c < KT; ++c) acc[c] = ffk::add22(acc[c], ffk::mul22(a, __ldg(dY + c * lddy + r)));
        }
#pragma unroll
        for (int c = 0; c < KT; ++c) o[c * out_ld + j] = acc[c];
    }
}

// dX[c, j] = ws[0][c][j] (+) ws[1][c][j] (+) ... in row-block order.
__global__ void __launch_bounds__(kGBlock)
gemv_t_combine(const float2* __restrict__ ws, int64_t n, int64_t k, int64_t nrb, float2* __restrict__ dX,
               int64_t lddx)
{
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * kGBlock + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t c = idx / n, j = idx - c * n;
    float2 acc = ws[c * n + j];
    for (int64_t rb = 1; rb < nrb; ++rb) acc = ffk::add22(acc, ws[(rb * k + c) * n + j]);
    dX[c * lddx + j] = acc;
}

template <int KT>
void launch_gemv_t_tile(const float2* A, int64_t m, int64_t n, int64_t lda, const float2* dY, int64_t lddy,
                        int64_t rows_per_block, int64_t nrb, float2* out, int64_t out_ld, int64_t out_rb_stride,
                        bool vec, cudaStream_t s)
{
    if (vec) {
        const int64_t pairs = n / 2;
        dim3 grid(static_cast<unsigned>((pairs + kGBlock - 1) / kGBlock), static_cast<unsigned>(nrb));
        gemv_t_kernel<KT, true><<<grid, kGBlock, 0, s>>>(A, m, n, lda, dY, lddy, rows_per_block, out, out_ld,
                                                           out_rb_stride);
    } else {
        dim3 grid(static_cast<unsigned>((n + kGBlock - 1) / kGBlock), static_cast<unsigned>(nrb));
        gemv_t_kernel<KT, false><<<grid, kGBlock, 0, s>>>(A, m, n, lda, dY, lddy, rows_per_block, out, out_ld,
                                                            out_rb_stride);
    }
}

const void* gemv_t_kernel_ptr(int kt, bool vec)
{
    switch (kt) {
    case 8: return vec ? reinterpret_cast<const void*>(&gemv_t_kernel<8, true>)
                       : reinterpret_cast<const void*>(&gemv_t_kernel<8, false>);
    case 7: return vec ? reinterpret_cast<const void*>(&gemv_t_kernel<7, true>)
                       : reinterpret_cast<const void*>(&gemv_t_kernel<7, false>);
    case 6: return vec ? reinterpret_cast<const void*>(&gemv_t_kernel<6, true>)
                       : reinterpret_cast<const void*>(&gemv_t_kernel<6, false>);
    case 5: return vec ? reinterpret_cast<const void*>(&gemv_t_kernel<5, true>)
                       : reinterpret_cast<const void*>(&gemv_t_kernel<5, false>);
    case 4: return vec ? reinterpret_cast<const void*>(&gemv_t_kernel<4, true>)
                       : reinterpret_cast<const void*>(&gemv_t_kernel<4, false>);
    case 3: return vec ? reinterpret_cast<const void*>(&gemv_t_kernel<3, true>)
                       : reinterpret_cast<const void*>(&gemv_t_kernel<3, false>);
    case 2: return vec ? reinterpret_cast<const void*>(&gemv_t_kernel<2, true>)
                       : reinterpret_cast<const void*>(&gemv_t_kernel<2, false>);
    default: return vec ? reinterpret_cast<const void*>(&gemv_t_kernel<1, true>)
                        : reinterpret_cast<const void*>(&gemv_t_kernel<1, false>);
    }
}

// Number of row blocks for the adjoint.  The grid is col_blocks x nrb blocks;
// nrb is chosen so that the grid fills whole waves of resident blocks (SMs x
// blocks per SM of the widest tile's kernel): the adjoint is FP32-issue
// bound for k > 2, and a last, partly filled wave would idle most SMs.
// Every row block keeps at least 32 rows; at most 64 row blocks.
int64_t row_blocks(int64_t m, int64_t n, int64_t k, bool vec, int sm_count)
{
    const int64_t cols = vec ? n / 2 : n;
    const int64_t col_blocks = (cols + kGBlock - 1) / kGBlock;
    if (col_blocks < 1 || m < 64) return 1;
    const int occ = ffh::occupancy(gemv_t_kernel_ptr(tile_for(k), vec), kGBlock);
    const int64_t resident = static_cast<int64_t>(sm_count) * (occ > 0 ? occ : 1);
    int64_t maxrb = m / 32;
    if (maxrb > 64) maxrb = 64;
    if (maxrb < 1) maxrb = 1;
    int64_t best = 1;
    double best_eff = -1.0;
    for (int64_t nrb = 1; nrb <= maxrb; ++nrb) {
        const int64_t blocks = nrb * col_blocks;
        const int64_t waves = (blocks + resident - 1) / resident;
        double eff = static_cast<double>(blocks) / static_cast<double>(waves * resident);
        if (blocks < resident) eff *= 0.999;  // prefer at least one full wave when possible
        if (eff > best_eff + 1e-3) {
            best_eff = eff;
            best = nrb;
        }
    }
    return best;
}

// ---------------------------------------------------------------------------
// dA = dY X^T.  Every element accumulates its k terms Mul22(dY[r, c], X[j, c])
// in order c = 0 .. k-1 from (0, 0), so the result is the oracle's
// left-to-right sum bit for bit.  With 16-byte access along the rows of dA,
// k <= 21 runs here in one or two passes (gemv_dA_small_kernel); without it,
// k <= 12 runs here with one thread per column (gemv_dA_scalar_kernel).
// Larger k runs as the matrix product op(dY) X on the GEMM kernel (the same
// terms in the same order).  Both kernels walk the rows with a grid of about
// one wave of blocks.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGBlock)
gemv_dA_scalar_kernel(const float2* __restrict__ dY, int64_t m, int64_t lddy, const float2* __restrict__ X,
                      int64_t n, int64_t ldx, int64_t k, float2* __restrict__ dA, int64_t ldda)
{
    const int64_t j = static_cast<int64_t>(blockIdx.x) * kGBlock + threadIdx.x;
    if (j >= n) return;
    for (int64_t r = blockIdx.y; r < m; r += gridDim.y) {
        float2 acc = make_float2(0.0f, 0.0f);
        for (int64_t c = 0; c < k; ++c) acc = ffk::add22(acc, ffk::mul22(__ldg(dY + c * lddy + r), X[c * ldx + j]));
        dA[r * ldda + j] = acc;
    }
}

// Rows per shared-memory chunk of dY in the weight-gradient kernel (even).
constexpr int kTChunk = 128;

// dA for up to 12 right-hand sides with 16-byte access along the rows of dA: one thread per
// pair of adjacent columns, the thread's k column-pair values of X in
// registers.  Block row y takes the rows [y rpb, (y + 1) rpb) (rpb even) in
// pairs, so a thread forms 4 elements per step; the block stages the dY
// values of kTChunk rows at a time in shared memory, where one 16-byte read
// gives both rows of a pair for one right-hand side.  Every element is
// Add22((0, 0), term_0), then Add22 of terms 1 .. k-1, in order (the first
// step through add22_from_zero, bit-identical).  With ACC the elements
// continue from the values dA holds (the partial sums of the right-hand
// sides before these k: the second pass for 12 < k <= 21), adding terms
// 0 .. k-1 in order.  Lanes past the last column pair work on the last pair
// and do not store, so that every lane of a warp takes part in the vote and
// every thread reaches the block barriers.
//
// Resident blocks per SM the register allocation must leave room for: a
// continuing pass of ten or more right-hand sides took 98-100 registers on
// its own (two blocks per SM) and ran at 0.82-0.83 of the FP32 roofline
// (32768^2, k = 18-20 as 8 + 10 .. 8 + 12); at 80 registers (three blocks)
// k = 20 as 10 + 10 runs at 0.92.
constexpr int dA_min_blocks(int kt, bool acc) { return acc && kt >= 10 ? 3 : 0; }

template <int KT, bool ACC>
__global__ void __launch_bounds__(kGBlock, dA_min_blocks(KT, ACC))
gemv_dA_small_kernel(const float2* __restrict__ dY, int64_t m, int64_t lddy, const float2* __restrict__ X, int64_t n,
                     int64_t ldx, float2* __restrict__ dA, int64_t ldda, int64_t rpb)
{
    __shared__ float4 sdy[KT][kTChunk / 2];
    const int64_t npairs = n >> 1;
    const int64_t jp_raw = static_cast<int64_t>(blockIdx.x) * kGBlock + threadIdx.x;
    if (static_cast<int64_t>(blockIdx.x) * kGBlock >= npairs) return;  // whole block past the end
    const bool store = jp_raw < npairs;
    const int64_t jp = store ? jp_raw : npairs - 1;
    float2 xl[KT], xh[KT];
#pragma unroll
    for (int c = 0; c < KT; ++c) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(X + c * ldx) + jp);
        xl[c] = make_float2(v.x, v.y);
        xh[c] = make_float2(v.z, v.w);
    }
    constexpr int C0 = ACC ? 0 : 1;   // first term added by the loop below
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    const int64_t rp = r0 + ((r1 > r0 ? r1 - r0 : 0) & ~static_cast<int64_t>(1));   // end of the row pairs
    for (int64_t cb = r0; cb < rp; cb += kTChunk) {
        const int rows = static_cast<int>(rp - cb < kTChunk ? rp - cb : kTChunk);
        __syncthreads();   // the previous chunk's reads are done
        for (int i = threadIdx.x; i < KT * kTChunk; i += kGBlock) {
            const int c = i / kTChunk, q = i - c * kTChunk;
            if (q < rows) reinterpret_cast<float2*>(sdy[c])[q] = __ldg(dY + c * lddy + cb + q);
        }
        __syncthreads();
        float4* row = reinterpret_cast<float4*>(dA + cb * ldda) + jp;
        const int64_t ldda4 = ldda >> 1;
        float4 n0, n1;   // ACC: the stored sums of the next row pair, loaded one pair ahead
        if constexpr (ACC) {
            n0 = __ldcs(row);
            n1 = __ldcs(row + ldda4);
        }
        for (int lp = 0; lp < rows / 2; ++lp, row += 2 * ldda4) {
            float2 a00, a01, a10, a11;
            if constexpr (ACC) {
                const float4 p0 = n0, p1 = n1;
                if (lp + 1 < rows / 2) {
                    n0 = __ldcs(row + 2 * ldda4);
                    n1 = __ldcs(row + 3 * ldda4);
                }
                a00 = make_float2(p0.x, p0.y);
                a01 = make_float2(p0.z, p0.w);
                a10 = make_float2(p1.x, p1.y);
                a11 = make_float2(p1.z, p1.w);
            } else {
                const float4 d01 = sdy[0][lp];
                const float2 t00 = ffk::mul22(make_float2(d01.x, d01.y), xl[0]);
                const float2 t01 = ffk::mul22(make_float2(d01.x, d01.y), xh[0]);
                const float2 t10 = ffk::mul22(make_float2(d01.z, d01.w), xl[0]);
                const float2 t11 = ffk::mul22(make_float2(d01.z, d01.w), xh[0]);
                const bool fast = __all_sync(0xffffffffu, ffk::from_zero_fast(t00) && ffk::from_zero_fast(t01) &&
                                                              ffk::from_zero_fast(t10) &&
                                                              ffk::from_zero_fast(t11));
                a00 = ffk::add22_from_zero(t00, fast);
                a01 = ffk::add22_from_zero(t01, fast);
                a10 = ffk::add22_from_zero(t10, fast);
                a11 = ffk::add22_from_zero(t11, fast);
            }
#pragma unroll
            for (int c = C0; c < KT; ++c) {
                const float4 d01 = sdy[c][lp];
                const float2 d0 = make_float2(d01.x, d01.y), d1 = make_float2(d01.z, d01.w);
                a00 = ffk::add22(a00, ffk::mul22(d0, xl[c]));
                a01 = ffk::add22(a01, ffk::mul22(d0, xh[c]));
                a10 = ffk::add22(a10, ffk::mul22(d1, xl[c]));
                a11 = ffk::add22(a11, ffk::mul22(d1, xh[c]));
            }
            if (store) {
                __stcs(row, make_float4(a00.x, a00.y, a01.x, a01.y));
                __stcs(row + ldda4, make_float4(a10.x, a10.y, a11.x, a11.y));
            }
        }
    }
    if (rp < r1) {  // the last row of an odd m
        const int64_t r = rp;
        float4* row = reinterpret_cast<float4*>(dA + r * ldda) + jp;
        float2 a0, a1;
        if constexpr (ACC) {
            const float4 p = __ldcs(row);
            a0 = make_float2(p.x, p.y);
            a1 = make_float2(p.z, p.w);
        } else {
            const float2 d = __ldg(dY + r);
            const float2 t0 = ffk::mul22(d, xl[0]), t1 = ffk::mul22(d, xh[0]);
            const bool fast = __all_sync(0xffffffffu, ffk::from_zero_fast(t0) && ffk::from_zero_fast(t1));
            a0 = ffk::add22_from_zero(t0, fast);
            a1 = ffk::add22_from_zero(t1, fast);
        }
#pragma unroll
        for (int c = C0; c < KT; ++c) {
            const float2 dc = __ldg(dY + c * lddy + r);
            a0 = ffk::add22(a0, ffk::mul22(dc, xl[c]));
            a1 = ffk::add22(a1, ffk::mul22(dc, xh[c]));
        }
        if (store) __stcs(row, make_float4(a0.x, a0.y, a1.x, a1.y));
    }
}

// Widest k that ff_gemv_dA runs on gemv_dA_small_kernel: one pass up to 12
// right-hand sides (32768^2, k = 9-12: 0.93-0.95 of the FP32 roofline in one
// pass against 0.87-0.89 in two), then two passes of ceil(k/2) and floor(k/2),
// the second continuing from the stored sums (loaded one row pair ahead), up
// to 21; the GEMM kernel takes larger k.  32768^2, fractions of the FP32
// roofline, two passes against the GEMM route: k = 13-21 0.90-0.92 against
// 0.87-0.90; k = 22-23 0.89-0.90 against 0.90; k = 24 (12 + 12, where the
// continuing pass spills at 80 registers) 0.85 against 0.91.
constexpr int kDAPass = 12;
constexpr int kDAMaxSmallK = 21;
// The continuing pass is the second of two and takes floor(k/2) <= 10
// right-hand sides: no wider continuing kernel is compiled (dA_kt maps the
// cases above ten of the switches below to it; the pass loop never takes
// them).
constexpr int kDAMaxAccKT = kDAMaxSmallK / 2;
constexpr int dA_kt(int kt, bool acc) { return acc && kt > kDAMaxAccKT ? kDAMaxAccKT : kt; }
static_assert((kDAMaxSmallK + 1) / 2 <= kDAPass && kDAMaxSmallK <= 2 * kDAPass,
              "beyond one pass, ff_gemv_dA runs exactly two passes of at most kDAPass right-hand sides");

template <bool ACC>
const void* dA_small_ptr(int k)
{
    switch (k) {
    case 1: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<1, ACC>);
    case 2: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<2, ACC>);
    case 3: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<3, ACC>);
    case 4: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<4, ACC>);
    case 5: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<5, ACC>);
    case 6: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<6, ACC>);
    case 7: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<7, ACC>);
    case 8: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<8, ACC>);
    case 9: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<9, ACC>);
    case 10: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<10, ACC>);
    case 11: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<dA_kt(11, ACC), ACC>);
    default: return reinterpret_cast<const void*>(&gemv_dA_small_kernel<dA_kt(12, ACC), ACC>);
    }
}

template <bool ACC>
void launch_dA_small(int k, dim3 grid, cudaStream_t s, const float2* dY, int64_t m, int64_t lddy, const float2* X,
                     int64_t n, int64_t ldx, float2* dA, int64_t ldda, int64_t rpb)
{
    switch (k) {
    case 1: gemv_dA_small_kernel<1, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 2: gemv_dA_small_kernel<2, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 3: gemv_dA_small_kernel<3, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 4: gemv_dA_small_kernel<4, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 5: gemv_dA_small_kernel<5, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 6: gemv_dA_small_kernel<6, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 7: gemv_dA_small_kernel<7, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 8: gemv_dA_small_kernel<8, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 9: gemv_dA_small_kernel<9, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 10: gemv_dA_small_kernel<10, ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb); break;
    case 11:
        gemv_dA_small_kernel<dA_kt(11, ACC), ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb);
        break;
    default:
        gemv_dA_small_kernel<dA_kt(12, ACC), ACC><<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, dA, ldda, rpb);
        break;
    }
}

// Grid of one wave of resident blocks of `kern` (rounded down so that every
// block is resident at once), block rows of an even number of rows.
void dA_small_grid(const void* kern, int64_t m, int64_t n, int sm_count, dim3* grid, int64_t* rpb)
{
    const int64_t col_blocks = (n / 2 + kGBlock - 1) / kGBlock;
    const int occ = ffh::occupancy(kern, kGBlock);
    int64_t gy = static_cast<int64_t>(sm_count) * (occ > 0 ? occ : 1) / col_blocks;
    if (gy > (m + 1) / 2) gy = (m + 1) / 2;
    if (gy > 65535) gy = 65535;
    if (gy < 1) gy = 1;
    int64_t r = (m + gy - 1) / gy;
    r += r & 1;
    *rpb = r;
    *grid = dim3(static_cast<unsigned>(col_blocks), static_cast<unsigned>((m + r - 1) / r));
}

// ---------------------------------------------------------------------------
// binary64 GEMV (one warp per row, fma accumulation, shuffle tree)
// ---------------------------------------------------------------------------
template <int KT>
__global__ void __launch_bounds__(kGBlock)
gemv_f64_kernel(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda, const double* __restrict__ X,
                int64_t ldx, double* __restrict__ Y, int64_t ldy)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * kGWarps + (threadIdx.x >> 5);
    if (r >= m) return;
    double acc[KT];
#pragma unroll
    for (int c = 0; c < KT; ++c) acc[c] = 0.0;
    const double* Ar = A + r * lda;
    for (int64_t j = lane; j < n; j += 32) {
        const double a = __ldcs(Ar + j);
#pragma unroll
        for (int c = 0; c < KT; ++c) acc[c] = __fma_rn(a, __ldg(X + c * ldx + j), acc[c]);
    }
#pragma unroll
    for (int c = 0; c < KT; ++c) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[c] = __dadd_rn(acc[c], __shfl_down_sync(0xffffffffu, acc[c], off));
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < KT; ++c) Y[c * ldy + r] = acc[c];
    }
}

bool bad_dims(int64_t m, int64_t n, int64_t k) { return m < 0 || n < 0 || k < 1 || k > kMaxK; }

size_t gemv_t_ws(int64_t m, int64_t n, int64_t k, bool vec, int sm_count)
{
    const int64_t nrb = row_blocks(m, n, k, vec, sm_count);
    if (nrb <= 1) return 16;
    return static_cast<size_t>(nrb) * static_cast<size_t>(n) * static_cast<size_t>(k) * sizeof(float2);
}

}  // namespace

extern "C" {

ff_status ff_gemv(const ff2* A_, int64_t m, int64_t n, int64_t lda, const ff2* X_, int64_t ldx, int64_t k,
                  ff2* Y_, int64_t ldy, cudaStream_t s)
{
    if (bad_dims(m, n, k) || lda < n || ldx < n || ldy < m) return FF_ERR_INVALID_ARG;
    const size_t an = static_cast<size_t>(m) * static_cast<size_t>(n);
    if (!ffh::ok_ptr(A_, an) || !ffh::ok_ptr(X_, static_cast<size_t>(n)) || !ffh::ok_ptr(Y_, static_cast<size_t>(m)))
        return FF_ERR_INVALID_ARG;
    if (m == 0) return FF_OK;
    auto* A = reinterpret_cast<const float2*>(A_);
    auto* X = reinterpret_cast<const float2*>(X_);
    auto* Y = reinterpret_cast<float2*>(Y_);
    const bool vec = (n % 2 == 0) && (lda % 2 == 0) && (ldx % 2 == 0) && ffh::aligned(A, 16) && ffh::aligned(X, 16);
    for (int64_t c0 = 0; c0 < k;) {
        const int kt = tile_for(k - c0);
        ff_status st;
        const float2* Xc = X + c0 * ldx;
        float2* Yc = Y + c0 * ldy;
        switch (kt) {
        case 8: st = launch_gemv_tile<8>(A, m, n, lda, Xc, ldx, Yc, ldy, vec, s); break;
        case 7: st = launch_gemv_tile<7>(A, m, n, lda, Xc, ldx, Yc, ldy, vec, s); break;
        case 6: st = launch_gemv_tile<6>(A, m, n, lda, Xc, ldx, Yc, ldy, vec, s); break;
        case 5: st = launch_gemv_tile<5>(A, m, n, lda, Xc, ldx, Yc, ldy, vec, s); break;
        case 4: st = launch_gemv_tile<4>(A, m, n, lda, Xc, ldx, Yc, ldy, vec, s); break;
        case 3: st = launch_gemv_tile<3>(A, m, n, lda, Xc, ldx, Yc, ldy, vec, s); break;
        case 2: st = launch_gemv_tile<2>(A, m, n, lda, Xc, ldx, Yc, ldy, vec, s); break;
        default: st = launch_gemv_tile<1>(A, m, n, lda, Xc, ldx, Yc, ldy, vec, s); break;
        }
        if (st != FF_OK) return st;
        c0 += kt;
    }
    return FF_OK;
}

size_t ff_gemv_t_workspace_bytes(int64_t m, int64_t n, int64_t k)
{
    if (bad_dims(m, n, k)) return 0;
    ffh::DeviceInfo di;
    if (ffh::device_info(&di) != FF_OK) return 0;
    // the workspace must cover either access path: take the larger
    const size_t a = gemv_t_ws(m, n, k, true, di.sm_count);
    const size_t b = gemv_t_ws(m, n, k, false, di.sm_count);
    return a > b ? a : b;
}

ff_status ff_gemv_t_launch_shape(const ff2* A, int64_t m, int64_t n, int64_t lda, int64_t k, int64_t* nrb,
                                 int* vector)
{
    if (bad_dims(m, n, k) || lda < n || nrb == nullptr || vector == nullptr) return FF_ERR_INVALID_ARG;
    ffh::DeviceInfo di;
    const ff_status st = ffh::device_info(&di);
    if (st != FF_OK) return st;
    const bool vec = (n % 2 == 0) && (lda % 2 == 0) && ffh::aligned(A, 16);
    *nrb = row_blocks(m, n, k, vec, di.sm_count);
    *vector = vec ? 1 : 0;
    return FF_OK;
}

ff_status ff_gemv_t(const ff2* A_, int64_t m, int64_t n, int64_t lda, const ff2* dY_, int64_t lddy, int64_t k,
                    ff2* dX_, int64_t lddx, void* ws, size_t ws_bytes, cudaStream_t s)
{
    if (bad_dims(m, n, k) || lda < n || lddy < m || lddx < n) return FF_ERR_INVALID_ARG;
    const size_t an = static_cast<size_t>(m) * static_cast<size_t>(n);
    if (!ffh::ok_ptr(A_, an) || !ffh::ok_ptr(dY_, static_cast<size_t>(m)) || !ffh::ok_ptr(dX_, static_cast<size_t>(n)))
        return FF_ERR_INVALID_ARG;
    if (n == 0) return FF_OK;
    ffh::DeviceInfo di;
    ff_status st = ffh::device_info(&di);
    if (st != FF_OK) return st;
    auto* A = reinterpret_cast<const float2*>(A_);
    auto* dY = reinterpret_cast<const float2*>(dY_);
    auto* dX = reinterpret_cast<float2*>(dX_);
    const bool vec = (n % 2 == 0) && (lda % 2 == 0) && ffh::aligned(A, 16);
    const int64_t nrb = row_blocks(m, n, k, vec, di.sm_count);
    const int64_t rpb = m > 0 ? (m + nrb - 1) / nrb : 0;
    float2* part = nullptr;
    if (nrb > 1) {
        if (ws == nullptr || ws_bytes < gemv_t_ws(m, n, k, vec, di.sm_count) || !ffh::aligned(ws, 16))
            return FF_ERR_WORKSPACE;
        part = static_cast<float2*>(ws);
    }
    for (int64_t c0 = 0; c0 < k;) {
        const int kt = tile_for(k - c0);
        const float2* dYc = dY + c0 * lddy;
        // one row block: write dX directly; else partials [rb][c][j]
        float2* out = nrb > 1 ? part + c0 * n : dX + c0 * lddx;
        const int64_t out_ld = nrb > 1 ? n : lddx;
        const int64_t rb_stride = nrb > 1 ? k * n : 0;
        const int64_t mm = m > 0 ? m : 0;
        switch (kt) {
        case 8: launch_gemv_t_tile<8>(A, mm, n, lda, dYc, lddy, rpb, nrb, out, out_ld, rb_stride, vec, s); break;
        case 7: launch_gemv_t_tile<7>(A, mm, n, lda, dYc, lddy, rpb, nrb, out, out_ld, rb_stride, vec, s); break;
        case 6: launch_gemv_t_tile<6>(A, mm, n, lda, dYc, lddy, rpb, nrb, out, out_ld, rb_stride, vec, s); break;
        case 5: launch_gemv_t_tile<5>(A, mm, n, lda, dYc, lddy, rpb, nrb, out, out_ld, rb_stride, vec, s); break;
        case 4: launch_gemv_t_tile<4>(A, mm, n, lda, dYc, lddy, rpb, nrb, out, out_ld, rb_stride, vec, s); break;
        case 3: launch_gemv_t_tile<3>(A, mm, n, lda, dYc, lddy, rpb, nrb, out, out_ld, rb_stride, vec, s); break;
        case 2: launch_gemv_t_tile<2>(A, mm, n, lda, dYc, lddy, rpb, nrb, out, out_ld, rb_stride, vec, s); break;
        default: launch_gemv_t_tile<1>(A, mm, n, lda, dYc, lddy, rpb, nrb, out, out_ld, rb_stride, vec, s); break;
        }
        st = ffh::check_launch();
        if (st != FF_OK) return st;
        c0 += kt;
    }
    if (nrb > 1) {
        const int64_t total = n * k;
        gemv_t_combine<<<static_cast<unsigned>((total + kGBlock - 1) / kGBlock), kGBlock, 0, s>>>(part, n, k, nrb, dX,
                                                                                                  lddx);
        st = ffh::check_launch();
        if (st != FF_OK) return st;
    }
    return FF_OK;
}

ff_status ff_gemv_dA(const ff2* dY_, int64_t m, int64_t lddy, const ff2* X_, int64_t n, int64_t ldx, int64_t k,
                     ff2* dA_, int64_t ldda, cudaStream_t s)
{
    if (bad_dims(m, n, k) || lddy < m || ldx < n || ldda < n) return FF_ERR_INVALID_ARG;
    const size_t an = static_cast<size_t>(m) * static_cast<size_t>(n);
    if (!ffh::ok_ptr(dY_, static_cast<size_t>(m)) || !ffh::ok_ptr(X_, static_cast<size_t>(n)) || !ffh::ok_ptr(dA_, an))
        return FF_ERR_INVALID_ARG;
    if (m == 0 || n == 0) return FF_OK;
    // beyond kDAMaxSmallK right-hand sides, dA is a matrix product op(dY) X
    // with dY read transposed in place: the GEMM kernel computes every
    // element with the same Mul22(dY[r, c], X[j, c]) terms in the same order
    // (bit-identical) at its higher arithmetic rate
    if (k > kDAMaxSmallK) return ff_gemm(1, 0, m, n, k, dY_, lddy, X_, ldx, dA_, ldda, s);
    auto* dY = reinterpret_cast<const float2*>(dY_);
    auto* X = reinterpret_cast<const float2*>(X_);
    auto* dA = reinterpret_cast<float2*>(dA_);
    const bool vec = (n % 2 == 0) && (ldx % 2 == 0) && (ldda % 2 == 0) && ffh::aligned(X, 16) && ffh::aligned(dA, 16);
    if (!vec && k > kDAPass) return ff_gemm(1, 0, m, n, k, dY_, lddy, X_, ldx, dA_, ldda, s);
    ffh::DeviceInfo di;
    const ff_status st = ffh::device_info(&di);
    if (st != FF_OK) return st;
    if (vec) {
        // up to kDAPass right-hand sides in one pass from (0, 0); more in
        // two passes of ceil(k/2) and floor(k/2), the second continuing from
        // the sums the first stored: a narrow pass is bound by re-reading dA
        // (32768^2: k = 9 as 8 + 1 measured 0.78 of the roofline, as 5 + 4
        // 0.86; k = 13 as 12 + 1 0.81, as 7 + 6 0.92)
        for (int64_t c0 = 0; c0 < k;) {
            const int64_t rest = k - c0;
            const int kt = static_cast<int>(rest <= kDAPass ? rest : (rest + 1) / 2);
            dim3 grid;
            int64_t rpb;
            if (c0 == 0) {
                dA_small_grid(dA_small_ptr<false>(kt), m, n, di.sm_count, &grid, &rpb);
                launch_dA_small<false>(kt, grid, s, dY, m, lddy, X, n, ldx, dA, ldda, rpb);
            } else {
                dA_small_grid(dA_small_ptr<true>(kt), m, n, di.sm_count, &grid, &rpb);
                launch_dA_small<true>(kt, grid, s, dY + c0 * lddy, m, lddy, X + c0 * ldx, n, ldx, dA, ldda, rpb);
            }
            const ff_status stp = ffh::check_launch();
            if (stp != FF_OK) return stp;
            c0 += kt;
        }
        return FF_OK;
    }
    const int64_t col_blocks = (n + kGBlock - 1) / kGBlock;
    const int occ = ffh::occupancy(reinterpret_cast<const void*>(&gemv_dA_scalar_kernel), kGBlock);
    int64_t gy64 = static_cast<int64_t>(di.sm_count) * (occ > 0 ? occ : 1) / col_blocks;
    if (gy64 > m) gy64 = m;
    if (gy64 > 65535) gy64 = 65535;
    if (gy64 < 1) gy64 = 1;
    dim3 grid(static_cast<unsigned>(col_blocks), static_cast<unsigned>(gy64));
    gemv_dA_scalar_kernel<<<grid, kGBlock, 0, s>>>(dY, m, lddy, X, n, ldx, k, dA, ldda);
    return ffh::check_launch();
}

ff_status ff_f64_gemv(const double* A, int64_t m, int64_t n, int64_t lda, const double* X, int64_t ldx, int64_t k,
                      double* Y, int64_t ldy, cudaStream_t s)
{
    if (bad_dims(m, n, k) || lda < n || ldx < n || ldy < m) return FF_ERR_INVALID_ARG;
    const size_t an = static_cast<size_t>(m) * static_cast<size_t>(n);
    if (!ffh::ok_ptr(A, an) || !ffh::ok_ptr(X, static_cast<size_t>(n)) || !ffh::ok_ptr(Y, static_cast<size_t>(m)))
        return FF_ERR_INVALID_ARG;
    if (m == 0) return FF_OK;
    const unsigned grid = static_cast<unsigned>((m + kGWarps - 1) / kGWarps);
    for (int64_t c0 = 0; c0 < k;) {
        const int kt = f64_tile_for(k - c0);
        const double* Xc = X + c0 * ldx;
        double* Yc = Y + c0 * ldy;
        switch (kt) {
        case 16: gemv_f64_kernel<16><<<grid, kGBlock, 0, s>>>(A, m, n, lda, Xc, ldx, Yc, ldy); break;
        case 8: gemv_f64_kernel<8><<<grid, kGBlock, 0, s>>>(A, m, n, lda, Xc, ldx, Yc, ldy); break;
        case 4: gemv_f64_kernel<4><<<grid, kGBlock, 0, s>>>(A, m, n, lda, Xc, ldx, Yc, ldy); break;
        case 2: gemv_f64_kernel<2><<<grid, kGBlock, 0, s>>>(A, m, n, lda, Xc, ldx, Yc, ldy); break;
        default: gemv_f64_kernel<1><<<grid, kGBlock, 0, s>>>(A, m, n, lda, Xc, ldx, Yc, ldy); break;
        }
        ff_status st = ffh::check_launch();
        if (st != FF_OK) return st;
        c0 += kt;
    }
    return FF_OK;
}

}  // extern "C"
