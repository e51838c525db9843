// ff_batch.cu -- many independent float-float dot and AXPY instances of
// uneven lengths in one persistent launch, a CUDA-graph wrapper around it,
// and the autotuner that picks its block size, values per thread and
// resident blocks per SM.
//
// Plan (host, once): every instance is cut into tiles of block x ppt values;
// the tiles of all instances form one list, instance after instance.  The
// plan copies the instance records and the tile list to device memory it
// owns.
//
// Run: a persistent grid of (SMs x blocks per SM) blocks walks the tile list
// round robin (block b takes tiles b, b + G, b + 2G, ...).
//   AXPY tile: z_i = Add22(Mul22(alpha, x_i), y_i) for the tile's values.
//   dot-gradient tile: dx_i = Mul22(dout, y_i), dy_i = Mul22(dout, x_i).
//   GEMV rows tile (rows of length <= 65536): eight lanes reduce one row,
//   so a warp works on four rows at a time, R groups of four rows per warp
//   per tile (R chosen at plan time so that a tile holds about 16K values);
//   the exact lane and chunk order is given at gemv_rows_tile_body.  Longer
//   GEMV rows become dot records (row r of the matrix with the vector).
//   Access: 16-byte vectors of two values when all of a record's arrays
//   start on a 16-byte boundary; when they all start 8 bytes past one,
//   thread 0 takes each tile's first value on its own and the rest of the
//   tile runs on 16-byte vectors; otherwise 8-byte loads.
//   dot tile:  each thread accumulates its values left to right with
//              Add22(acc, Mul22(x_i, y_i)) (thread 0 the tile's first value
//              first when it is taken on its own, and an odd last value
//              last); the block combines threads with
//              the shuffle-down Add22 tree of ff_dot and stores the tile's
//              partial; the tile that finishes its instance last (atomic
//              counter per instance) adds the instance's tile partials in
//              tile order and writes the result.
// No block waits for another; the per-instance counters are zeroed by a
// memset at the start of every run (and left zero by the last tile).
//
// Plans made only of GEMV rows run a kernel of their own: their tiles differ
// in cost (a tile holds 4 x warps x R rows, and R cannot drop below one for
// rows longer than 16K / (4 x warps) values), so the plan sorts the tiles by
// cost, largest first, and the blocks take the next tile from an atomic
// counter (zeroed by the same memset) instead of round robin.  Each such
// tile writes whole rows, so the order changes no result.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ff_core.cuh"
#include "ff_host.cuh"

// Internal record kind: rows of a GEMV instance, eight lanes per row.
constexpr int32_t kGemvRows = 100;
// GEMV rows up to this length are reduced by eight lanes each; longer rows
// become dot records reduced by whole blocks over several tiles.
constexpr int64_t kWarpRowMax = 65536;

struct DevInst {
    const float2* x;
    const float2* y;
    float2* out;
    float2* out2;
    const float2* dout;
    float2 alpha;
    int64_t lda;   // GEMV rows: row stride of x
    int64_t m;     // GEMV rows: number of rows
    int64_t n;
    int64_t first_tile;
    int32_t ntiles;
    int32_t kind;
    int32_t vec;   // 1: 16-byte access; 2: one value, then 16-byte access; 0: 8-byte access
    int32_t rows_per_warp;  // GEMV rows: rows each warp reduces per tile
};

struct Tile {
    int32_t inst;
    int32_t pad;
    int64_t start;
};

struct ff_batch_plan {
    int count;
    bool has_gemv_rows;
    bool only_gemv_rows;
    ff_tune tune;
    int64_t ntiles;
    int64_t ndot;
    int64_t total_values;
    int device;
    unsigned grid;
    DevInst* d_inst;
    Tile* d_tiles;
};

struct ff_batch_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

constexpr size_t kCountersAlign = 256;

__device__ __forceinline__ float2 shfl_down2(float2 v, int off)
{
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, off), __shfl_down_sync(0xffffffffu, v.y, off));
}

template <int BLOCK>
__device__ __forceinline__ float2 block_reduce(float2 v, float2* sm)
{
    constexpr int W = BLOCK / 32;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = ffk::add22(v, shfl_down2(v, off));
    if (lane == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (lane < W) ? sm[lane] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int off = W / 2; off > 0; off >>= 1) v = ffk::add22(v, shfl_down2(v, off));
    }
    __syncthreads();
    return v;
}

// One tile of GEMV rows (see the header comment).  Eight lanes reduce one
// row, so a warp works on four rows at once: lane group g (lanes 8g .. 8g+7)
// of warp w takes rows start + 4 (w R + k) + g for k = 0 .. R-1, lane l of
// the group accumulates the row's two-value chunks l + 16i into its first
// and l + 8 + 16i into its second accumulator (a leftover chunk into the
// first), adds them, the group combines its eight lanes with a shuffle-down
// Add22 tree (offsets 4, 2, 1) and its lane 0 writes out[r].  Kept out of
// line (for the mixed kernel), with its arguments by value.
__device__ __forceinline__ void gemv_rows_tile_body(const float2* A, const float2* xv, float2* out, int64_t n,
                                                   int64_t lda, int64_t m, int vec, int rpw, int64_t start)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 3;
    const int l8 = lane & 7;
    const int64_t w = threadIdx.x >> 5;
    for (int k = 0; k < rpw; ++k) {
        const int64_t r0 = start + 4 * (w * rpw + k);
        if (r0 >= m) break;  // warp-uniform
        const int64_t r = r0 + g;
        float2 acc = make_float2(0.0f, 0.0f);
        if (r < m) {
            const float2* Ar = A + r * lda;
            if (vec) {
                const float4* A4 = reinterpret_cast<const float4*>(Ar);
                const float4* x4 = reinterpret_cast<const float4*>(xv);
                const int64_t nch = n >> 1;
                float2 acc1 = make_float2(0.0f, 0.0f);
                int64_t c = l8;
                for (; c + 8 < nch; c += 16) {
                    const float4 a0 = __ldcs(A4 + c), a1 = __ldcs(A4 + c + 8);
                    const float4 x0 = __ldg(x4 + c), x1 = __ldg(x4 + c + 8);
                    acc = ffk::add22(acc, ffk::mul22(make_float2(a0.x, a0.y), make_float2(x0.x, x0.y)));
                    acc = ffk::add22(acc, ffk::mul22(make_float2(a0.z, a0.w), make_float2(x0.z, x0.w)));
                    acc1 = ffk::add22(acc1, ffk::mul22(make_float2(a1.x, a1.y), make_float2(x1.x, x1.y)));
                    acc1 = ffk::add22(acc1, ffk::mul22(make_float2(a1.z, a1.w), make_float2(x1.z, x1.w)));
                }
                for (; c < nch; c += 8) {
                    const float4 a0 = __ldcs(A4 + c);
                    const float4 x0 = __ldg(x4 + c);
                    acc = ffk::add22(acc, ffk::mul22(make_float2(a0.x, a0.y), make_float2(x0.x, x0.y)));
                    acc = ffk::add22(acc, ffk::mul22(make_float2(a0.z, a0.w), make_float2(x0.z, x0.w)));
                }
                acc = ffk::add22(acc, acc1);
                if ((n & 1) && l8 == 0) acc = ffk::add22(acc, ffk::mul22(Ar[n - 1], xv[n - 1]));
            } else {
                for (int64_t j = l8; j < n; j += 8) acc = ffk::add22(acc, ffk::mul22(Ar[j], xv[j]));
            }
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1)
            acc = ffk::add22(acc, make_float2(__shfl_down_sync(0xffffffffu, acc.x, off, 8),
                                              __shfl_down_sync(0xffffffffu, acc.y, off, 8)));
        if (l8 == 0 && r < m) out[r] = acc;
    }
}

__device__ __noinline__ void gemv_rows_tile(const float2* A, const float2* xv, float2* out, int64_t n,
                                            int64_t lda, int64_t m, int vec, int rpw, int64_t start)
{
    gemv_rows_tile_body(A, xv, out, n, lda, m, vec, rpw, start);
}

// PPT values per thread per tile (even).  Values of a tile are visited as
// two-value chunks c = threadIdx.x + j * BLOCK, j = 0 .. PPT/2 - 1, UN
// chunks per input loaded before they are used (UN = 4 keeps more bytes in
// flight per thread, UN = 2 needs fewer registers and so fits more warps).
template <int BLOCK, int PPT, int UN, bool GEMV_ROWS>
__global__ void __launch_bounds__(BLOCK)
batch_kernel(const DevInst* __restrict__ insts, const Tile* __restrict__ tiles, int64_t ntiles,
             float2* __restrict__ partials, unsigned* __restrict__ counters, unsigned long long*)
{
    __shared__ float2 sm[BLOCK / 32];
    __shared__ int is_last;
    constexpr int CH = PPT / 2;   // chunks per thread per tile
    constexpr int U = CH < UN ? CH : UN;

    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const DevInst I = insts[tl.inst];
        // compiled only into the kernels used by plans that hold GEMV rows:
        // its presence measurably slows the other paths (about 7% on the best
        // launch shape, 45% on the default one)
        if (GEMV_ROWS && I.kind == kGemvRows) {
            gemv_rows_tile(I.x, I.y, I.out, I.n, I.lda, I.m, I.vec, I.rows_per_warp, tl.start);
            continue;
        }
        const int64_t s0 = tl.start;
        const int64_t s1 = min(s0 + static_cast<int64_t>(BLOCK) * PPT, I.n);
        // vec == 2: the instance's arrays all start 8 bytes past a 16-byte
        // boundary, and so does every tile (tiles hold an even number of
        // values); thread 0 takes the tile's first value on its own and the
        // rest runs on 16-byte access
        const int64_t h = (I.vec == 2 && s1 > s0) ? 1 : 0;
        if (I.kind == FF_BATCH_DOT) {
            float2 acc = make_float2(0.0f, 0.0f);
            if (I.vec) {
                if (h && threadIdx.x == 0) acc = ffk::add22(acc, ffk::mul22(I.x[s0], I.y[s0]));
                const float4* xv = reinterpret_cast<const float4*>(I.x + s0 + h);
                const float4* yv = reinterpret_cast<const float4*>(I.y + s0 + h);
                const int64_t len = s1 - s0 - h;
                const int64_t nch = len >> 1;
#pragma unroll 1
                for (int j0 = 0; j0 < CH; j0 += U) {
                    float4 xs[U], ys[U];
                    bool ok[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int64_t c = threadIdx.x + static_cast<int64_t>(j0 + u) * BLOCK;
                        ok[u] = c < nch;
                        if (ok[u]) {
                            xs[u] = __ldcs(xv + c);
                            ys[u] = __ldcs(yv + c);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (ok[u]) {
                            acc = ffk::add22(acc, ffk::mul22(make_float2(xs[u].x, xs[u].y), make_float2(ys[u].x, ys[u].y)));
                            acc = ffk::add22(acc, ffk::mul22(make_float2(xs[u].z, xs[u].w), make_float2(ys[u].z, ys[u].w)));
                        }
                    }
                }
                if ((len & 1) && threadIdx.x == 0) acc = ffk::add22(acc, ffk::mul22(I.x[s1 - 1], I.y[s1 - 1]));
            } else {
                for (int j = 0; j < PPT; ++j) {
                    const int64_t i = s0 + threadIdx.x + static_cast<int64_t>(j) * BLOCK;
                    if (i < s1) acc = ffk::add22(acc, ffk::mul22(I.x[i], I.y[i]));
                }
            }
            acc = block_reduce<BLOCK>(acc, sm);
            if (I.ntiles == 1) {
                if (threadIdx.x == 0) *I.out = acc;
            } else {
                if (threadIdx.x == 0) {
                    partials[t] = acc;
                    __threadfence();
                    const unsigned old = atomicAdd(counters + tl.inst, 1u);
                    is_last = (old == static_cast<unsigned>(I.ntiles) - 1u);
                }
                __syncthreads();
                if (is_last) {
                    __threadfence();
                    float2 a2 = make_float2(0.0f, 0.0f);
                    for (int p = threadIdx.x; p < I.ntiles; p += BLOCK)
                        a2 = ffk::add22(a2, __ldcg(partials + I.first_tile + p));
                    a2 = block_reduce<BLOCK>(a2, sm);
                    if (threadIdx.x == 0) {
                        *I.out = a2;
                        counters[tl.inst] = 0u;
                    }
                }
                __syncthreads();
            }
        } else if (I.kind == FF_BATCH_DOT_GRAD) {
            const float2 d = __ldg(I.dout);
            if (I.vec) {
                if (h && threadIdx.x == 0) {
                    I.out[s0] = ffk::mul22(d, I.y[s0]);
                    I.out2[s0] = ffk::mul22(d, I.x[s0]);
                }
                const float4* xv = reinterpret_cast<const float4*>(I.x + s0 + h);
                const float4* yv = reinterpret_cast<const float4*>(I.y + s0 + h);
                float4* dxv = reinterpret_cast<float4*>(I.out + s0 + h);
                float4* dyv = reinterpret_cast<float4*>(I.out2 + s0 + h);
                const int64_t len = s1 - s0 - h;
                const int64_t nch = len >> 1;
#pragma unroll 1
                for (int j0 = 0; j0 < CH; j0 += U) {
                    float4 xs[U], ys[U];
                    bool ok[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int64_t c = threadIdx.x + static_cast<int64_t>(j0 + u) * BLOCK;
                        ok[u] = c < nch;
                        if (ok[u]) {
                            xs[u] = __ldcs(xv + c);
                            ys[u] = __ldcs(yv + c);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (ok[u]) {
                            const int64_t c = threadIdx.x + static_cast<int64_t>(j0 + u) * BLOCK;
                            const float2 gx0 = ffk::mul22(d, make_float2(ys[u].x, ys[u].y));
                            const float2 gx1 = ffk::mul22(d, make_float2(ys[u].z, ys[u].w));
                            const float2 gy0 = ffk::mul22(d, make_float2(xs[u].x, xs[u].y));
                            const float2 gy1 = ffk::mul22(d, make_float2(xs[u].z, xs[u].w));
                            __stcs(dxv + c, make_float4(gx0.x, gx0.y, gx1.x, gx1.y));
                            __stcs(dyv + c, make_float4(gy0.x, gy0.y, gy1.x, gy1.y));
                        }
                    }
                }
                if ((len & 1) && threadIdx.x == 0) {
                    I.out[s1 - 1] = ffk::mul22(d, I.y[s1 - 1]);
                    I.out2[s1 - 1] = ffk::mul22(d, I.x[s1 - 1]);
                }
            } else {
                for (int j = 0; j < PPT; ++j) {
                    const int64_t i = s0 + threadIdx.x + static_cast<int64_t>(j) * BLOCK;
                    if (i < s1) {
                        I.out[i] = ffk::mul22(d, I.y[i]);
                        I.out2[i] = ffk::mul22(d, I.x[i]);
                    }
                }
            }
        } else {
            const float2 al = I.alpha;
            if (I.vec) {
                if (h && threadIdx.x == 0) I.out[s0] = ffk::add22(ffk::mul22(al, I.x[s0]), I.y[s0]);
                const float4* xv = reinterpret_cast<const float4*>(I.x + s0 + h);
                const float4* yv = reinterpret_cast<const float4*>(I.y + s0 + h);
                float4* zv = reinterpret_cast<float4*>(I.out + s0 + h);
                const int64_t len = s1 - s0 - h;
                const int64_t nch = len >> 1;
#pragma unroll 1
                for (int j0 = 0; j0 < CH; j0 += U) {
                    float4 xs[U], ys[U];
                    bool ok[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int64_t c = threadIdx.x + static_cast<int64_t>(j0 + u) * BLOCK;
                        ok[u] = c < nch;
                        if (ok[u]) {
                            xs[u] = __ldcs(xv + c);
                            ys[u] = __ldcs(yv + c);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (ok[u]) {
                            const int64_t c = threadIdx.x + static_cast<int64_t>(j0 + u) * BLOCK;
                            const float2 r0 = ffk::add22(ffk::mul22(al, make_float2(xs[u].x, xs[u].y)),
                                                         make_float2(ys[u].x, ys[u].y));
                            const float2 r1 = ffk::add22(ffk::mul22(al, make_float2(xs[u].z, xs[u].w)),
                                                         make_float2(ys[u].z, ys[u].w));
                            __stcs(zv + c, make_float4(r0.x, r0.y, r1.x, r1.y));
                        }
                    }
                }
                if ((len & 1) && threadIdx.x == 0)
                    I.out[s1 - 1] = ffk::add22(ffk::mul22(al, I.x[s1 - 1]), I.y[s1 - 1]);
            } else {
                for (int j = 0; j < PPT; ++j) {
                    const int64_t i = s0 + threadIdx.x + static_cast<int64_t>(j) * BLOCK;
                    if (i < s1) I.out[i] = ffk::add22(ffk::mul22(al, I.x[i]), I.y[i]);
                }
            }
        }
    }
}

// Kernel for plans whose records are all GEMV rows: the same tile walk and
// row reduction, without the other paths, so that it needs few registers and
// keeps many warps resident: the rows are latency-bound (two 16-byte loads
// of A in flight per lane), so the register budget is set for a full SM of
// 64 warps (1024-GEMV batch: 0.86 of the HBM rate at 48 registers, 0.92 at
// 32).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 2048 / BLOCK)
batch_gemv_kernel(const DevInst* __restrict__ insts, const Tile* __restrict__ tiles, int64_t ntiles,
                  float2* __restrict__, unsigned* __restrict__, unsigned long long* __restrict__ next)
{
    __shared__ unsigned long long s_t;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(next, 1ull);
        __syncthreads();
        const unsigned long long t = s_t;
        __syncthreads();  // every thread has read s_t before thread 0 takes the next tile
        if (t >= static_cast<unsigned long long>(ntiles)) break;
        const Tile tl = tiles[t];
        const DevInst& I = insts[tl.inst];
        gemv_rows_tile_body(I.x, I.y, I.out, I.n, I.lda, I.m, I.vec, I.rows_per_warp, tl.start);
    }
}

using KernelFn = void (*)(const DevInst*, const Tile*, int64_t, float2*, unsigned*, unsigned long long*);

struct Variant {
    int block;
    int ppt;
    int unroll;
    KernelFn fn;            // plans without GEMV rows
    KernelFn fn_gemv;       // plans with GEMV rows and other records
    KernelFn fn_gemv_only;  // plans whose records are all GEMV rows
};

#define FF_BV(B, P, UN) {B, P, UN, batch_kernel<B, P, UN, false>, batch_kernel<B, P, UN, true>, batch_gemv_kernel<B>}
#define FF_BATCH_VARIANTS(UN)                                                                              \
    FF_BV(128, 16, UN), FF_BV(128, 32, UN), FF_BV(128, 64, UN), FF_BV(128, 128, UN), FF_BV(256, 8, UN),        \
        FF_BV(256, 16, UN), FF_BV(256, 32, UN), FF_BV(256, 64, UN), FF_BV(256, 128, UN), FF_BV(512, 8, UN),    \
        FF_BV(512, 16, UN), FF_BV(512, 32, UN), FF_BV(512, 64, UN)

const Variant kVariants[] = {FF_BATCH_VARIANTS(4), FF_BATCH_VARIANTS(2)};
#undef FF_BV
#undef FF_BATCH_VARIANTS

const Variant* find_variant(const ff_tune& t)
{
    const int un = t.unroll == 0 ? 4 : t.unroll;
    for (const Variant& v : kVariants)
        if (v.block == t.block && v.ppt == t.pairs_per_thread && v.unroll == un) return &v;
    return nullptr;
}

const ff_tune kDefaultTune = {256, 32, 0, 4};

KernelFn kernel_for(const Variant& v, const ff_batch_plan& p)
{
    return p.only_gemv_rows ? v.fn_gemv_only : (p.has_gemv_rows ? v.fn_gemv : v.fn);
}

// Workspace: the per-record counters (4 B each), the tile scheduler's 8-byte
// counter after them, padded to kCountersAlign; then one partial per tile.
size_t sched_offset(size_t nrec) { return (nrec * 4 + 7) / 8 * 8; }
size_t counters_bytes(size_t nrec) { return (sched_offset(nrec) + 8 + kCountersAlign - 1) / kCountersAlign * kCountersAlign; }

size_t ws_bytes_for(const ff_batch_plan* p)
{
    return counters_bytes(static_cast<size_t>(p->count)) + static_cast<size_t>(p->ntiles) * sizeof(float2) + 16;
}

ff_status validate(const ff_batch_instance* inst, int count)
{
    if (count < 0 || (count > 0 && inst == nullptr)) return FF_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        const ff_batch_instance& b = inst[i];
        if (b.n < 0 || (b.kind != FF_BATCH_DOT && b.kind != FF_BATCH_AXPY && b.kind != FF_BATCH_DOT_GRAD &&
                         b.kind != FF_BATCH_GEMV))
            return FF_ERR_INVALID_ARG;
        const size_t n = static_cast<size_t>(b.n);
        if (b.kind == FF_BATCH_GEMV) {
            if (b.m < 0 || b.lda < b.n || b.m > INT32_MAX) return FF_ERR_INVALID_ARG;
            const size_t m = static_cast<size_t>(b.m);
            if (!ffh::ok_ptr(b.x, m * static_cast<size_t>(b.lda)) || !ffh::ok_ptr(b.y, n) || !ffh::ok_ptr(b.out, m))
                return FF_ERR_INVALID_ARG;
            continue;
        }
        if (!ffh::ok_ptr(b.x, n) || !ffh::ok_ptr(b.y, n)) return FF_ERR_INVALID_ARG;
        if (b.kind == FF_BATCH_DOT && !ffh::ok_ptr(b.out, 1)) return FF_ERR_INVALID_ARG;
        if (b.kind == FF_BATCH_AXPY && !ffh::ok_ptr(b.out, n)) return FF_ERR_INVALID_ARG;
        if (b.kind == FF_BATCH_DOT_GRAD &&
            (!ffh::ok_ptr(b.out, n) || !ffh::ok_ptr(b.out2, n) || (n > 0 && !ffh::ok_ptr(b.dout, 1))))
            return FF_ERR_INVALID_ARG;
    }
    return FF_OK;
}

}  // namespace

extern "C" {

ff_status ff_batch_plan_create(const ff_batch_instance* inst, int count, const ff_tune* tune_or_null,
                               ff_batch_plan** out)
{
    if (!out) return FF_ERR_INVALID_ARG;
    *out = nullptr;
    ff_status st = validate(inst, count);
    if (st != FF_OK) return st;
    ff_tune tune = tune_or_null ? *tune_or_null : kDefaultTune;
    const Variant* var = find_variant(tune);
    if (!var || tune.blocks_per_sm < 0 || tune.blocks_per_sm > 32) return FF_ERR_INVALID_ARG;
    ffh::DeviceInfo di;
    st = ffh::device_info(&di);
    if (st != FF_OK) return st;

    const int64_t tile = static_cast<int64_t>(tune.block) * tune.pairs_per_thread;
    // one record per dot / AXPY / gradient instance and per GEMV row
    struct Rec {
        int kind;
        int64_t n;
        const void* x;
        const void* y;
        void* out;
        void* out2;
        const void* dout;
        ff2 alpha;
        int64_t lda;
        int64_t m;
    };
    std::vector<Rec> recs;
    recs.reserve(static_cast<size_t>(count));
    for (int i = 0; i < count; ++i) {
        const ff_batch_instance& b = inst[i];
        if (b.kind == FF_BATCH_GEMV && b.n <= kWarpRowMax) {
            if (b.m > 0) recs.push_back(Rec{kGemvRows, b.n, b.x, b.y, b.out, nullptr, nullptr, b.alpha, b.lda, b.m});
        } else if (b.kind == FF_BATCH_GEMV) {
            for (int64_t r = 0; r < b.m; ++r)
                recs.push_back(Rec{FF_BATCH_DOT, b.n, b.x + r * b.lda, b.y, b.out + r, nullptr, nullptr, b.alpha, 0, 0});
        } else {
            recs.push_back(Rec{b.kind, b.n, b.x, b.y, b.out, b.out2, b.dout, b.alpha, 0, 0});
        }
    }
    if (recs.size() > static_cast<size_t>(INT32_MAX)) return FF_ERR_INVALID_ARG;
    std::vector<DevInst> hi(recs.size());
    std::vector<Tile> ht;
    int64_t ndot = 0, total = 0;
    for (size_t i = 0; i < recs.size(); ++i) {
        const Rec& b = recs[i];
        DevInst& d = hi[i];
        d.x = static_cast<const float2*>(b.x);
        d.y = static_cast<const float2*>(b.y);
        d.out = static_cast<float2*>(b.out);
        d.out2 = static_cast<float2*>(b.out2);
        d.dout = static_cast<const float2*>(b.dout);
        d.alpha = make_float2(b.alpha.hi, b.alpha.lo);
        d.n = b.n;
        d.kind = b.kind;
        d.lda = b.lda;
        d.m = b.m;
        d.first_tile = static_cast<int64_t>(ht.size());
        d.rows_per_warp = 0;
        if (b.kind == kGemvRows) {
            // rows of 16-byte-aligned storage when the matrix, its row stride
            // and the vector allow it
            d.vec = (ffh::aligned(b.x, 16) && ffh::aligned(b.y, 16) && (b.lda % 2 == 0)) ? 1 : 0;
            // four rows per warp at a time, rpw groups of four per warp per
            // tile: about 16K values per tile
            const int64_t warps = tune.block / 32;
            int64_t rpw = 16384 / (4 * warps * (b.n > 0 ? b.n : 1));
            rpw = rpw < 1 ? 1 : (rpw > 16 ? 16 : rpw);
            d.rows_per_warp = static_cast<int32_t>(rpw);
            const int64_t rows_per_tile = 4 * warps * rpw;
            const int64_t nt = (b.m + rows_per_tile - 1) / rows_per_tile;
            if (nt > INT32_MAX) return FF_ERR_INVALID_ARG;
            d.ntiles = static_cast<int32_t>(nt);
            for (int64_t k = 0; k < nt; ++k) ht.push_back(Tile{static_cast<int32_t>(i), 0, k * rows_per_tile});
            total += b.m * b.n;
            continue;
        }
        // 16-byte access when every array the record reads or writes value
        // by value starts on a 16-byte boundary, or when all of them start 8
        // bytes past one (a one-value head realigns each tile); otherwise
        // 8-byte access
        {
            const uintptr_t m = reinterpret_cast<uintptr_t>(b.x) & 15u;
            bool same = (reinterpret_cast<uintptr_t>(b.y) & 15u) == m;
            if (b.kind != FF_BATCH_DOT) same = same && (reinterpret_cast<uintptr_t>(b.out) & 15u) == m;
            if (b.kind == FF_BATCH_DOT_GRAD) same = same && (reinterpret_cast<uintptr_t>(b.out2) & 15u) == m;
            d.vec = !same ? 0 : (m == 0 ? 1 : (m == 8 ? 2 : 0));
        }
        // a dot of length 0 still needs one tile to write its (0, 0)
        const int64_t nt = b.n > 0 ? (b.n + tile - 1) / tile : (b.kind == FF_BATCH_DOT ? 1 : 0);
        if (nt > INT32_MAX) return FF_ERR_INVALID_ARG;
        d.ntiles = static_cast<int32_t>(nt);
        for (int64_t k = 0; k < nt; ++k) ht.push_back(Tile{static_cast<int32_t>(i), 0, k * tile});
        ndot += (b.kind == FF_BATCH_DOT);
        total += b.n;
    }
    auto* p = new (std::nothrow) ff_batch_plan();
    if (!p) return FF_ERR_UNSUPPORTED;
    p->count = static_cast<int>(recs.size());
    p->has_gemv_rows = false;
    p->only_gemv_rows = !recs.empty();
    for (const Rec& r : recs) {
        p->has_gemv_rows |= (r.kind == kGemvRows);
        p->only_gemv_rows &= (r.kind == kGemvRows);
    }
    if (p->only_gemv_rows) {
        // largest tiles first (values + a fixed cost per row of 64 values),
        // taken in this order by the blocks of the GEMV-only kernel
        const int64_t warps = tune.block / 32;
        auto cost = [&](const Tile& t) {
            const DevInst& d = hi[static_cast<size_t>(t.inst)];
            const int64_t rows = std::min<int64_t>(4 * warps * d.rows_per_warp, d.m - t.start);
            return rows * (d.n + 64);
        };
        std::stable_sort(ht.begin(), ht.end(), [&](const Tile& a, const Tile& b) { return cost(a) > cost(b); });
    }
    p->tune = tune;
    p->ntiles = static_cast<int64_t>(ht.size());
    p->ndot = ndot;
    p->total_values = total;
    p->device = di.device;
    int bps = tune.blocks_per_sm;
    if (bps == 0)
        bps = ffh::occupancy(reinterpret_cast<const void*>(kernel_for(*var, *p)), tune.block);
    int64_t grid = static_cast<int64_t>(di.sm_count) * (bps > 0 ? bps : 1);
    if (grid > p->ntiles) grid = p->ntiles > 0 ? p->ntiles : 1;
    p->grid = static_cast<unsigned>(grid);
    p->d_inst = nullptr;
    p->d_tiles = nullptr;
    if (!hi.empty()) {
        cudaError_t e = cudaMalloc(&p->d_inst, hi.size() * sizeof(DevInst));
        if (e == cudaSuccess && !ht.empty()) e = cudaMalloc(&p->d_tiles, ht.size() * sizeof(Tile));
        if (e == cudaSuccess) e = cudaMemcpy(p->d_inst, hi.data(), hi.size() * sizeof(DevInst), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !ht.empty())
            e = cudaMemcpy(p->d_tiles, ht.data(), ht.size() * sizeof(Tile), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(p->d_inst);
            cudaFree(p->d_tiles);
            delete p;
            return ffh::cuda_status(e);
        }
    }
    *out = p;
    return FF_OK;
}

size_t ff_batch_workspace_bytes(const ff_batch_plan* p) { return p ? ws_bytes_for(p) : 0; }

ff_status ff_batch_plan_info(const ff_batch_plan* p, ff_tune* tune, int64_t* ntiles, unsigned* grid)
{
    if (!p) return FF_ERR_INVALID_ARG;
    if (tune) *tune = p->tune;
    if (ntiles) *ntiles = p->ntiles;
    if (grid) *grid = p->grid;
    return FF_OK;
}

ff_status ff_batch_run(const ff_batch_plan* p, void* ws, size_t ws_bytes, cudaStream_t s)
{
    if (!p) return FF_ERR_INVALID_ARG;
    if (p->ntiles == 0) return FF_OK;
    if (ws == nullptr || ws_bytes < ws_bytes_for(p) || !ffh::aligned(ws, 16)) return FF_ERR_WORKSPACE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return FF_ERR_INVALID_ARG;
    const Variant* var = find_variant(p->tune);
    if (!var) return FF_ERR_INVALID_ARG;
    auto* counters = static_cast<unsigned*>(ws);
    const size_t so = sched_offset(static_cast<size_t>(p->count));
    auto* next = reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + so);
    auto* partials = reinterpret_cast<float2*>(static_cast<char*>(ws) + counters_bytes(static_cast<size_t>(p->count)));
    ff_status st = ffh::cuda_status(cudaMemsetAsync(counters, 0, so + 8, s));
    if (st != FF_OK) return st;
    kernel_for(*var, *p)<<<p->grid, p->tune.block, 0, s>>>(p->d_inst, p->d_tiles, p->ntiles, partials, counters,
                                                           next);
    return ffh::check_launch();
}

void ff_batch_plan_destroy(ff_batch_plan* p)
{
    if (!p) return;
    cudaFree(p->d_inst);
    cudaFree(p->d_tiles);
    delete p;
}

ff_status ff_batch_graph_create(const ff_batch_plan* p, void* ws, size_t ws_bytes, ff_batch_graph** out)
{
    if (!p || !out) return FF_ERR_INVALID_ARG;
    *out = nullptr;
    if (p->ntiles > 0 && (ws == nullptr || ws_bytes < ws_bytes_for(p) || !ffh::aligned(ws, 16)))
        return FF_ERR_WORKSPACE;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return ffh::cuda_status(e);
    auto* g = new (std::nothrow) ff_batch_graph();
    if (!g) {
        cudaStreamDestroy(cs);
        return FF_ERR_UNSUPPORTED;
    }
    g->graph = nullptr;
    g->exec = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    ff_status st = FF_OK;
    if (e == cudaSuccess) {
        st = ff_batch_run(p, ws, ws_bytes, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
        if (st == FF_OK && e2 != cudaSuccess) st = ffh::cuda_status(e2);
    } else {
        st = ffh::cuda_status(e);
    }
    if (st == FF_OK) st = ffh::cuda_status(cudaGraphInstantiate(&g->exec, g->graph, 0));
    cudaStreamDestroy(cs);
    if (st != FF_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return st;
    }
    *out = g;
    return FF_OK;
}

ff_status ff_batch_graph_launch(ff_batch_graph* g, cudaStream_t s)
{
    if (!g) return FF_ERR_INVALID_ARG;
    return ffh::cuda_status(cudaGraphLaunch(g->exec, s));
}

void ff_batch_graph_destroy(ff_batch_graph* g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

int ff_batch_tune_candidates(ff_tune* out, int max)
{
    const int per = 3;  // blocks per SM: occupancy-limited (0), 2, 4
    const int bps[per] = {0, 2, 4};
    int k = 0;
    for (const Variant& v : kVariants)
        for (int b = 0; b < per; ++b) {
            if (out && k < max) out[k] = ff_tune{v.block, v.ppt, bps[b], v.unroll};
            ++k;
        }
    return k;
}

size_t ff_batch_autotune_workspace_bytes(const ff_batch_instance* inst, int count)
{
    if (count < 0 || (count > 0 && !inst)) return 0;
    // the smallest tile of any candidate gives the most tiles
    int64_t smallest = INT64_MAX;
    for (const Variant& v : kVariants) smallest = std::min<int64_t>(smallest, static_cast<int64_t>(v.block) * v.ppt);
    size_t ntiles = 0, nrec = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t n = inst[i].n;
        const size_t reps = (inst[i].kind == FF_BATCH_GEMV) ? static_cast<size_t>(inst[i].m > 0 ? inst[i].m : 0) : 1;
        ntiles += reps * static_cast<size_t>(n > 0 ? (n + smallest - 1) / smallest : 1);
        nrec += reps;
    }
    return counters_bytes(nrec) + ntiles * sizeof(float2) + 16;
}

ff_status ff_batch_autotune(const ff_batch_instance* inst, int count, void* ws, size_t ws_bytes, cudaStream_t s,
                            int reps, ff_tune* best, float* best_ms)
{
    if (!best) return FF_ERR_INVALID_ARG;
    ff_status st = validate(inst, count);
    if (st != FF_OK) return st;
    if (reps < 1) reps = 1;
    const int nc = ff_batch_tune_candidates(nullptr, 0);
    std::vector<ff_tune> cands(static_cast<size_t>(nc));
    ff_batch_tune_candidates(cands.data(), nc);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    st = ffh::cuda_status(cudaEventCreate(&e0));
    if (st == FF_OK) st = ffh::cuda_status(cudaEventCreate(&e1));
    float best_t = -1.0f;
    ff_tune best_tune = kDefaultTune;
    for (int c = 0; c < nc && st == FF_OK; ++c) {
        ff_batch_plan* p = nullptr;
        st = ff_batch_plan_create(inst, count, &cands[static_cast<size_t>(c)], &p);
        if (st != FF_OK) break;
        if (ws_bytes < ws_bytes_for(p)) {
            ff_batch_plan_destroy(p);
            st = FF_ERR_WORKSPACE;
            break;
        }
        st = ff_batch_run(p, ws, ws_bytes, s);  // warm-up
        if (st == FF_OK) st = ffh::cuda_status(cudaEventRecord(e0, s));
        for (int r = 0; r < reps && st == FF_OK; ++r) st = ff_batch_run(p, ws, ws_bytes, s);
        if (st == FF_OK) st = ffh::cuda_status(cudaEventRecord(e1, s));
        if (st == FF_OK) st = ffh::cuda_status(cudaEventSynchronize(e1));
        float ms = 0.0f;
        if (st == FF_OK) st = ffh::cuda_status(cudaEventElapsedTime(&ms, e0, e1));
        ff_batch_plan_destroy(p);
        if (st != FF_OK) break;
        ms /= static_cast<float>(reps);
        if (best_t < 0.0f || ms < best_t) {
            best_t = ms;
            best_tune = cands[static_cast<size_t>(c)];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != FF_OK) return st;
    *best = best_tune;
    if (best_ms) *best_ms = best_t;
    return FF_OK;
}

}  // extern "C"
