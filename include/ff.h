/*
 * ff.h -- C ABI of the GB300 float-float library (libff.so).
 *
 * Float-float arithmetic after Da Graca & Defour, "Implementation of
 * float-float operators on graphics hardware" (arXiv cs/0603115): a number is
 * the unevaluated sum hi + lo of two IEEE binary32 values (the format of
 * Section 4), about 44 bits of precision with the exponent range of binary32
 * (Section 7).
 *
 * Conventions that hold for every entry point unless its comment says
 * otherwise:
 *   - Memory.  Every array argument is a DEVICE pointer owned by the caller,
 *     at least 8-byte aligned (the alignment of ff2); 16-byte alignment is
 *     not required.  The library never allocates device memory inside a
 *     call (ff_batch_plan_create, which builds a plan, is the one exception):
 *     scratch space is a caller-owned workspace whose size the matching
 *     *_workspace_bytes() function returns.
 *   - Streams.  Calls only enqueue work on the caller's stream `s` (0 = the
 *     legacy default stream) and return at once; results, including the
 *     scalar result of a reduction, stay on the device.  No call
 *     synchronises.  A call is safe to capture in a CUDA graph when its
 *     arguments stay valid for the graph's lifetime.
 *   - Errors.  Arguments are checked on the host before anything is
 *     enqueued: a NULL pointer with n > 0, a pointer not 8-byte aligned, a
 *     negative size or stride, or a stride smaller than its extent returns
 *     FF_ERR_INVALID_ARG; a workspace that is NULL or too small returns
 *     FF_ERR_WORKSPACE.  A failed launch returns FF_ERR_CUDA and keeps the
 *     CUDA error code for ff_last_cuda_error().  Nothing is enqueued when a
 *     call returns an argument or workspace error; when a call that makes
 *     several launches (a GEMV of several column tiles, a weight gradient
 *     in two passes, a GEMV adjoint and its combination) fails to launch
 *     one, the launches before it stay enqueued.
 *   - Sizes.  n == 0 is a no-op returning FF_OK, except that a reduction
 *     with n == 0 writes (0, 0) to its result.
 *   - Aliasing.  An elementwise output may be exactly one of its inputs
 *     (in place); any other overlap is undefined.
 *   - Results.  Every elementwise result is the exact op sequence of the
 *     cited algorithm in binary32 round-to-nearest-even, with subnormals
 *     kept: bit-for-bit reproducible.  Reductions follow the fixed tree order
 *     documented with ff_sum and are bit-for-bit reproducible for a given n,
 *     device and build.
 */
#ifndef FF_GB300_H
#define FF_GB300_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define FF_API __attribute__((visibility("default")))
#else
#define FF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* One float-float value, layout-compatible with CUDA float2: hi in x, lo in
 * y.  For the error-free transformations an ff2 is also used for a packed
 * pair of binary32 operands (a, b) or results (s, e). */
typedef struct ff2 {
    float hi;
    float lo;
} ff2;

typedef enum ff_status {
    FF_OK = 0,
    FF_ERR_INVALID_ARG = 1,
    FF_ERR_WORKSPACE = 2,
    FF_ERR_CUDA = 3,
    FF_ERR_TIMEOUT = 4,
    FF_ERR_UNSUPPORTED = 5
} ff_status;

/* ------------------------------------------------------------------------ */
/* Error-free transformations (Section 4.1)                                  */
/* ------------------------------------------------------------------------ */

/* Add12 theorem (Knuth, branch free): for each i, with (a, b) = ab[i],
 * se[i] = (s, e) where s = RN(a + b) and s + e = a + b exactly.
 * ab: n packed binary32 operand pairs; se: n result pairs. */
FF_API ff_status ff_add12(const ff2* ab, ff2* se, size_t n, cudaStream_t s);

/* Mul12 theorem (Dekker): for each i, pe[i] = (p, e) with p = RN(a * b) and
 * p + e = a * b exactly (no under- or overflow).  Computed as
 * e = fma(a, b, -p), equal to the paper's Split form wherever both are
 * defined. */
FF_API ff_status ff_mul12(const ff2* ab, ff2* pe, size_t n, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Float-float operators (elementwise, n values each)                        */
/* ------------------------------------------------------------------------ */

/* Add22 theorem: out[i] = Add22(a[i], b[i]),
 * |err| <= max(2^-24 |al + bl|, 2^-44 |a + b|). */
FF_API ff_status ff_add(const ff2* a, const ff2* b, ff2* out, size_t n, cudaStream_t s);

/* Accurate float-float addition (the paper leaves Add22's cancellation error
 * as open work, Sections 6.1 and 7): Joldes, Muller and Popescu (2017),
 * Algorithm 6 -- TwoSum of the high parts, TwoSum of the low parts, two
 * Fast2Sum renormalisations.  out[i] = a[i] + b[i] with relative error
 * <= 3 2^-48 / (1 - 2^-22), also under cancellation. */
FF_API ff_status ff_add_accurate(const ff2* a, const ff2* b, ff2* out, size_t n, cudaStream_t s);

/* Mul22 theorem: out[i] = Mul22(a[i], b[i]), relative error <= 2^-44. */
FF_API ff_status ff_mul(const ff2* a, const ff2* b, ff2* out, size_t n, cudaStream_t s);

/* Division a[i] / b[i] (not in the paper; Dekker's div2, the construction the
 * paper's Split and Mul12 come from, finished with the paper's Add12).
 * Divisors are expected to satisfy |b.hi| >= 2^-60; b.hi == 0 gives the IEEE
 * infinities or NaN of ah / bh. */
FF_API ff_status ff_div(const ff2* a, const ff2* b, ff2* out, size_t n, cudaStream_t s);

/* Square root of a[i] (not in the paper; Dekker's sqrt2 finished with
 * Add12).  a.hi == +-0 gives (a.hi, 0); a.hi < 0 gives (NaN, NaN). */
FF_API ff_status ff_sqrt(const ff2* a, ff2* out, size_t n, cudaStream_t s);

/* z[i] = Add22(Mul22(alpha, x[i]), y[i]); alpha is passed by value. */
FF_API ff_status ff_axpy(ff2 alpha, const ff2* x, const ff2* y, ff2* z, size_t n, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Compensated reductions (future work of Section 7)                       */
/* ------------------------------------------------------------------------ */

/* Workspace bytes for ff_sum / ff_dot / ff_sum2 / ff_dot2 / ff_f64_dot on
 * the current device (independent of n above a small size; always > 0).
 * A reduction workspace starts with a 4-byte arrival ticket that must be
 * zero before the first call that uses the workspace (clear the whole
 * buffer once when it is allocated, e.g. with cudaMemsetAsync); every call
 * leaves it zero again when its kernel ends, so later calls need no
 * clearing.  Storing anything else in the workspace between calls (or a
 * device fault during a call) requires clearing it again. */
FF_API size_t ff_reduce_workspace_bytes(size_t n);

/* *out_dev = the float-float sum of x[0..n) by Add22.  Order: thread t of a
 * grid of T threads accumulates, left to right, its elements of a
 * grid-stride sweep over the array (in two-value chunks), starting from
 * (0, 0); each warp then combines its 32 lanes by a shuffle-down tree, each
 * block its warps likewise, and the last block to finish combines the
 * per-block partials in block order.  ws: caller-owned device workspace of
 * at least ff_reduce_workspace_bytes(n) bytes, 16-byte aligned, its ticket
 * zero (see ff_reduce_workspace_bytes); it is written by the call and must
 * not be used concurrently by another call.  One launch, no memset.
 * Error bound for the stored result r: |r - sum x_i| <= n 2^-46 sum |x_i|. */
FF_API ff_status ff_sum(const ff2* x, size_t n, ff2* out_dev, void* ws, size_t ws_bytes, cudaStream_t s);

/* *out_dev = sum_i Mul22(x[i], y[i]) with the same Add22 tree as ff_sum.
 * |r - sum x_i y_i| <= n 2^-46 sum |x_i y_i|. */
FF_API ff_status ff_dot(const ff2* x, const ff2* y, size_t n, ff2* out_dev, void* ws, size_t ws_bytes,
                 cudaStream_t s);

/* ff_dot without a workspace argument, for callers that cannot allocate
 * device memory: a plugin whose host application owns every device
 * allocation through its own pool and budget, or a latency-critical path on
 * which cudaMalloc and cudaFree (which can synchronise the whole device) are
 * not allowed.  The paper has no counterpart to this entry point.
 *
 * Same result as ff_dot (same launch shape, same combination order), but
 * its scratch -- the arrival ticket and up to 2048 per-block partial sums,
 * 16,640 bytes -- is one fixed array inside the library, present on every
 * GPU that loads the library until the process exits.  The call allocates
 * nothing; it clears the ticket with an asynchronous memset on stream s
 * before its kernel.
 *   - All calls share the one array, which keeps the previous call's
 *     contents: calls that overlap on the GPU (on different streams, or from
 *     different host threads without ordering) race and give wrong results.
 *     Order them on one stream.
 *   - The first call on each device looks up the array's device address,
 *     with that device current; make that first call before any stream
 *     capture.
 *   - Returns FF_ERR_WORKSPACE when the launch would need more than 2048
 *     partial sums (more than 256 SMs); a 152-SM GB300 needs at most 1216. */
FF_API ff_status ff_dot_noalloc(const ff2* x, const ff2* y, size_t n, ff2* out_dev, cudaStream_t s);

/* Launch shape ff_sum / ff_dot use for these arguments (nothing is
 * launched): *grid blocks of 256 threads; *head = 1 when one leading element
 * is accumulated alone by thread 0 to reach a 16-byte boundary; *vector = 1
 * for the two-value chunk sweep, 0 for the one-value sweep used when x and y
 * have different offsets modulo 16 bytes.  y may be NULL (ff_sum).  Lets a
 * caller reproduce the documented combination order exactly. */
FF_API ff_status ff_reduce_launch_shape(const ff2* x, const ff2* y, size_t n, unsigned* grid, int* head,
                                        int* vector);

/* Adjoint of d = ff_dot(x, y): given the float-float cotangent *dout_dev
 * (device), dx[i] = Mul22(dout, y[i]) and dy[i] = Mul22(dout, x[i]).  The
 * gradient of a float-float value is a float-float value holding
 * dL/d(hi + lo). */
FF_API ff_status ff_dot_backward(const ff2* dout_dev, const ff2* x, const ff2* y, ff2* dx, ff2* dy,
                          size_t n, cudaStream_t s);

/* Compensated sum and dot product of plain binary32 vectors (the paper's
 * compensated algorithms, future work in Section 7): Ogita, Rump and Oishi's Sum2 and
 * Dot2 (2005) with Add12 as TwoSum and the fused Mul12 as TwoProduct, per
 * thread in the sweep order of ff_sum (16-byte chunks of four values, up to
 * three leading values alone on thread 0), combined across threads, warps and
 * blocks by (p, q) = TwoSum(a.p, b.p), s = a.s + (b.s + q).  *out_dev is the
 * float-float Add12(p, s).  x, y: 4-byte aligned binary32 arrays; ws as for
 * ff_sum.  Reads 4 (Sum2) or 8 (Dot2) bytes per value, half of ff_sum /
 * ff_dot, for about twice the binary32 precision. */
FF_API ff_status ff_sum2(const float* x, size_t n, ff2* out_dev, void* ws, size_t ws_bytes, cudaStream_t s);
FF_API ff_status ff_dot2(const float* x, const float* y, size_t n, ff2* out_dev, void* ws, size_t ws_bytes,
                         cudaStream_t s);

/* Launch shape of ff_sum2 / ff_dot2 (as ff_reduce_launch_shape; *head is up
 * to 3 leading values, the vector sweep moves four values per step). */
FF_API ff_status ff_reduce2_launch_shape(const float* x, const float* y, size_t n, unsigned* grid, int* head,
                                         int* vector);

/* ------------------------------------------------------------------------ */
/* Float-float GEMV and its adjoint                                          */
/* ------------------------------------------------------------------------ */

/* Y = A X with the paper's operators (Section 4.1; the GEMV itself is not in
 * the paper): every term a Mul22, every accumulation an Add22.  A: m x n
 * row-major with row stride lda >= n (elements); X: n x k column-major,
 * column stride ldx >= n; Y: m x k column-major, column stride ldy >= m,
 * overwritten.  1 <= k <= 64.
 * Order: row r is reduced by one warp; lane l accumulates, from (0, 0), the
 * two-value chunks l, l + 32, l + 64, ... of the row in order (the single
 * values l, l + 32, ... when the row or X is not 16-byte aligned), then the
 * lanes are combined by a shuffle-down Add22 tree (offsets 16, 8, 4, 2, 1).
 * The order does not depend on k, so Y is bit-reproducible for any k and
 * launch.  Error per element: within n 2^-44 sum_j |A[r, j] X[j, c]| of the
 * exact value (the Add22 and Mul22 bounds of Section 4.1 summed over the
 * terms). */
FF_API ff_status ff_gemv(const ff2* A, int64_t m, int64_t n, int64_t lda, const ff2* X, int64_t ldx,
                  int64_t k, ff2* Y, int64_t ldy, cudaStream_t s);

/* Workspace bytes for ff_gemv_t on the current device. */
FF_API size_t ff_gemv_t_workspace_bytes(int64_t m, int64_t n, int64_t k);

/* dX = A^T dY (the adjoint of ff_gemv with respect to X).  dY: m x k
 * column-major (stride lddy >= m); dX: n x k column-major (stride
 * lddx >= n), overwritten.  1 <= k <= 64.
 * Order: A is cut into row blocks (their number depends on m, n, k and the
 * device's SM count); within a block each column accumulates its rows in
 * order with Add22 from (0, 0); the blocks' partial sums go to the workspace
 * (caller-owned, ff_gemv_t_workspace_bytes, 16-byte aligned) and are added
 * in row-block order.  Bit-reproducible for a given device and build; error
 * within m 2^-44 sum_r |A[r, j] dY[r, c]|. */
FF_API ff_status ff_gemv_t(const ff2* A, int64_t m, int64_t n, int64_t lda, const ff2* dY,
                    int64_t lddy, int64_t k, ff2* dX, int64_t lddx, void* ws, size_t ws_bytes,
                    cudaStream_t s);

/* The row-block count ff_gemv_t uses for these arguments on the current
 * device, and whether it takes 16-byte access (1) or not (0): the block
 * b covers rows [b * ceil(m / row_blocks), (b + 1) * ceil(m / row_blocks)).
 * Lets a test replay the adjoint's order exactly.  Invalid sizes or NULL
 * outputs return FF_ERR_INVALID_ARG. */
FF_API ff_status ff_gemv_t_launch_shape(const ff2* A, int64_t m, int64_t n, int64_t lda, int64_t k,
                                        int64_t* row_blocks, int* vector);

/* Weight gradient of Y = A X: dA = dY X^T, dA[r, j] = sum over c of
 * Mul22(dY[r, c], X[j, c]), accumulated with Add22 in order c = 0 .. k-1
 * (bit-reproducible).  dY: m x k column-major (lddy >= m); X: n x k
 * column-major (ldx >= n); dA: m x n row-major (ldda >= n), overwritten;
 * it must not overlap dY or X.  1 <= k <= 64.  Every element starts from
 * (0, 0) as the sum's definition says; its first Add22 (with the zero) is
 * formed in two additions when the term is a finite normalised pair (the
 * same bits), the full Add22 otherwise.  Up to k = 21 (with even n, ldx and
 * ldda and 16-byte aligned X and dA; up to 12 otherwise) it runs its own
 * kernel, in one pass up to k = 12 and in two above (the second continuing
 * from the sums the first stored); from there on it runs ff_gemm
 * (transa = 1 on dY), which forms the same terms in the same order. */
FF_API ff_status ff_gemv_dA(const ff2* dY, int64_t m, int64_t lddy, const ff2* X, int64_t n, int64_t ldx,
                            int64_t k, ff2* dA, int64_t ldda, cudaStream_t s);

/* Float-float matrix product (a GEMV with many right-hand sides; not in the
 * paper): C = op(A) op(B) with
 *   C[i, j] = acc over p = 0 .. k-1 of Add22(acc, Mul22(op(A)[i, p], op(B)[p, j])),
 * acc starting at (0, 0), p in increasing order (Section 4.1 operators).
 * The order does not depend on the launch, so every element is bit-identical
 * to that plain loop; its error is at most k 2^-44 sum_p |op(A)[i,p] op(B)[p,j]|.
 * All matrices are row-major device arrays owned by the caller:
 *   op(A) is m x k: A[i * lda + p] (transa = 0, lda >= k) or A[p * lda + i]
 *     (transa = 1: A is stored k x m, lda >= m);
 *   op(B) is k x n: B[p * ldb + j] (transb = 0, ldb >= n) or B[j * ldb + p]
 *     (transb = 1: B is stored n x k, ldb >= k);
 *   C is m x n, C[i * ldc + j] (ldc >= n), overwritten; it must not overlap A
 *     or B.
 * k = 0 writes (0, 0) to C; m = 0 or n = 0 is a no-op (no pointer is
 * checked or read).  Negative sizes,
 * transa / transb other than 0 or 1, short leading dimensions or NULL /
 * non-8-byte-aligned pointers return FF_ERR_INVALID_ARG before anything is
 * enqueued.  The adjoints of C = A B are dA = dC B^T (transb = 1) and
 * dB = A^T dC (transa = 1). */
FF_API ff_status ff_gemm(int transa, int transb, int64_t m, int64_t n, int64_t k, const ff2* A, int64_t lda,
                         const ff2* B, int64_t ldb, ff2* C, int64_t ldc, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Batched dot / AXPY: many instances in one persistent launch               */
/* ------------------------------------------------------------------------ */

typedef enum ff_batch_kind {
    FF_BATCH_DOT = 0,
    FF_BATCH_AXPY = 1,
    FF_BATCH_DOT_GRAD = 2,
    FF_BATCH_GEMV = 3
} ff_batch_kind;

/* One instance.
 *   DOT:      *out = sum_i Mul22(x[i], y[i]) (out: one ff2), with the Add22
 *             accumulation of ff_dot.
 *   AXPY:     out[i] = Add22(Mul22(alpha, x[i]), y[i]) for i < n (out: n
 *             values), bit-identical to ff_axpy.
 *   DOT_GRAD: the adjoint of a dot: out[i] = Mul22(*dout, y[i]) and
 *             out2[i] = Mul22(*dout, x[i]) (dout: one ff2 read on the device
 *             when the run executes), bit-identical to ff_dot_backward.
 *   GEMV:     out[r] = sum_j Mul22(x[r * lda + j], y[j]) for r < m: x is an
 *             m x n row-major matrix (row stride lda >= n), y a vector of n
 *             values, out m values; each row is reduced like a DOT instance.
 * All pointers are device pointers owned by the caller and must stay valid
 * while any plan or graph built from the instance is used; unused pointers
 * may be NULL.  Arrays need 8-byte alignment; an instance whose arrays all
 * share their offset modulo 16 bytes runs on 16-byte access (after one
 * value when that offset is 8), others on 8-byte access. */
typedef struct ff_batch_instance {
    int32_t kind;
    int32_t reserved;
    int64_t n;
    const ff2* x;
    const ff2* y;
    ff2* out;
    ff2* out2;
    const ff2* dout;
    ff2 alpha;
    int64_t m;   /* GEMV: rows */
    int64_t lda; /* GEMV: row stride of x */
} ff_batch_instance;

/* Launch configuration of the batched kernel: threads per block (128, 256
 * or 512), values per thread per tile (pairs_per_thread: 8 .. 128, tile =
 * block x pairs_per_thread values), resident blocks per SM (0 = as many as
 * fit) and two-value chunks per input loaded ahead of use (unroll: 2 or 4;
 * 0 = 4). */
typedef struct ff_tune {
    int32_t block;
    int32_t pairs_per_thread;
    int32_t blocks_per_sm;
    int32_t unroll;
} ff_tune;

typedef struct ff_batch_plan ff_batch_plan;
typedef struct ff_batch_graph ff_batch_graph;

/* Build a plan on the current device: cut every instance into tiles and copy
 * the instance records and the tile list to device memory the plan owns
 * (the only allocation of the library, made here, never in a run).
 * tune_or_null == NULL uses {256, 32, 0, 4}.  Unsupported tunes return
 * FF_ERR_INVALID_ARG. */
FF_API ff_status ff_batch_plan_create(const ff_batch_instance* inst, int count, const ff_tune* tune_or_null,
                                      ff_batch_plan** out);

/* Workspace bytes ff_batch_run needs for this plan. */
FF_API size_t ff_batch_workspace_bytes(const ff_batch_plan* plan);

/* The plan's tune, tile count and grid (any pointer may be NULL). */
FF_API ff_status ff_batch_plan_info(const ff_batch_plan* plan, ff_tune* tune, int64_t* ntiles, unsigned* grid);

/* Run every instance of the plan: one memset of the per-instance counters
 * and the tile counter, and one persistent kernel launch on stream s.
 * Graph-capturable.  The workspace (ff_batch_workspace_bytes, 16-byte
 * aligned, owned by the caller) must not be shared by runs that overlap. */
FF_API ff_status ff_batch_run(const ff_batch_plan* plan, void* ws, size_t ws_bytes, cudaStream_t s);

/* Free the plan's device and host memory (NULL is a no-op).  The caller must
 * make sure no run of it is still executing. */
FF_API void ff_batch_plan_destroy(ff_batch_plan* plan);

/* Capture ff_batch_run(plan, ws) into a CUDA graph (on a private stream)
 * and instantiate it. */
FF_API ff_status ff_batch_graph_create(const ff_batch_plan* plan, void* ws, size_t ws_bytes,
                                       ff_batch_graph** out);

/* Launch the instantiated graph on stream s. */
FF_API ff_status ff_batch_graph_launch(ff_batch_graph* g, cudaStream_t s);

/* Destroy the graph (NULL is a no-op). */
FF_API void ff_batch_graph_destroy(ff_batch_graph* g);

/* The autotuner's candidate tunes: writes up to max of them to out (out may
 * be NULL) and returns how many there are. */
FF_API int ff_batch_tune_candidates(ff_tune* out, int max);

/* Workspace bytes that suffice for ff_batch_autotune on these instances. */
FF_API size_t ff_batch_autotune_workspace_bytes(const ff_batch_instance* inst, int count);

/* Time every candidate tune on these instances (one warm-up run, then reps
 * runs each, CUDA events on stream s; the instances' outputs are
 * overwritten) and return the fastest in *best and its mean time per run in
 * *best_ms (may be NULL).  Synchronises with stream s. */
FF_API ff_status ff_batch_autotune(const ff_batch_instance* inst, int count, void* ws, size_t ws_bytes,
                                   cudaStream_t s, int reps, ff_tune* best, float* best_ms);

/* ------------------------------------------------------------------------ */
/* Native baselines on the same GPU (measurement only)                       */
/* ------------------------------------------------------------------------ */

/* Binary64: out[i] = a[i] op b[i] (op = +, *, /) and sqrt(a[i]). */
FF_API ff_status ff_f64_add(const double* a, const double* b, double* out, size_t n, cudaStream_t s);
FF_API ff_status ff_f64_mul(const double* a, const double* b, double* out, size_t n, cudaStream_t s);
FF_API ff_status ff_f64_div(const double* a, const double* b, double* out, size_t n, cudaStream_t s);
FF_API ff_status ff_f64_sqrt(const double* a, double* out, size_t n, cudaStream_t s);
/* Binary64 dot product (fma accumulation, same tree shape as ff_dot); ws as
 * for ff_sum (a reduction workspace, its ticket zero). */
FF_API ff_status ff_f64_dot(const double* x, const double* y, size_t n, double* out_dev, void* ws,
                     size_t ws_bytes, cudaStream_t s);
/* Binary64 GEMV, same layouts as ff_gemv. */
FF_API ff_status ff_f64_gemv(const double* A, int64_t m, int64_t n, int64_t lda, const double* X,
                      int64_t ldx, int64_t k, double* Y, int64_t ldy, cudaStream_t s);

/* Plain binary32 add, multiply and multiply-add (two roundings), the
 * normalisation baseline of the paper's timing tables (Section 6). */
FF_API ff_status ff_f32_add(const float* a, const float* b, float* out, size_t n, cudaStream_t s);
FF_API ff_status ff_f32_mul(const float* a, const float* b, float* out, size_t n, cudaStream_t s);
FF_API ff_status ff_f32_mad(const float* a, const float* b, const float* c, float* out, size_t n,
                     cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Measurement                                                               */
/* ------------------------------------------------------------------------ */

/* FMA throughput probe (not in the paper: it measures the arithmetic peak
 * that the FP32-issue-bound kernels and the FP64 baselines are compared
 * with).  Launches `blocks` x `threads` threads; each runs eight independent
 * chains x <- fma(x, 1, 1) (binary32 when f64 == 0, binary64 when f64 == 1)
 * for `iters` rounds and writes the sum of its chains to out[thread] (a
 * device array of blocks * threads floats or doubles, 8-byte aligned, owned
 * by the caller); chain c starts at c and ends at c + iters, so every
 * thread writes 28 + 8 iters.
 * One launch performs 16 * iters * blocks * threads floating-point
 * operations; the caller times it (CUDA events on `s`).  Invalid arguments
 * (f64 not 0/1, iters < 0, blocks < 1, threads not a multiple of 32 in
 * 32..1024, NULL or misaligned out) return FF_ERR_INVALID_ARG. */
FF_API ff_status ff_fma_peak(int f64, int64_t iters, int blocks, int threads, void* out, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Status                                                                    */
/* ------------------------------------------------------------------------ */

/* Static string naming a status code. */
FF_API const char* ff_status_string(ff_status st);

/* The CUDA error code kept by the last call of this thread that returned
 * FF_ERR_CUDA (0 if none); returns FF_OK, or FF_ERR_INVALID_ARG for a NULL
 * argument. */
FF_API ff_status ff_last_cuda_error(int* cuda_err);

/* A string identifying this build (used to key autotuning caches). */
FF_API const char* ff_build_id(void);

#ifdef __cplusplus
}
#endif

#endif /* FF_GB300_H */
