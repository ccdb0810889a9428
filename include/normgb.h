/*
 * normgb.h -- C ABI of libnormgb, batched accurate normalization of vectors
 * and quaternions on GB300 (sm_103a), following W. F. Mascarenhas, "Fast and
 * accurate normalization of vectors and quaternions" (arXiv 1606.06508).
 *
 * For each vector x (length n) the library computes, with one correctly
 * rounded IEEE operation per step and no fused multiply-add:
 *   m = max |x_k|; the zero result when every x_k is zero;
 *   x~ = c x with c = 1, sigma_min or sigma_max, the power of two that puts m
 *        into [tau_min, tau_max]                    (Section 2, Eqs. (5)-(10),
 *                                                    Table 2, Algs. 3 and 4);
 *   r~ = sqrt(x~_1^2 + ... + x~_n^2), h = 1/r~;
 *   y_k = h x~_k  (the normalized vector x/|x|) and r = c^{-1} r~  (its norm)
 *                                                   (Algs. 5, 6, 7; Eqs. (1), (2)).
 * n <= 4 follows the printed algorithms (left-to-right sums); n >= 5 sums in
 * a fixed canonical order (256 slots and a halving tree) with
 * tau_max = 2^53 (binary32) or 2^501 (binary64) so that up to 2^20 squares
 * cannot overflow.  Every kernel mapping (thread, warp or block per vector)
 * returns the same bits, and they equal a sequential evaluation of the same
 * steps.
 *
 * Conventions for every entry point:
 *   - Array arguments are addresses the GPU can access, owned by the caller:
 *     device memory, or pinned host memory (cudaHostAlloc, cudaMallocHost,
 *     cudaHostRegister), which the kernels then read and write directly over
 *     the host link (zero-copy: no staging copy; on Grace-Blackwell the
 *     NVLink-C2C link).  Vectors are stored contiguously: a dense batch is
 *     [count][dim] row-major (AoS); a ragged batch packs vector i at
 *     x[offsets[i] .. offsets[i+1]).
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream).  Argument errors are detected on the host before any
 *     work is queued.  Data-dependent errors (bad ragged offsets) never stop a
 *     kernel: the vector is skipped and a status word in the plan is set,
 *     read back by ngb_query_status().
 *   - count == 0 is a no-op returning NGB_OK.  Output arrays may alias the
 *     corresponding input arrays (y == x, grad == g) but must not partly
 *     overlap them.  No exception crosses the ABI; ngb_last_error() gives a
 *     message for the last failing call of the calling thread.
 */
#ifndef NORMGB_H
#define NORMGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ngb_stream_t; /* same type as cudaStream_t */
typedef struct ngb_plan ngb_plan;

typedef enum ngb_status {
  NGB_OK = 0,
  NGB_ERR_INVALID_ARG = 1, /* null pointer, negative size, bad flag combination */
  NGB_ERR_UNSUPPORTED = 2, /* dim or length beyond NGB_MAX_LEN, unsupported dtype */
  NGB_ERR_BAD_OFFSETS = 3, /* ngb_query_status: some ragged vector had bad offsets */
  NGB_ERR_CUDA = 4,        /* a CUDA runtime call failed (see ngb_last_error) */
  NGB_ERR_NO_PLAN = 5      /* a ragged call without a plan, or a plan of another size/dtype */
} ngb_status;

/* flags of the normalize calls */
#define NGB_VECTOR_SEMANTICS 0x1u /* dim == 4: zero input gives y = 0, not the quaternion (0,0,1,0) */
#define NGB_VALIDATE_OFFSETS 0x2u /* ragged: also require offsets[0] == 0 */

/* saved_code values (the factor c applied to x) */
#define NGB_CODE_ONE 0       /* c = 1 */
#define NGB_CODE_SIGMA_MIN 1 /* c = sigma_min: 2^100 (binary32), 2^592 (binary64) */
#define NGB_CODE_SIGMA_MAX 2 /* c = sigma_max: 2^-66 / 2^-514 for n <= 4, 2^-75 / 2^-523 for n >= 5 */
#define NGB_CODE_ZERO 3      /* zero input: zero result, no factor */

#define NGB_MAX_LEN (1 << 20) /* longest vector */

/*
 * normalize_f32 / normalize_f64 -- forward normalization
 * (Eqs. (1)-(2); Algorithms 3-7 of Sections 2-4).
 *
 *   x          input, count vectors (dense: count*dim values; ragged: offsets[count] values)
 *   y          output x/|x|, same layout as x; may equal x; may be NULL to compute norms only
 *   norm       nullable, [count]: r = c^{-1} r~ (+0 for a zero or zero-length vector)
 *   saved_h    nullable, [count]: h = 1/r~ (needed by the backward pass)
 *   saved_code nullable, [count] int8: NGB_CODE_* (needed by the backward pass)
 *   count      number of vectors, 0 <= count < 2^31
 *   dim        > 0: dense batch of vectors of this length (1 .. NGB_MAX_LEN);
 *              0:   ragged batch described by offsets
 *   offsets    ragged only: device int64[count+1], nondecreasing; NULL for dense
 *   plan       ragged only: from ngb_plan_create (count and dtype must match); NULL for dense
 *   flags      NGB_VECTOR_SEMANTICS, NGB_VALIDATE_OFFSETS
 * Dense dim == 4 uses the quaternion zero result (0, 0, 1, 0) of Algorithm 7
 * unless NGB_VECTOR_SEMANTICS is set; ragged vectors always use the vector
 * rule.  A NaN component makes every output of its vector NaN.
 * Ragged x (and y) may be NULL when the batch has no elements
 * (offsets[count] == offsets[0], e.g. a zero-element tensor): the empty
 * vectors are finished as usual, and a vector of positive length in such a
 * call is skipped and reported as bad offsets (nothing is read through the
 * NULL pointer).  A dense call with count > 0 needs x.
 * Returns NGB_OK once the work is queued; NGB_ERR_INVALID_ARG (negative
 * count or dim, unknown flag, offsets given for a dense batch or missing for
 * a ragged one, NULL x for a dense batch), NGB_ERR_UNSUPPORTED (dim >
 * NGB_MAX_LEN, ragged count >= 2^31), NGB_ERR_NO_PLAN, NGB_ERR_CUDA.
 */
ngb_status normalize_f32(const float* x, float* y, float* norm, float* saved_h, int8_t* saved_code, int64_t count,
                         int32_t dim, const int64_t* offsets, ngb_plan* plan, uint32_t flags, ngb_stream_t stream);
ngb_status normalize_f64(const double* x, double* y, double* norm, double* saved_h, int8_t* saved_code,
                         int64_t count, int32_t dim, const int64_t* offsets, ngb_plan* plan, uint32_t flags,
                         ngb_stream_t stream);

/*
 * normalize_backward_f32 / _f64 -- vector-Jacobian product of y = x/|x|
 * (the derivative of Eq. (1); the paper has no backward pass):
 *   grad = (g - y (y . g)) / |x|, evaluated as dot = y . g (left to right for
 *   n <= 4, the canonical order for n >= 5), grad_k = ((g_k - y_k dot) h) c,
 * from the forward's y, saved_h and saved_code, so x is not read again.
 * grad = +0 for a zero input vector.  grad may equal g.  Same layout, count,
 * dim, offsets and plan rules as the forward call.  saved_h and saved_code
 * are required when count > 0; y, g and grad are required for a dense batch
 * and, for a ragged batch, may be NULL only when it has no elements (as for
 * the forward call: vectors of positive length are then skipped and reported).
 */
ngb_status normalize_backward_f32(const float* y, const float* g, const float* saved_h, const int8_t* saved_code,
                                  float* grad, int64_t count, int32_t dim, const int64_t* offsets, ngb_plan* plan,
                                  uint32_t flags, ngb_stream_t stream);
ngb_status normalize_backward_f64(const double* y, const double* g, const double* saved_h,
                                  const int8_t* saved_code, double* grad, int64_t count, int32_t dim,
                                  const int64_t* offsets, ngb_plan* plan, uint32_t flags, ngb_stream_t stream);

/*
 * Ragged plans.  A plan holds the device work lists (12 bytes per vector in
 * binary32, 20 in binary64, which has two more length classes, plus
 * a few counters) for ragged batches of exactly `count` vectors of one dtype
 * (dtype_bytes 4 or 8), the thread/warp/block mapping, and the CUDA graphs
 * that replay the two launches of a call.  It is bound to count and dtype,
 * not to the contents of the offsets, which may change between calls.
 *   capacity    number of elements in the caller's x / y / g buffers, or 0 if
 *               unknown; when > 0, a vector reaching past it is skipped and
 *               reported as bad offsets instead of being read.
 * ngb_plan_create allocates device memory (cudaMalloc) on the current device
 * and synchronizes nothing; ngb_plan_destroy frees it (synchronizing the device).
 * A plan must not be used by two streams at once.
 */
ngb_status ngb_plan_create(ngb_plan** out, int64_t count, int32_t dtype_bytes, int64_t capacity);
ngb_status ngb_plan_destroy(ngb_plan* plan);

/* The mapping: vectors with n <= thread_max (4..16) go one per thread, those
 * with n <= warp_max (thread_max..NGB_MAX_LEN) one per warp, longer ones one
 * per block of block_threads (128 or 256) threads; grid_blocks persistent
 * blocks (0: one full wave).  Default 8, 8192, 256, 0.  Results do not depend
 * on it. */
ngb_status ngb_plan_set_mapping(ngb_plan* plan, int32_t thread_max, int32_t warp_max, int32_t block_threads,
                                int32_t grid_blocks);
ngb_status ngb_plan_get_mapping(const ngb_plan* plan, int32_t* thread_max, int32_t* warp_max,
                                int32_t* block_threads, int32_t* grid_blocks);

/* Autotuner: times the candidate mappings on these offsets (device
 * int64[count+1]) with CUDA events, using a scratch buffer of offsets[count]
 * elements it allocates and frees, and keeps the fastest.  With a non-NULL
 * cache_path the choice is read from / appended to that text file, keyed by
 * GPU name, dtype, count, element total and a length histogram.
 * Synchronizes the stream. */
ngb_status ngb_plan_autotune(ngb_plan* plan, const int64_t* offsets, const char* cache_path, ngb_stream_t stream);

/* Use (1) or stop using (0) CUDA-graph replay for this plan's calls.
 * On by default.  Calls on a stream that is itself being captured launch
 * directly. */
ngb_status ngb_plan_set_graphs(ngb_plan* plan, int32_t enable);

/* Synchronizes `stream`, then reports and clears the plan's status word:
 * NGB_ERR_BAD_OFFSETS if a call since the last query skipped a vector with
 * negative length, length > NGB_MAX_LEN, an end beyond `capacity`, or (with
 * NGB_VALIDATE_OFFSETS) offsets[0] != 0. */
ngb_status ngb_query_status(ngb_plan* plan, ngb_stream_t stream);

/* The opt-in bulk-copy path for binary32 quaternions: with the environment
 * variable NGB_QUAT_BULK set to "1" when the library first normalizes dense
 * binary32 quaternions, calls on 16-byte aligned device memory stage the
 * input through shared memory with bulk copies (cp.async.bulk) instead of
 * registers; same results, measured slower on GB300, so off by default.
 * Writes the path's state on the current device to *state: bit 0 once its
 * kernel has run in this process, bit 1 if one of its bounded waits gave up
 * (never expected; the outputs of the tiles it did not reach are then not
 * written).  Synchronous (a device-to-host copy). */
ngb_status ngb_quat_bulk_state(uint32_t* state);

/*
 * normalize_to_rotation_f32 / _f64 -- Section 4: normalize quaternions
 * q = (q1, q2, q3, q4) (scalar part q4) with Algorithm 7 and write the
 * rotation matrix of the unit quaternion, row-major, 9 values per quaternion:
 *   [1-2(q2^2+q3^2)  2(q1q2-q3q4)    2(q1q3+q2q4)  ]
 *   [2(q1q2+q3q4)    1-2(q1^2+q3^2)  2(q2q3-q1q4)  ]
 *   [2(q1q3-q2q4)    2(q2q3+q1q4)    1-2(q1^2+q2^2)]
 * (the two diagonal entries printed with 2 q3^2 and 2 q2^2 are read as the
 * unit-norm form of the general matrix).  q: [count][4]; R: [count][9];
 * norm nullable [count].  The zero quaternion gives q^ = (0,0,1,0).
 */
ngb_status normalize_to_rotation_f32(const float* q, float* R, float* norm, int64_t count, ngb_stream_t stream);
ngb_status normalize_to_rotation_f64(const double* q, double* R, double* norm, int64_t count, ngb_stream_t stream);

/* Measurement aids (not the method): a streaming device copy of `bytes`
 * bytes, the bandwidth ceiling for the same traffic; and the naive
 * normalization y = x / sqrt(sum x_k^2) without scaling (it overflows and
 * underflows), the baseline of Table 4, for dim 2..4. */
ngb_status ngb_copy(void* dst, const void* src, int64_t bytes, ngb_stream_t stream);
ngb_status naive_normalize_f32(const float* x, float* y, int64_t count, int32_t dim, ngb_stream_t stream);
ngb_status naive_normalize_f64(const double* x, double* y, int64_t count, int32_t dim, ngb_stream_t stream);

/* The quotient algorithms the paper compares its method with (Section 1,
 * Algorithms 1 and 2), for three components; not the method, built to
 * measure the paper's Table 3 ratio time(quotient) / time(scaling).
 * alg = 1: m = max |x_k| (zero: r = 0, y = x); t_k = x_k / m; r = m sqrt(t1^2 +
 *          t2^2 + t3^2); y_k = x_k / r (the input components divided by r).
 * alg = 2: pivot p = the component of largest magnitude, in the printed
 *          branch order; q = (other components) / x_p; h = sqrt(1 + q1^2 + q2^2);
 *          r = |x_p| h; y_p = sign(x_p) / h, other y = q s; the zero return
 *          when x1 = x3 = 0 (so a NaN input gives NaN outputs).
 * x, y: [count][3] device arrays owned by the caller (y may alias x); norm:
 * [count] device array or NULL.  Every step is one correctly rounded IEEE
 * operation.  Errors: NGB_ERR_INVALID_ARG for count < 0, alg not 1 or 2, or a
 * null x or y; NGB_ERR_CUDA for a launch failure. */
ngb_status quotient_normalize3_f32(const float* x, float* y, float* norm, int64_t count, int32_t alg,
                                   ngb_stream_t stream);
ngb_status quotient_normalize3_f64(const double* x, double* y, double* norm, int64_t count, int32_t alg,
                                   ngb_stream_t stream);

/* Measurement aid (not the method): the binary64 pipe's throughput.  Launches
 * `blocks` blocks of 256 threads; each thread runs 4 independent chains of
 * `iters` steps a <- RN(RN(a * b) + c), two FP64 instructions per step, and
 * writes one double to out[blocks * 256] (device memory owned by the caller).
 * *fp64_ops (host, nullable) receives the number of FP64 operations issued;
 * the caller times the launch on `stream`.  Errors: NGB_ERR_INVALID_ARG for a
 * null out or non-positive sizes, NGB_ERR_CUDA for a launch failure. */
ngb_status ngb_fp64_probe(double* out, int32_t blocks, int32_t iters, int64_t* fp64_ops, ngb_stream_t stream);

/*
 * ngb_shard_range -- one process per GPU, every vector independent: the
 * contiguous vectors [*begin, *end) that rank `rank` of `world` normalizes,
 * with no data exchanged between ranks.  Dense batch (offsets == NULL):
 * split by vector count, begin = floor(count rank / world).  Ragged batch:
 * offsets is a HOST int64[count + 1] array (nondecreasing); the split
 * balances the element count: rank r starts at the first vector whose start
 * offset is at least offsets[0] + floor(total r / world), total =
 * offsets[count] - offsets[0], so each shard's element count is within one
 * vector's length of total / world.  The ranges of ranks 0 .. world-1 are
 * disjoint and cover [0, count).  Host-only; no CUDA call.  Errors:
 * NGB_ERR_INVALID_ARG for a NULL begin or end, count < 0, world < 1 or rank
 * outside [0, world).
 */
ngb_status ngb_shard_range(const int64_t* offsets, int64_t count, int32_t world, int32_t rank, int64_t* begin,
                           int64_t* end);

/* Largest batch accepted by normalize_ragged_f32_noalloc. */
#define NGB_NOALLOC_MAX_COUNT 262144

/*
 * normalize_ragged_f32_noalloc -- the ragged binary32 forward pass of
 * normalize_f32 (dim == 0) for callers that must not allocate device memory.
 * The paper has no counterpart: it is a deployment variant of the library.
 * Some callers cannot call cudaMalloc: code running under another
 * framework's memory pool (a direct allocation would bypass the pool or fail
 * because the pool has already reserved the device memory), latency-bound
 * loops where an allocation could synchronize the device, and plugins whose
 * host forbids them to allocate.  They pass inputs and outputs only.
 *
 * The work lists that a plan would allocate live instead in one file-scope
 * device array of (8 + 3 * NGB_NOALLOC_MAX_COUNT) 32-bit words (about 3 MiB),
 * which every device that loads the library holds until the process exits.
 * count > NGB_NOALLOC_MAX_COUNT returns NGB_ERR_UNSUPPORTED (no work queued).
 * The first call on a device looks up the device address of that array (with
 * that device current); make that first call before any stream capture.
 * Every call shares the array and clears its counters on `stream` before
 * use, so calls that overlap on the GPU (two streams, or two threads with
 * different streams) race and must be serialized by the caller.  Vectors
 * with a negative length, a length above NGB_MAX_LEN, a negative start or
 * (with NGB_VALIDATE_OFFSETS) offsets[0] != 0 are skipped, and nothing
 * reports that they were: there is no plan status word to read.  An end
 * offset past the caller's x buffer is NOT detected on this path (there is no
 * capacity argument); the caller must pass offsets that stay inside x.  x and
 * y may be NULL for a batch without elements, as for normalize_f32.  Results
 * are bit-identical to normalize_f32 with a plan.  No cudaMalloc, cudaFree
 * or allocating library routine is called.
 * x, y, norm, saved_h, saved_code, count, offsets: as normalize_f32 (dim == 0);
 * flags: NGB_VALIDATE_OFFSETS or 0.
 */
ngb_status normalize_ragged_f32_noalloc(const float* x, float* y, float* norm, float* saved_h, int8_t* saved_code,
                                        int64_t count, const int64_t* offsets, uint32_t flags, ngb_stream_t stream);

/* Message of the last failing call on this thread ("" if none). */
const char* ngb_last_error(void);
/* Library version string. */
const char* ngb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NORMGB_H */
