/*
 * wsfft -- multidimensional complex-to-complex FFT for sm_103a GPUs.
 *
 * The operation is the k-superstep multidimensional FFT of "Wafer-Scale Fast
 * Fourier Transforms" (Orenes-Vera et al.): for a rank-k array of complex
 * numbers, one superstep per axis applies a batch of 1D Cooley-Tukey FFTs
 * along that axis (Section 1; Section 2.1, pencil decomposition; Section 4.1,
 * pencil computation).  Between supersteps the paper redistributes the data
 * over its processor mesh (Section 4.3); here that redistribution is done on
 * the chip, inside the kernels' strided loads and stores.
 *
 * Definition (Section 1, with the sign numpy uses; numpy is the paper's
 * validator, Section 4.1):
 *
 *   forward:  X[k] = sum_j x[j] exp(-2 pi i sum_d j_d k_d / n_d)
 *   inverse:  x[j] = s * sum_k X[k] exp(+2 pi i sum_d j_d k_d / n_d)
 *
 * where s depends on the normalisation (wsfft_plan_set_norm).
 *
 * Conventions shared by every entry point:
 *  - Layout: row-major; dims[rank-1] is the contiguous axis (Section 1:
 *    element (i,j,k) is element k of pencil (i,j)).  A batch of independent
 *    transforms is the outermost dimension, with stride prod(dims).
 *  - Complex numbers are interleaved (re, im): WSFFT_C32 = two float32 (8 B),
 *    WSFFT_C16F = two IEEE float16 (4 B), WSFFT_C16BF = two bfloat16 (4 B).
 *    Reduced-precision storage is computed in float32 with float32 twiddles
 *    and rounded to the storage type (round-to-nearest-even) at the end of
 *    each pass (Section 4.1 offers FP16 and FP32 storage).
 *  - Sizes: every axis a power of two (Section 4.4: power-of-two sizes only);
 *    axes up to 4096 for rank 2 and 3, up to 2^24 for rank 1.  Other sizes
 *    return WSFFT_ERR_INVALID_SIZE.
 *  - Pointers passed to execute are device pointers (unless named host_*),
 *    owned by the caller, 16-byte aligned, and must stay valid until the
 *    enqueued work completes.  in == out (in place) is allowed; otherwise in
 *    and out must not overlap (a partial overlap of the two arrays returns
 *    WSFFT_ERR_INVALID_ARG).  `in` is never written when in != out.
 *  - Streams are cudaStream_t values passed as wsfft_stream (NULL = the legacy
 *    default stream).  Execute calls are asynchronous on that stream.  The
 *    one-launch-per-superstep kernels of arrays up to 2 GiB are launched with
 *    programmatic stream serialization and let the next kernel on the stream
 *    begin launching early; work the caller enqueues afterwards is ordered
 *    as usual, except a kernel the caller itself launches with that attribute,
 *    which must wait for its predecessor (griddepcontrol.wait) before reading
 *    the output.
 *  - Every function returns a wsfft_status.  No other error state is kept,
 *    except the per-plan device status word, which a device-side timeout
 *    sets; it is reported by wsfft_plan_sync_status.
 *  - A plan belongs to the CUDA device that was current when it was created
 *    and must be used with that device current.  Plans are not thread-safe:
 *    do not call execute on one plan from two host threads at once.
 */
#ifndef WSFFT_H_
#define WSFFT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wsfft_plan_s *wsfft_plan;   /* opaque, owned by the library */
typedef struct CUstream_st *wsfft_stream;  /* same type as cudaStream_t */

typedef enum {
    WSFFT_C32 = 0,   /* complex64: float32 re, float32 im */
    WSFFT_C16F = 1,  /* float16 re, float16 im */
    WSFFT_C16BF = 2  /* bfloat16 re, bfloat16 im */
} wsfft_dtype;

typedef enum {
    WSFFT_FORWARD = -1, /* exponent sign -1 */
    WSFFT_INVERSE = 1   /* exponent sign +1 (conjugated roots, Section 4.2) */
} wsfft_direction;

typedef enum {
    /* Section 4.2: the inverse multiplies the result of each compute stage by
     * 1/n of that stage's axis, 1/N in total; the forward is unscaled. */
    WSFFT_NORM_PAPER = 0,
    /* never scaled: the inverse is then the adjoint of the forward */
    WSFFT_NORM_NONE = 1,
    /* each superstep scaled by 1/sqrt(n_d), both directions (unitary); the
     * default for reduced-precision storage, which keeps values in range */
    WSFFT_NORM_ORTHO = 2,
    /* the forward scaled by 1/n_d per superstep, the inverse unscaled: the
     * adjoint of an inverse under WSFFT_NORM_PAPER */
    WSFFT_NORM_FORWARD = 3
} wsfft_norm;

typedef enum {
    /* spectral data in natural row-major order, the same layout as the
     * spatial data (numpy's fftn) */
    WSFFT_LAYOUT_NATURAL = 0,
    /* spectral data with the last two axes swapped: a rank-3 n0 x n1 x n2
     * spectrum is stored as [n0][n2][n1], a rank-2 n0 x n1 one as [n1][n0].
     * The middle axis ends contiguous, as on the wafer after its two
     * transposes (Section 4.2: each PE ends holding a pencil of that axis);
     * the two axes the wafer spreads over its mesh keep the input's order */
    WSFFT_LAYOUT_SWAPPED = 1,
    /* rank 3 only: the wafer's own arrangement of the spectrum, [n2][n0][n1]
     * -- X[k0][k1][k2] at k2*n0*n1 + k0*n1 + k1.  Section 4.2 transforms z,
     * swaps x and z within mesh rows, transforms x, swaps x and y within
     * mesh columns, transforms y; with the PEs numbered the way the input
     * is (x outer), the spectrum ends on PE (k2, k0) holding the k1 pencil */
    WSFFT_LAYOUT_WAFER = 2
} wsfft_layout;

typedef enum {
    WSFFT_SUCCESS = 0,
    WSFFT_ERR_INVALID_ARG = -1,   /* null/misaligned pointer, bad enum, bad rank */
    WSFFT_ERR_INVALID_SIZE = -2,  /* non-power-of-two or out-of-range axis */
    WSFFT_ERR_UNSUPPORTED = -3,   /* valid request the library does not handle */
    WSFFT_ERR_ALLOC = -4,         /* device or host allocation failed */
    WSFFT_ERR_CUDA = -5,          /* a CUDA runtime call failed */
    WSFFT_ERR_DEVICE_TIMEOUT = -6 /* a bounded device-side wait ran out */
} wsfft_status;

/* Create a plan for `batch` independent rank-`rank` transforms of shape
 * dims[0..rank-1] (row-major, dims[rank-1] contiguous).
 *   plan      out: the new plan (NULL on failure)
 *   dims      host array of `rank` axis lengths, each a power of two
 *   rank      1, 2 or 3
 *   dtype     a wsfft_dtype; direction a wsfft_direction
 *   batch     >= 1
 * Builds the pass schedule and the twiddle tables (computed in FP64 on the
 * host, rounded to FP32, uploaded once) on the current device.  Default
 * normalisation: WSFFT_NORM_PAPER for WSFFT_C32, WSFFT_NORM_ORTHO otherwise.
 * Errors: INVALID_ARG, INVALID_SIZE, ALLOC, CUDA.  Sections 1, 4.1, 4.2. */
int wsfft_plan_create(wsfft_plan *plan, const int64_t *dims, int rank, int dtype,
                      int direction, int64_t batch);

/* Create a plan for one superstep: `batch` x `inner` independent 1D
 * transforms of length n along an axis whose consecutive elements are
 * `inner` elements apart -- the array is [batch][n][inner] (row-major) and
 * pencil (b, i) is its elements (b, 0..n-1, i).  inner = 1 is a batch of
 * contiguous transforms.  This is the superstep of Section 4.1 on its own,
 * for arrays whose other axes are transformed elsewhere (the x superstep of
 * a slab-distributed 3D transform runs on each GPU's y-slab with it).
 *   n: power of two, 2..4096; inner: power of two >= 1; batch >= 1.
 * Normalisation: scale 1/n on the inverse under WSFFT_NORM_PAPER (the
 * default for WSFFT_C32), 1/sqrt(n) both ways under WSFFT_NORM_ORTHO (the
 * default for the 16-bit types); wsfft_plan_set_norm changes it.  Layouts
 * other than natural return UNSUPPORTED.  Executes through wsfft_execute /
 * wsfft_execute_host like any plan.
 * Errors: INVALID_ARG, INVALID_SIZE, ALLOC, CUDA. */
int wsfft_plan_create_axis(wsfft_plan *plan, int64_t n, int64_t inner, int dtype,
                           int direction, int64_t batch);

/* out[b][a][c] = in[a][b][c] for a < A, b < B, c < C elements of `dtype`:
 * swap the two outer axes of a row-major [A][B][C] array, moving each run of
 * C elements whole.  The redistribution of a slab-distributed transform
 * (Section 2.1, data distribution; Section 4.3, redistribution between
 * supersteps): before an all-to-all a rank's [rows][destination][share]
 * becomes [destination][rows][share], one contiguous send block per rank,
 * and after the inverse's all-to-all the received [source][rows][share]
 * goes back to row order.  in and out: device pointers, must not overlap;
 * asynchronous on `stream`.  Moves 16-byte vectors when C's byte length and
 * both pointers are multiples of 16.
 * Errors: INVALID_ARG (null, overlapping, bad dtype or size), UNSUPPORTED
 * (more than 2^31 - 1 runs of c elements), CUDA. */
int wsfft_transpose_outer(const void *in, void *out, int64_t A, int64_t B, int64_t C,
                          int dtype, wsfft_stream stream);

/* Change the normalisation (a wsfft_norm).  Section 4.2.
 * Errors: INVALID_ARG. */
int wsfft_plan_set_norm(wsfft_plan plan, int norm);

/* Choose the layout of the spectral side (a wsfft_layout): the forward
 * writes its output in it, the inverse reads its input in it; the spatial
 * side stays natural.  WSFFT_LAYOUT_SWAPPED needs rank 2 or 3 with both of
 * the last two axes in [64, 4096]; it runs the first superstep with a
 * transposing store into a plan-owned workspace (one array, at most 4 GiB of
 * transforms at a time), so it moves the same bytes as the natural layout
 * (three trips for rank 3, two for rank 2) and never uses the fused
 * schedules of wsfft_plan_set_engine.  On this hardware the layouts cost
 * about the same (512^3 complex64: 0.95-0.97 ms per transform, the wafer
 * order fastest: its first axis is transformed at the short stride); the
 * swapped one serves callers that work on a spectrum with the middle axis
 * in memory.  WSFFT_LAYOUT_WAFER needs rank
 * 3 with every axis in [64, 4096]; its forward runs z with the transposing
 * store (natural -> [n2][n0][n1], into the workspace), then y (now
 * contiguous) and x; its inverse runs y and then x with the transposing
 * store and z last -- again three trips.  Resets pass-shape choices
 * (wsfft_plan_set_pass_variant).
 * Errors: INVALID_ARG (bad enum), UNSUPPORTED (rank or sizes, ragged plan),
 * ALLOC. */
int wsfft_plan_set_layout(wsfft_plan plan, int layout);

/* Enqueue the transform of `batch` arrays from `in` to `out` on `stream`.
 * in/out: device pointers to batch*prod(dims) elements of the plan's dtype.
 * Section 1 (supersteps), Section 4.2 (3D sequence), Section 4.3
 * (redistribution, here fused into the kernels' loads and stores).
 * Errors: INVALID_ARG (null or misaligned pointer), CUDA (launch failure).
 * A device-side timeout is not reported here (the call does not wait for
 * the device); wsfft_plan_sync_status reports it.  The call only enqueues
 * work on `stream` (kernel launches, and a counter reset for the persistent
 * schedules) and allocates nothing (tables and workspace belong to the
 * plan), so it may be captured into a CUDA graph and the graph replayed on
 * new data in the same buffers; the plan must outlive the graph. */
int wsfft_execute(wsfft_plan plan, const void *in, void *out, wsfft_stream stream);

/* Same transform with HOST buffers: copies host_in to a plan-owned device
 * buffer, transforms, copies back to host_out, and waits for the stream.
 * host_in/host_out should be page-locked for full copy speed; they may be
 * the same buffer.  For rank-3 plans with one launch per superstep the
 * copies overlap the compute: slab chunks come in on a second stream (owned
 * by the plan) and are transformed along the last axis as they arrive, the
 * first axis is transformed over the whole array, and the middle axis slab
 * chunk by slab chunk, each chunk copied back on a third stream (also the
 * plan's) as soon as it is done; with batch > 1 the next transform's copies
 * in run while the previous one's go out (the result equals wsfft_execute's
 * up to rounding: the axes are taken in another order).  The first call
 * allocates the device buffer
 * (batch * prod(dims) elements).  Errors: as wsfft_execute, plus ALLOC. */
int wsfft_execute_host(wsfft_plan plan, const void *host_in, void *host_out,
                       wsfft_stream stream);

/* Release the plan and every device allocation it owns.  Waits first for
 * the plan's own work: every stream the plan was executed on, up to its last
 * execute there (executes enqueued while a stream was being captured into a
 * graph are the caller's to wait for), and the plan's internal streams; other
 * work on the device is not waited for.  NULL is accepted.  Errors: CUDA. */
int wsfft_destroy(wsfft_plan plan);

/* Plan for `count` independent rank-3 transforms of uneven shapes
 * dims[3*i .. 3*i+2] (each axis a power of two, 32..256), executed by one
 * persistent launch that pulls (instance, superstep, tile) tasks from a
 * queue; a superstep's tiles wait (bounded) until the previous superstep of
 * the same instance is complete.  Section 4.4 (more than one pencil per
 * processor) generalised to one thread block per tile.  Normalisation as
 * wsfft_plan_create (PAPER for WSFFT_C32, ORTHO otherwise).  The launch and
 * its table upload can be captured in a CUDA graph (the upload is skipped
 * when the pointers are unchanged).
 * Errors: INVALID_ARG, INVALID_SIZE, ALLOC, CUDA. */
int wsfft_plan_create_ragged(wsfft_plan *plan, int count, const int64_t *dims,
                             int dtype, int direction);

/* Enqueue a ragged plan: in[i], out[i] are device pointers for instance i
 * (host arrays of `count` pointers, 16-byte aligned; in[i] == out[i]
 * allowed; instances must not overlap).  Errors: as wsfft_execute. */
int wsfft_execute_ragged(wsfft_plan plan, const void *const *in, void *const *out,
                         wsfft_stream stream);

/* Time the kernel variants that apply to this plan on `stream` (with
 * temporary buffers) and keep the fastest; results are cached in the JSON
 * file named by WSFFT_TUNE_CACHE (if set), keyed by device name, SM count,
 * shape, batch, dtype, direction, normalisation and spectral layout.  For a
 * ragged plan the candidates are the tile shape of each axis length that
 * occurs and the queue lag (wsfft_plan_set_ragged_variant), the key holds
 * the sorted multiset of instance shapes, and a ragged plan created later
 * with the same key takes the cached choice.  A cached entry that does not
 * describe a schedule this build can launch (an unknown schedule, values out
 * of range, a kernel shape that is not instantiated) is ignored: plan
 * creation keeps the default schedule and wsfft_autotune times afresh.
 * Errors: ALLOC, CUDA. */
int wsfft_autotune(wsfft_plan plan, wsfft_stream stream);

/* Ragged plans: choose the tile shape per axis length and the queue lag.
 * Bit k of shape_select (k = log2(N) - 5, N in 32..256) selects the second
 * tile shape for axes of length N (values per thread: 16 instead of 8 for
 * N <= 64, 8 instead of 16 for N >= 128; a tile is always 256 threads);
 * `lag` L puts the y tiles of instance s - L and the x tiles of instance
 * s - 2L after the z tiles of instance s in the queue (1 = the default).
 * Waits for the plan's own work, then rebuilds its tile queue.  Used by
 * wsfft_autotune.  Errors: INVALID_ARG (shape_select outside 0..15, lag
 * outside 1..64), UNSUPPORTED (not a ragged plan), ALLOC, CUDA. */
int wsfft_plan_set_ragged_variant(wsfft_plan plan, int shape_select, int lag);

/* Choose the kernel shape of pass `pass` (0-based, in launch order) of this
 * plan: `values_per_thread` complex values per thread (the radix of the
 * register stages, 8, 16 or 32) and `tile` pencils per thread block; 0 and 0
 * restore the default.  Tile codes 1000 + W select the pencil-pair strided
 * kernel with W pencils per block, 3000 + W the same tile with the pair held
 * in split form (real parts together, imaginary parts together) so that its
 * butterflies run as packed FP32x2 instructions; tile code 2000 selects the
 * tensor-core contiguous superstep (16-bit storage, N = 512; the
 * values-per-thread argument is then ignored).  Used by the autotuner.
 * Errors: INVALID_ARG, UNSUPPORTED (that shape is not built for this pass).
 * A shape that needs whole tiles (either pencil-pair kernel) on a pass whose
 * pencil count or stride is not a multiple of its tile makes wsfft_execute
 * return CUDA without launching. */
int wsfft_plan_set_pass_variant(wsfft_plan plan, int pass, int values_per_thread, int tile);

/* Choose the schedule of a rank-3 transform n0 x n x n (n in {128, 256, 512,
 * 1024}, any n0; the pipelined engine needs n0 == n):
 *   0 (default): one launch per superstep (three trips through HBM);
 *   4 (n in {256, 512}): two trips through HBM -- one thread-block cluster
 *      per n x n slab runs its z superstep, meets at a cluster barrier, and
 *      runs its y superstep on the slab as the z tiles left it in L2; then
 *      one launch runs the outer axis (Sections 4.2-4.3 with the
 *      redistribution between z and y kept inside a cluster).  At 512^3 it
 *      measured slower than mode 0 on GB300 (fused pass 0.70 ms against
 *      0.64 ms for the two launches it replaces), so it is an option;
 *   3 (n <= 512): two trips through HBM with warp-per-pencil
 *      kernels -- a persistent kernel runs the supersteps along the two inner
 *      axes slab by slab, re-reading each slab from L2, then one launch runs
 *      the outer axis;
 *   1: the same two trips with one-tile-per-block style tiles;
 *   2: the same two trips on the pipelined engine (one producer warp
 *      streaming tiles into shared memory with bulk asynchronous copies).
 * wsfft_autotune times the modes and keeps the fastest.  A mode a shape does not support falls back to one launch per superstep.
 * Other shapes ignore the setting.  The autotuner uses it.
 * Errors: INVALID_ARG. */
int wsfft_plan_set_engine(wsfft_plan plan, int mode);

/* Testing aid for the bounded device-side waits of the persistent engine
 * (used by rank-3 cube plans): withhold != 0 drops the completion signal of
 * one tile in later executes, so the tiles that wait for it run out their
 * budget of timeout_ns nanoseconds per wait; the execute then finishes
 * early, nothing faults or hangs, and wsfft_plan_sync_status reports
 * WSFFT_ERR_DEVICE_TIMEOUT.  withhold = 0 restores normal operation (the
 * budget stays timeout_ns; the default is one second).
 * Errors: INVALID_ARG, UNSUPPORTED (the plan has no waits). */
int wsfft_plan_set_wait_test(wsfft_plan plan, int withhold, int64_t timeout_ns);

/* Synchronise `stream`, then return and clear the plan's device status word
 * (WSFFT_SUCCESS or WSFFT_ERR_DEVICE_TIMEOUT).  Errors: CUDA. */
int wsfft_plan_sync_status(wsfft_plan plan, wsfft_stream stream);

/* Number of passes over the array one execute makes, and the minimum number
 * of bytes one execute reads plus writes in HBM for that schedule. */
int wsfft_plan_passes(wsfft_plan plan, int *passes, int64_t *bytes_per_execute);

/* Per-launch timing (the paper times compute and communication phases
 * separately, Section 5.2).  capacity > 0 makes every later kernel launch of
 * this plan record a pair of CUDA events on the execute stream, for up to
 * `capacity` launches; 0 turns recording off and frees the events.
 * Errors: INVALID_ARG, ALLOC, CUDA. */
int wsfft_plan_profile(wsfft_plan plan, int capacity);

/* Wait for the recorded launches, write the elapsed milliseconds of each
 * (in launch order, at most `capacity` values) to ms[], the number of
 * launches recorded to *count, and start a new recording.  ms may be NULL
 * to only reset.  Errors: INVALID_ARG, CUDA. */
int wsfft_plan_launch_times(wsfft_plan plan, float *ms, int capacity, int *count);

/* Allocation-free n^3 transform (the paper has no counterpart: it is an
 * interface for callers that cannot allocate device memory -- code that runs
 * while a CUDA graph is being captured, code whose device memory is owned by
 * another framework's allocator, or programs that reserve all device memory
 * up front).  Computes the same transform as a complex64 plan of dims
 * (n, n, n), `batch` transforms, in `direction`, with WSFFT_NORM_PAPER, from
 * device pointer `in` to device pointer `out` (16-byte aligned; in == out
 * allowed) on `stream`, and calls no cudaMalloc or cudaFree: its scratch
 * counters (16 KiB) and twiddle tables (16 KiB) live in static device arrays
 * that every GPU loading the library keeps until the process exits.
 *   n: 128, 256 or 512; batch * n <= 4096.  Larger sizes return
 *   WSFFT_ERR_INVALID_SIZE; null or misaligned pointers, in and out that
 *   share bytes without being equal, and bad directions return
 *   WSFFT_ERR_INVALID_ARG.
 * The first call on each device does that device's set-up (table upload on
 * `stream`, which it then synchronises, symbol lookup, occupancy query) with
 * the device current.  All calls on a device share the scratch array, which keeps the last call's contents (each
 * call clears the counters it uses): calls that overlap on the GPU race and
 * must not be made.  A bounded device-side wait that runs out leaves that
 * call's output incomplete and is reported only by
 * wsfft_noalloc_sync_status.
 * Errors: INVALID_ARG, INVALID_SIZE, UNSUPPORTED, CUDA. */
int wsfft_execute_cube_noalloc(const void *in, void *out, int64_t n, int64_t batch,
                               int direction, wsfft_stream stream);

/* Report and clear the status word of wsfft_execute_cube_noalloc on the
 * current device: synchronises `stream`, then returns WSFFT_ERR_DEVICE_TIMEOUT
 * if a bounded device-side wait of any call since the last report ran out
 * (that call's output is incomplete), else WSFFT_SUCCESS (also when no call
 * has run on this device).  Allocates nothing.  Like the entry point it
 * reports on, it has no counterpart in the paper.  Errors: CUDA, UNSUPPORTED
 * (device index beyond the library's table of devices). */
int wsfft_noalloc_sync_status(wsfft_stream stream);

/* Static text for a status code. */
const char *wsfft_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* WSFFT_H_ */
