/*
 * pac.h — permutation-avoiding FFT convolution on one GB300 (sm_103a).
 *
 * The library computes the d-dimensional circular convolution
 *
 *     y = F_h(x) = DFT^-1( DFT(h) o DFT(x) ),   n_1 x ... x n_d,  d in {1,2,3}
 *
 * (the convolution operator of the paper's Section 2, eq. "convolution";
 * 2-D form Section 3; d-D form Section 4) without ever executing an
 * index-reversal permutation: the forward transform is the decimation-in-
 * frequency product A^T (natural order in, index-reversed order out), the
 * filter spectrum A^T h is computed once and kept on the device, and the
 * inverse is the conjugate decimation-in-time product conj(A) (reversed in,
 * natural out), Eq. (35) in 1-D, Eq. (80) in 2-D and the d-D form of
 * Section 4.1.  The spectrum is stored in the order in which the kernel
 * that multiplies by it reads it (a fixed rearrangement of the
 * index-reversed order, applied once when the spectrum is made), so the
 * convolution itself never permutes anything.  Per axis, n = r^t or a
 * mixed-radix product (Section 7.1).
 *
 * Conventions shared by every entry point:
 *  - Arrays are complex, interleaved (re, im), row-major with the last index
 *    fastest (the row-major vec of Section 4), dense, 16-byte aligned.
 *    dtype PAC_C64 = complex float (8 bytes/element), PAC_C128 = complex
 *    double (16 bytes/element), PAC_C128_DF = complex double arrays
 *    computed in double-float arithmetic (see pac_plan_create).
 *  - Pointers named *_dev are device pointers on the current CUDA device;
 *    pointers named *_host are host pointers (pinned memory gives the fastest
 *    copies).  The caller owns every array it passes; the library owns plans,
 *    queues, twiddle/index tables, filter spectra and its staging buffers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that take a stream only enqueue work; they do not
 *    synchronise unless stated.
 *  - Every function returns a pac_status (0 = PAC_OK).  Nothing throws and no
 *    kernel traps.  pac_last_error() returns a thread-local message for the
 *    last failing call of the calling thread.  Asynchronous device faults
 *    surface at a later call or synchronisation as PAC_ERR_CUDA.
 *  - Forward sign: w_n = exp(-2 pi i / n) (Section 2).  The inverse applies
 *    1/N once (N = n_1 ... n_d), folded into the stored filter spectrum.
 */
#ifndef PAC_H
#define PAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pac_plan_s* pac_plan;   /* opaque, library-owned */
typedef struct pac_queue_s* pac_queue; /* opaque, library-owned */
typedef struct pac_pfa_s* pac_pfa;     /* opaque, library-owned */

typedef enum { PAC_C64 = 0, PAC_C128 = 1, PAC_C128_DF = 2 } pac_dtype;

typedef enum {
    PAC_OK = 0,
    PAC_PENDING = 1,          /* pac_poll: request not finished yet */
    PAC_ERR_ARG = -1,         /* null pointer, bad enum, misaligned pointer */
    PAC_ERR_SIZE = -2,        /* a dim does not fit the radix or stage list, or is too large */
    PAC_ERR_NO_SPECTRUM = -3, /* pac_convolve before pac_filter_spectrum */
    PAC_ERR_NOMEM = -4,       /* device or host allocation failed / over budget */
    PAC_ERR_CUDA = -5,        /* a CUDA runtime call failed */
    PAC_ERR_BUSY = -6,        /* request queue full */
    PAC_ERR_TIMEOUT = -7,     /* a bounded wait gave up */
    PAC_ERR_NOT_FOUND = -8    /* unknown ticket */
} pac_status;

/* ------------------------------------------------------------------ plans */

/*
 * Create a plan for d-D convolutions of shape dims[0] x ... x dims[ndim-1].
 * ndim in {1,2,3}; radix in {0,2,3,4,5,8}.  For radix r != 0 each dim must
 * be a power of the radix's prime p (p = 2 for radix 4 and 8).  The per-axis
 * decimation-in-frequency stage list is [r, r, ..., r] (Section 2.1); when
 * the exponent is not a multiple of log_p r the leftover factor becomes one
 * smaller stage of base p placed last (e.g. 128 with radix 4 -> [4,4,4,2];
 * with radix 8 -> [8,8,2]), the mixed-radix framework of Section 7.1.
 * radix 0 (mixed radix, Section 7.1): each dim is any 2^a 3^b 5^c, with the
 * stage list [4,..,4,(2), 3,..,3, 5,..,5] (the factor 2^a in radix-4 stages,
 * a leftover 2 last, then the 3s and the 5s).  Each run of stages of one
 * base becomes one or more passes; where groups spanning the bases are fewer
 * and each has a compiled kernel (48, 120, 1000 and 6000 points; a whole
 * axis of 6000 is one group), those run instead (PAC_MIXED=0 / 1 / rt in
 * the environment forces one-base groups / groups spanning bases / groups of
 * at most 2048 points in the runtime-radix kernel; PAC_NARROW=1 / 0 forces
 * the narrow tile of the group passes on / off, see pac_tune).  A dim of 1 is allowed
 * (empty stage list).  Builds twiddle tables in FP64, rounds them once to
 * dtype and uploads them to the current device.  On success *out owns device
 * memory until pac_plan_destroy.  Errors: PAC_ERR_ARG, PAC_ERR_SIZE,
 * PAC_ERR_NOMEM, PAC_ERR_CUDA.
 *
 * PAC_C128_DF: the same complex FP64 arrays in and out as PAC_C128 (h, x,
 * y), the same stage groups, but every butterfly, twiddle and product in
 * double-float arithmetic (a value as the unevaluated sum of two FP32
 * numbers, about 48 significant bits) on the FP32 pipes, which GB300 runs at
 * 64 times its FP64 rate; the twiddles are the FP64 tables split once into
 * two FP32 parts.  The relative L2 error stays within the FP64 tolerance
 * (1e-12) for magnitudes within FP32's range (about 1e-38 to 3e38; 48-bit
 * precision down to about 2e-31, gradually less below; smaller than 1e-38
 * flushes to 0).  One-base stage groups only (no plane pass, no groups
 * spanning prime bases); pac_convolve, pac_convolve_host, pac_submit and
 * pac_tune take such plans, the other entry points return PAC_ERR_ARG.
 */
int pac_plan_create(int ndim, const int64_t* dims, int radix, pac_dtype dtype, pac_plan* out);

/*
 * The same from explicit per-axis DIF stage lists, in any order (the
 * mixed-radix framework of Section 7.1: A_rho with rho the list reversed,
 * so stages[0] of an axis acts first, on the full length).  nstages[a]
 * stages for axis a, concatenated in `stages` (host memory, read only
 * during the call).  Each stage is a power of 2, 3 or 5 in [2, 32]; the
 * stages of axis a multiply to dims[a] (nstages[a] = 0 for a dim of 1).
 * The unordered transform (pac_forward_unordered) leaves frequency
 * k = k_1 + s_1 k_2 + s_1 s_2 k_3 + ... at position
 * sum_i k_i prod_{j>i} s_j of each axis.  Stages of one prime base that are
 * adjacent run in one pass; each change of base starts a new pass unless
 * groups spanning bases are formed (the rule of pac_plan_create).  Such
 * plans are not autotuned.  Errors: PAC_ERR_ARG (ndim, null pointers, more
 * than 64 stages), PAC_ERR_SIZE (a stage or product rule broken), as
 * pac_plan_create otherwise.
 */
int pac_plan_create_stages(int ndim, const int64_t* dims, const int* nstages, const int* stages, pac_dtype dtype,
                           pac_plan* out);

/* Release a plan and everything it owns. Waits for the plan's pending work. */
int pac_plan_destroy(pac_plan p);

/*
 * The filter-spectrum step of Algorithm 11: store Hhat = A^T h / N (all axes, with the
 * inverse's 1/N folded in) in plan-owned device memory, in the order the
 * fused forward/product/inverse pass reads it.
 * h_dev is read, not retained.  Synchronises the plan's internal stream.
 * Calling it again replaces the spectrum.
 */
int pac_filter_spectrum(pac_plan p, const void* h_dev);

/*
 * The convolution of Algorithm 11 (permutation-avoiding, Eq. 35/80):
 * y = conj(A)((A^T x) o Hhat).  x_dev and y_dev hold N elements of the plan's
 * dtype; y_dev may equal x_dev (in place).  y_dev is also the working buffer
 * of the intermediate passes.  Asynchronous on `stream`.
 * Errors: PAC_ERR_ARG, PAC_ERR_NO_SPECTRUM, PAC_ERR_CUDA.
 */
int pac_convolve(pac_plan p, const void* x_dev, void* y_dev, void* stream);

/*
 * As pac_convolve, with x and y in HOST memory (pinned for asynchronous
 * copies): copies x to plan-owned device staging, convolves, copies y back,
 * then synchronises `stream`.  The end-to-end form of the call.  For arrays
 * of 64 MiB and more whose first pass is a rows pass of axis 0 with enough
 * tiles (2-D and 3-D plans, 1-D plans of several groups), the copies run in
 * 8 column blocks of that pass on two plan-owned copy streams: block k + 1
 * comes in while the first pass works on block k, and block k goes out
 * while the last pass works on block k + 1 (the plan's device work stays on
 * `stream`, which waits for the copies in through events).  Errors:
 * PAC_ERR_ARG, PAC_ERR_NO_SPECTRUM, PAC_ERR_NOMEM, PAC_ERR_CUDA.
 */
int pac_convolve_host(pac_plan p, const void* x_host, void* y_host, void* stream);

/*
 * Many independent convolutions in one call: plans[i] applied to x_dev[i] ->
 * y_dev[i] for i < count (the batching pattern; the paper has one
 * convolution per call).  When every plan is complex FP32 and every pass has
 * a shape the persistent kernel carries (one-base groups up to 4096 / 2187 /
 * 3125 points, square planes), the whole batch is ONE launch of a persistent
 * kernel: resident CTAs pull the tiles of all instances' passes from a
 * device work list, and each pass of an instance waits (bounded, on device
 * counters) for the pass before it.  Otherwise (or with PAC_BATCH=graph in
 * the environment) the work is merged into one launch per pass level and
 * kernel shape.  Either way the launch sequence is recorded once per
 * distinct batch (plans, x and y pointers) and replayed as a CUDA graph.
 * Plans may repeat.  Each plan needs its spectrum.  Asynchronous on
 * `stream`; calls for the same batch must not overlap on the device (the
 * persistent form keeps its work counters per batch).
 */
int pac_convolve_many(int count, const pac_plan* plans, const void* const* x_dev, void* const* y_dev,
                      void* stream);

/*
 * Kernel launches one pac_convolve_many call over these plans makes (1 for
 * the persistent form, else the merged launches of its captured graph; plus
 * one per N = 1 plan).  Host
 * only; no device work.
 */
int pac_convolve_many_launches(int count, const pac_plan* plans, int* launches);

/* ------------------------------------------------------ prime factor form */

/*
 * Prime factor convolution (Section 7.2) of a 1-D length n = 2^a 3^b 5^c:
 * with the pairwise coprime factors n_1 < ... < n_t (the nonzero prime
 * powers of n, t <= 3),
 *   y = Gamma (conj A_{n_t} x ... x conj A_{n_1})
 *         [((A^T_{n_t} x ... x A^T_{n_1}) Gamma^T h) o ((...) Gamma^T x)] / n,
 * where Gamma^T gathers a length-n vector into the tensor of shape
 * (n_t, ..., n_1) (entry (i_t, ..., i_1) = element i with i = i_q mod n_q,
 * Chinese remainders) and Gamma gathers it back (y[k] = tensor entry
 * (k mod n_t, ..., k mod n_1)).  Three permutations per convolution
 * (Gamma^T h is made once by pac_pfa_filter_spectrum); the bracket is the
 * t-D convolution of a radix-0 plan of that shape.  The result equals
 * pac_convolve of a 1-D plan of length n.
 * pac_pfa_create: errors PAC_ERR_ARG (dtype, null out), PAC_ERR_SIZE (n not
 * 2^a 3^b 5^c or >= 2^31), as pac_plan_create otherwise.  The object owns
 * the inner plan and one n-element scratch array: calls of
 * pac_pfa_convolve on one object must not overlap (one stream, or ordered
 * streams).  pac_pfa_filter_spectrum synchronises the device.
 * pac_pfa_convolve is asynchronous on `stream` (3 + inner launches); y_dev
 * may equal x_dev.  Pointers as pac_convolve.
 */
int pac_pfa_create(int64_t n, pac_dtype dtype, pac_pfa* out);
int pac_pfa_destroy(pac_pfa p);
int pac_pfa_filter_spectrum(pac_pfa p, const void* h_dev);
int pac_pfa_convolve(pac_pfa p, const void* x_dev, void* y_dev, void* stream);
/* t and the tensor shape, padded on the left with 1s to three axes */
int pac_pfa_shape(pac_pfa p, int* t, int64_t* dims);
/* PAC_Q_* keys: NDIM = t, N_TOTAL = n, LAUNCHES_CONVOLVE and DEVICE_BYTES of
 * the whole object, others of the inner plan */
int pac_pfa_query(pac_pfa p, int key, int64_t* value);
/* The inner t-D plan (owned by the object; not to be destroyed by the caller). */
int pac_pfa_plan(pac_pfa p, pac_plan* inner);

/* ----------------------------------------------------------------- serving */

/*
 * A request queue with continuous batching.  Requests (plan, x_dev, y_dev)
 * are admitted in arrival order while (a) fewer than max_inflight are
 * running and (b) the device bytes of running requests (2 * N * elem size
 * each) stay within the admission budget: hbm_budget_bytes, or the device
 * memory cudaMemGetInfo reports free when the queue is created if that is
 * less (a request larger than the budget runs alone); a request that does
 * not fit waits (it is never dropped).  At most two large complex FP64
 * requests (FP64-pipe bound, milliseconds each) run at once
 * (PAC_QUEUE_FP64_LARGE in the environment overrides).  Admitted requests
 * run on a pool of streams so their kernels overlap on the device.  Plans
 * and spectra stay resident; the queue does not own them.  Requests of at
 * most 8 MiB of device bytes are "small": they run on high-priority streams
 * and a quarter of the slots is kept for them, so large requests cannot hold
 * every slot; within each class admission is in arrival order.  Requests
 * run on max_inflight streams: set CUDA_DEVICE_MAX_CONNECTIONS (in the
 * environment, before CUDA starts in the process) to at least max_inflight,
 * else streams share the GPU's hardware work queues (8 by default) and a
 * small request's kernels can wait behind a large request's.
 */
int pac_queue_create(size_t hbm_budget_bytes, int max_inflight, pac_queue* out);

/* Enqueue one request; returns a ticket. PAC_ERR_BUSY when 65536 requests are waiting. */
int pac_submit(pac_queue q, pac_plan p, const void* x_dev, void* y_dev, uint64_t* ticket);

/*
 * Non-blocking completion check.  Returns PAC_OK (done; *latency_us, if not
 * NULL, is submit-to-completion time in microseconds), PAC_PENDING, or an
 * error (PAC_ERR_NOT_FOUND for an unknown or already-reaped ticket, or the
 * request's own failure status).  A finished ticket is reaped by the first
 * poll that returns its final status.
 */
int pac_poll(pac_queue q, uint64_t ticket, double* latency_us);

/* Block until every submitted request has finished (bounded wait: timeout_ms). */
int pac_queue_drain(pac_queue q, int timeout_ms);

/* Drain and free the queue. */
int pac_queue_destroy(pac_queue q);

/* Thread-local message describing the last failing call of this thread. */
const char* pac_last_error(void);

/* --------------------------------------------------------------- test hooks */

/* Per-axis DIF stage list of a plan: radices[0..*count), s_1 first (full length). */
int pac_plan_stages(pac_plan p, int axis, int* radices, int* count);

/*
 * Per-axis index-reversal table of a plan: pos_to_freq[p] = the frequency that
 * the unordered (A^T) output holds at position p along that axis (F = P A^T,
 * Section 2.1; F = P_rho A_rho^T, Section 7.1).  Host copy of dims[axis] entries.
 */
int pac_plan_reverse_table(pac_plan p, int axis, int64_t* pos_to_freq);

/* Unordered forward transform only: xhat = A^T x (all axes), Algorithms 2-4 (uFFT2). */
int pac_forward_unordered(pac_plan p, const void* x_dev, void* xhat_dev, void* stream);

/*
 * Comparator, the standard FFT-based convolution (Algorithm 10): the same
 * stage kernels plus explicit index-reversal permutation passes (Algorithm 1)
 * after the forward transform and before the inverse (FFT2 of Algorithm 5 and
 * iFFT of Algorithm 9), with the filter spectrum kept in natural order.
 * Uses a plan-owned scratch buffer of N elements.  Asynchronous on `stream`.
 */
int pac_convolve_permuted(pac_plan p, const void* x_dev, void* y_dev, void* stream);

/*
 * Ordered DFT with an explicit index-reversal pass, the standard FFT of the
 * paper's comparison: inverse = 0 gives out = F in in natural frequency
 * order (FFT2 of Algorithm 5: the DIF passes A^T, then the permutation P of
 * Algorithm 1); inverse = 1 gives out = F^-1 in = conj(A) P in / N (iFFT of
 * Algorithm 9).  Forward sign w_n = exp(-2 pi i / n).  Uses plan-owned
 * scratch (N elements) and index tables made on first use; in_dev may equal
 * out_dev.  pac_convolve_timed-style timing of its launches: kernel ids 0
 * (DIF pass), 2 (DIT pass), 3 (permutation).  Asynchronous on `stream`.
 */
int pac_fft(pac_plan p, const void* in_dev, void* out_dev, int inverse, void* stream);

/*
 * Profiling form of pac_convolve (which = 0), pac_convolve_permuted
 * (which = 1), pac_fft forward (which = 2) or pac_fft inverse (which = 3):
 * the same launches, with a CUDA event recorded on `stream`
 * before and after each one; synchronises `stream` and writes each launch's
 * device time (ms) to launch_ms[0..*n_launches) and a kernel id to
 * kernel_ids[] (0 = forward DIF pass, 1 = fused DIF+product+DIT pass,
 * 2 = inverse DIT pass, 3 = permutation, 4 = pointwise product, 5 = whole
 * pass sequence in one cooperative launch, 6 = plane pass: the last two
 * axes forward, product and inverse with whole planes in one CTA).
 * max_launches bounds both arrays; PAC_ERR_ARG if it is too small.
 */
int pac_convolve_timed(pac_plan p, int which, const void* x_dev, void* y_dev, void* stream, int max_launches,
                       float* launch_ms, int* kernel_ids, int* n_launches);

/*
 * Test hook of the bounded device waits (no counterpart in the paper): runs
 * the plan's convolution as the single-launch cooperative kernel (the passes
 * as phases separated by grid-wide barriers), with every barrier waiting for
 * one arrival more than the grid can make and each wait limited to
 * spin_limit polls (1 .. 2^20).  Every wait therefore runs out: the CTA
 * records 1 in the device error word (read and cleared by
 * pac_plan_query(PAC_Q_DEVICE_ERROR)) and goes on, so the kernel ends
 * without a hang and the device stays usable.  y_dev receives passes run
 * without synchronisation between them, not the convolution.  Needs a plan
 * whose passes all have one group size and no plane pass (e.g. 1-D 2^16,
 * radix 2), else PAC_ERR_ARG.  Asynchronous on `stream`.
 */
int pac_test_barrier_timeout(pac_plan p, const void* x_dev, void* y_dev, void* stream, int spin_limit);

/*
 * Test hook of the persistent batched kernel's bounded waits (no
 * counterpart in the paper): runs the batch as one launch of the persistent
 * kernel (as pac_convolve_many does), with every pass' wait for the pass
 * before it in its instance set one finished tile beyond what that pass has,
 * and each wait limited to about wait_us microseconds (1 .. 10^6).  Every
 * such wait runs out: the unit records 1 in the device error word (read and
 * cleared by pac_plan_query(PAC_Q_DEVICE_ERROR)) and goes on, so the launch
 * ends and the device stays usable; y receives passes run out of order, not
 * the convolutions.  Synchronises `stream`.  PAC_ERR_ARG when the batch has
 * no form of the persistent kernel or no instance of more than one pass.
 */
int pac_test_batch_timeout(int count, const pac_plan* plans, const void* const* x_dev, void* const* y_dev,
                           void* stream, int wait_us);

/*
 * Allocation-free form of pac_convolve_permuted, for callers that cannot
 * allocate device memory: processes whose GPU memory is owned by another
 * allocator that reserved nearly all of it up front, services under a hard
 * device-memory quota that forbids growth after start-up, and latency-critical
 * paths that cannot afford cudaMalloc's implicit synchronisation.  The paper
 * has no counterpart; it is an interface convenience of this library.
 *
 * Computes the same result as pac_convolve_permuted (same stage kernels and
 * explicit index-reversal passes) but allocates nothing: its N-element
 * intermediate lives in one fixed 8 MiB static device buffer inside the
 * library (held by every GPU that loads the library until exit), and the
 * index-reversal positions are computed, not read from allocated tables.
 * Limit: N * elem size <= 8 MiB (1,048,576 complex64 or 524,288 complex128
 * elements); larger plans return PAC_ERR_SIZE.  All calls share the buffer:
 * calls whose work overlaps on the GPU race (serialise them on one stream).
 * The buffer needs no clearing (every element is written before it is read).
 * The first call on each device looks up the buffer's device address; make it
 * before any stream capture.  That address is kept for the life of the
 * process: after cudaDeviceReset (or anything else that destroys the
 * device's primary context) it is stale, like every plan made before the
 * reset, so the library must not be used across a device reset.
 * Asynchronous on `stream`; y_dev may equal x_dev.
 */
int pac_convolve_permuted_noalloc(pac_plan p, const void* x_dev, void* y_dev, void* stream);

/*
 * Autotuner: time the candidate pass schedules of this problem on the current
 * device (the largest group per pass, i.e. how many DIF stages one pass fuses,
 * from the largest a CTA holds down to small groups; and, in 2-D/3-D, the
 * plane pass on or off and its tile: a whole plane per CTA or a plane split
 * over a cluster of K CTAs; and the tile of the group passes: the default
 * width or, for groups whose tile rows span 256 bytes or more, the narrow tile
 * of half the columns, twice the CTAs), `reps` convolutions each after a warm-up, and keep
 * the fastest.  Plans created afterwards with the same (dims, radix, dtype)
 * use it.  With PAC_TUNE_FILE set in the environment, tuned schedules are
 * read from that file on first use and appended to it.  Allocates and frees
 * device memory (twice the problem) and synchronises the device.
 * best_us (may be NULL) receives the winner's median time per convolution.
 * With PAC_TUNE=search in the environment, pac_plan_create tunes a problem
 * the first time a plan is made for it.  PAC_LOG=1 makes every plan print
 * its pass schedule (groups, plane pass) to stderr.  For stage lists of
 * several prime bases (radix 0) the candidates include groups spanning bases
 * (compiled kernels for 48, 120, 1000 and 6000 points, the runtime-radix
 * kernel for other sizes) and one-base groups; PAC_MIXED in the environment overrides
 * the choice for every plan (see pac_plan_create).
 */
int pac_tune(int ndim, const int64_t* dims, int radix, pac_dtype dtype, int reps, double* best_us);

/* Plan facts for benches and tests: see PAC_Q_* keys. */
int pac_plan_query(pac_plan p, int key, int64_t* value);
enum {
    PAC_Q_NDIM = 0,
    PAC_Q_N_TOTAL = 1,            /* N */
    PAC_Q_ELEM_BYTES = 2,         /* 8 or 16 */
    PAC_Q_LAUNCHES_CONVOLVE = 3,  /* kernel launches per pac_convolve */
    PAC_Q_LAUNCHES_PERMUTED = 4,  /* kernel launches per pac_convolve_permuted */
    PAC_Q_LAUNCHES_FORWARD = 5,   /* kernel launches per pac_forward_unordered */
    PAC_Q_DEVICE_BYTES = 6,       /* device memory the plan owns (tables it shares with plans of the
                                     same shape, radix, dtype and schedule counted in full) */
    PAC_Q_HAS_SPECTRUM = 7,
    PAC_Q_DEVICE_ERROR = 8,       /* synchronises; returns and clears the device error word
                                     (1: a bounded grid-barrier wait gave up) */
    PAC_Q_GROUPS = 9,             /* stage groups (one pass each) over all axes */
    PAC_Q_PLANE = 10,             /* CTAs per plane of the plane pass, 0 when the plan has none */
    PAC_Q_GROUP_CAP = 11,         /* the schedule's group-exponent cap (0: none) */
    PAC_Q_NARROW = 12             /* group passes that take the narrow tile (half the columns) */
};

/*
 * Measured peak fused multiply-add rate of the current device in GFLOP/s
 * (2 flops per FMA) for the real type of dtype (FP32 for PAC_C64, FP64 for
 * PAC_C128): the ALU roofline of passes that the FP64 pipe bounds.  Runs a
 * short probe kernel and synchronises.
 */
int pac_measure_fma_peak(int dtype, double* gflops);

/*
 * Host only (no device): the pass groups a plan of this problem gets, in
 * forward order (axis 0 first), without the plane pass.  flags bit 0:
 * groups may span prime bases (as PAC_MIXED=1); bit 1 (bit 0 ignored): the
 * default rule of pac_plan_create, groups span bases only where every such
 * group has a compiled kernel (sizes 48, 120, 1000, 6000); cap: a schedule's
 * group-exponent cap (0: none).  For group g: axis[g], size[g] (its M) and
 * rounds[8 g .. 8 g + 7] (its in-CTA round radices, 0-padded).  *count: in,
 * the room of the arrays (groups; ignored when all three are NULL); out, the
 * number of groups.  PAC_C128_DF: one-base groups only (flags ignored) and
 * the double-float kernels' rounds (at most 4, 3 or 5 points).  Errors as
 * pac_plan_create, before any device call.
 */
int pac_plan_groups(int ndim, const int64_t* dims, int radix, pac_dtype dtype, int flags, int cap, int* axis,
                    int* size, int* rounds, int* count);

/*
 * Host only (no device): the twiddle table `which` of group `group` of the
 * schedule pac_plan_groups gives for this problem (same flags and cap),
 * exactly the values a plan of that problem uploads: each root
 * w_L^e = exp(-2 pi i e / L) (Section 2, twiddles of Eq. 25) computed in
 * FP64 with the exponent reduced in integers to the first eighth turn, then
 * rounded once to the plan's precision.  which 0: the round twiddles w_M^u,
 * u < M; 1: the external factor's low table w_L^u, u < T; 2: its high table
 * w_L^{T v}, v < ceil(L/T) (tables 1 and 2 are empty when the group has no
 * external factor).  out (may be NULL): *count interleaved complex values of
 * the dtype (PAC_C128_DF: 16 bytes an entry, each FP64 part split into the
 * FP32 pair {hi, lo}, hi = the FP64 value rounded to FP32, lo = the rest
 * rounded to FP32); *count in: room (entries), out: the table's length.  L, T (may
 * be NULL): the table's root order and the two-level split.  PAC_ERR_ARG for
 * a bad group or table or too little room; size errors as pac_plan_create.
 */
int pac_plan_twiddles(int ndim, const int64_t* dims, int radix, pac_dtype dtype, int flags, int cap, int group,
                      int which, void* out, int64_t* count, int64_t* L, int64_t* T);

/*
 * Test hook (host only, no device; no counterpart in the paper): the steps of
 * a convolution plan of this problem, for the CPU tests that run the pass
 * kernels' own code on the host.  The plan is built with one-base groups
 * (flags bit 1: also groups spanning prime bases where they have compiled
 * kernels, pac_plan_create's default rule; bit 2: groups spanning bases in
 * the runtime-radix kernel, as PAC_MIXED=rt), the group-exponent cap `cap`
 * (0: none) and per-axis passes, or with flags bit 0 the plane pass where
 * the shape has one of one CTA per plane;
 * its tables are written to `tables` (host memory, *table_bytes bytes) and
 * every step record points into the caller's host buffers: h, x (inputs,
 * N elements of the dtype's 16 or 8 bytes), y (output), scratch (N
 * elements), spec (*spec_elems elements).  `steps` (may be NULL) receives
 * *nsteps records of the library's internal HostStep layout (pass_args.h):
 * the forward passes of the spectrum (h -> scratch), its reorder with 1/N
 * (scratch -> spec), then the convolution's passes and plane pass (x -> y).  Call first
 * with tables and steps NULL for the sizes (*nsteps = the step count).
 * Errors: PAC_ERR_ARG (bad arguments, too little room, PAC_NARROW or
 * PAC_MIXED in the environment giving narrow tiles or runtime-radix
 * groups), size errors as pac_plan_create.
 */
int pac_test_host_steps(int ndim, const int64_t* dims, int radix, pac_dtype dtype, int cap, int flags,
                        const void* h, const void* x, void* y, void* spec, void* scratch, void* tables,
                        int64_t* table_bytes, int64_t* spec_elems, void* steps, int* nsteps);

/* Host-only helpers (no device needed): the stage list of pac_plan_create
 * (radix 0 included) and the reversal table of a stage list. */
int pac_stage_list(int64_t n, int radix, int* radices, int* count);
int pac_reverse_table(int nstages, const int* radices, int64_t* pos_to_freq);

/* Library version string. */
const char* pac_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PAC_H */
