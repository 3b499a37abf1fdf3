/*
 * pmh.h -- C ABI of the GB300-native ProbMinHash library (libpmh.so).
 *
 * ProbMinHash (Ertl, arXiv 1911.00675) computes m-component signatures of
 * weighted sets for the probability Jaccard similarity J_P (Sec.
 * Incorporating Weights, Eq. def_hash_jp): component k holds the element
 * minimising h_k(d), the first point of d's increasing random sequence whose
 * label is k (Eq. def_new_exp, Eq. signature_def).  J_P is estimated from the
 * fraction of equal components (Eq. jaccard_estimator).
 *
 * Conventions for every entry point:
 *   - Pointers documented as "device" must point to memory of the handle's
 *     device; "host" pointers to host memory.  The caller owns every input and
 *     output buffer; the library owns only workspace inside the handle.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream).  Errors detected from the arguments
 *     on the host are returned immediately and nothing is launched.  Errors in
 *     the data (bad weights, iteration limits) are reported per set in
 *     `set_status` once the stream reaches that point.
 *   - A handle is not thread-safe: use one handle per host thread.
 *   - The last error message of a handle is available from pmh_last_error.
 */
#ifndef PMH_H_
#define PMH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PMH_OK = 0,
    PMH_ERR_INVALID_ARG = 1,   /* argument rejected on the host, or bad offsets (per set) */
    PMH_ERR_BAD_WEIGHT = 2,    /* per set: a weight is < 0, NaN, +-inf, or 1/w is not finite */
    PMH_ERR_ITER_LIMIT = 3,    /* per set: an iteration cap was hit (Sec. Experiments), or a redo list was full */
    PMH_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    PMH_ERR_NO_MEMORY = 5,     /* workspace allocation failed */
    PMH_ERR_UNSUPPORTED = 6    /* a size outside the supported limits */
} pmh_status;

/* The six algorithms of the paper.  1 and 1a (resp. 3 and 3a) are logically
 * equivalent and produce identical signatures (Sec. Interleaved Element
 * Processing); each is still computed as its own item.  The last three are
 * the binary-weight specialisations of Sec. Conventional Jaccard Similarity
 * (for J rather than J_P): every element with w > 0 counts with weight 1,
 * ProbMinHash3/3a/4 draw Uniform([0,1)) instead of their truncated
 * exponentials, and gamma_i = i; PMH_V4U is SuperMinHash with a q_max stop. */
typedef enum {
    PMH_V1 = 0,   /* Algorithm ProbMinHash1: with replacement, uncorrelated */
    PMH_V1A = 1,  /* Algorithm ProbMinHash1a: interleaved ProbMinHash1 */
    PMH_V2 = 2,   /* Algorithm ProbMinHash2: without replacement, uncorrelated */
    PMH_V3 = 3,   /* Algorithm ProbMinHash3: with replacement, correlated (m >= 2) */
    PMH_V3A = 4,  /* Algorithm ProbMinHash3a: interleaved ProbMinHash3 (m >= 2) */
    PMH_V4 = 5,   /* Algorithm ProbMinHash4: without replacement, correlated (m >= 2) */
    PMH_V3U = 6,  /* ProbMinHash3 with binary weights */
    PMH_V3AU = 7, /* ProbMinHash3a with binary weights (identical to PMH_V3U) */
    PMH_V4U = 8   /* ProbMinHash4 with binary weights */
} pmh_variant;

typedef enum {
    PMH_FP64 = 0,          /* every point value in FP64 */
    PMH_FP32_RECHECK = 1   /* FP32 candidates with an error bound; FP64 recomputation of the
                              candidates within the bound of each other.  Same output as PMH_FP64. */
} pmh_precision;

typedef struct pmh_handle_s *pmh_handle;

/* Limits. */
#define PMH_MAX_M 8192u                 /* signature size m <= 8192 */
#define PMH_MAX_VARIANTS 16             /* variants per pmh_sketch_batch call (repeats allowed) */
#define PMH_MAX_SET_ELEMENTS 0xFFFFFFFFll /* elements per set < 2^32 */

/* Device counters written by pmh_sketch_batch when `counters` is non-NULL
 * (device array of PMH_NUM_COUNTERS uint64, accumulated, never cleared). */
enum {
    PMH_CNT_ELEMENTS = 0,     /* elements with w > 0 visited (all rounds) */
    PMH_CNT_POINTS32 = 1,     /* point values evaluated in FP32 */
    PMH_CNT_POINTS64 = 2,     /* point values evaluated in FP64 */
    PMH_CNT_CONTENDERS = 3,   /* FP32 near-margin contender records */
    PMH_CNT_RESOLVED = 4,     /* exact FP64 re-evaluations of contenders */
    PMH_CNT_ROUNDS = 5,       /* threshold rounds beyond the first */
    PMH_CNT_DEEP = 6,         /* elements processed warp-cooperatively */
    PMH_CNT_PREFILTERED = 7,  /* elements rejected without evaluating a logarithm */
    /* SM clock cycles spent per phase, summed over warps (timers read by lane 0); recorded only
     * by a library built with -DPMH_CYCLE_COUNTERS=1 (their clock reads cost about 6 % of the
     * sketch kernels' time), else left unchanged */
    PMH_CNT_CYC_PASS0 = 8,    /* item setup: empty signature, threshold */
    PMH_CNT_CYC_FIRST = 9,    /* threshold rounds: filter, survivors, deep mode, team barrier at their end */
    PMH_CNT_CYC_DEEP = 10,    /* warp-cooperative expansion of long sequences (part of CYC_SURV) */
    PMH_CNT_CYC_REFRESH = 11, /* q_max refreshes */
    PMH_CNT_CYC_FINISH = 12,  /* contender resolution and write-out */
    PMH_CNT_ITEMS = 13,       /* items processed */
    PMH_CNT_CYC_SURV = 14,    /* survivor expansion, lane-sequential and deep (part of CYC_FIRST) */
    PMH_CNT_CYC_ITEM = 15,    /* whole items, from the queue fetch to the barrier after write-out */
    PMH_CNT_CYC_WARP = 16,    /* warp lifetime in the sketch kernels (start to exit) */
    PMH_CNT_CYC_BARRIER = 17, /* waiting for the team's other warps at the end of a round (part of CYC_FIRST) */
    PMH_CNT_SEQ_STEPS = 18,   /* warp steps of lane-sequential survivor expansion (32 lane slots each) */
    PMH_CNT_SEQ_POINTS = 19,  /* points evaluated lane-sequentially (part of POINTS32/POINTS64) */
    PMH_CNT_REDO = 20,        /* FP32 items whose contender log overflowed, sketched again in FP64 */
    PMH_CNT_LISTED = 21,      /* prefilter list entries visited (part of ELEMENTS; see pmh_set_prefilter) */
    PMH_CNT_LIST_HASHED = 22, /* elements hashed once for all variants by the prefilter pass */
    PMH_CNT_LIST_SKIPPED = 23,/* elements the prefilter rejected for a variant (part of ELEMENTS and PREFILTERED) */
    PMH_NUM_COUNTERS = 24
};

/* Creates a handle bound to CUDA device `device` (the device is made current
 * for every later call on this handle).  *out receives the handle.
 * Returns PMH_ERR_CUDA if the device cannot be used. */
pmh_status pmh_create(pmh_handle *out, int device);

/* Releases the handle and its workspace (synchronises its device first).
 * NULL is ignored. */
void pmh_destroy(pmh_handle h);

/* The last error message recorded on `h` ("" if none); valid until the next
 * call on `h`.  With h == NULL: the message of the last failed pmh_create. */
const char *pmh_last_error(pmh_handle h);

/*
 * pmh_sketch_batch -- signatures of a CSR batch of weighted sets, for one or
 * several variants in one persistent launch.
 *
 * Defines: Algorithms ProbMinHash1/1a/2/3/3a/4 (Sec. ProbMinHash1 ...
 * Interleaved Element Processing).  Random draws come from a counter-based
 * SplitMix64 stream keyed by mix(id ^ mix(seed)): point i uses stream words
 * 2i-2 (value) and 2i-1 (label).  Ties are broken by the lexicographic
 * minimum of (value, id), and an element stops once a point exceeds q_max.
 *
 *   ids       device uint64[N]: element ids; set s owns ids[offsets[s] .. offsets[s+1]).
 *             Ids must be distinct within a set (precondition, not checked).
 *   weights   device float64[N]: weights; w = 0 (or -0) elements are skipped.
 *   offsets   device int64[num_sets+1], offsets[0] >= 0 (usually 0), non-decreasing; a set
 *             whose offsets are decreasing gets PMH_ERR_INVALID_ARG in set_status.
 *   num_sets  >= 0.
 *   m         signature size, 1 <= m <= PMH_MAX_M (m >= 2 for V3/V3A/V4).
 *   variants  host int32[num_variants] of pmh_variant values (repeats allowed),
 *             1 <= num_variants <= PMH_MAX_VARIANTS;
 *             item (v, s) is set s sketched with variants[v].
 *   precision pmh_precision.
 *   seed      stream seed; signatures are comparable only for equal (m, seed)
 *             and variant family.
 *   out_ids   device uint64[num_variants * num_sets * m], row (v*num_sets + s):
 *             the winning element id of each component; 0 for empty sets.
 *   out_q     device float64[same] or NULL: the component minima h (exact FP64);
 *             +inf for empty sets.  With PMH_FP32_RECHECK this costs one exact
 *             FP64 evaluation per component.
 *   set_status device int32[num_variants * num_sets] or NULL: per-item pmh_status.
 *   counters  device uint64[PMH_NUM_COUNTERS] or NULL: accumulated work counters.
 *   stream    cudaStream_t.
 * Workspace (the work queue) is allocated on the first call and grown when a
 * larger batch arrives; repeated calls with the same arguments replay a cached
 * CUDA graph.
 * Returns PMH_OK once launched, or a host-side error.
 */
pmh_status pmh_sketch_batch(pmh_handle h, const uint64_t *ids, const double *weights, const int64_t *offsets,
                            int64_t num_sets, uint32_t m, const int32_t *variants, int32_t num_variants,
                            int32_t precision, uint64_t seed, uint64_t *out_ids, double *out_q,
                            int32_t *set_status, uint64_t *counters, void *stream);

/*
 * pmh_sync_status -- waits for `stream` to reach this call, then reduces the
 * per-item statuses a pmh_sketch_batch call wrote (set_status of n items).
 *   counts     host int64[8] or NULL: counts[c] = items with status c for
 *              c = 0..6; counts[7] = items with any other value.
 *   first_bad  host int64 or NULL: index of the first item whose status is not
 *              PMH_OK, or -1.
 * Returns PMH_OK when every item is PMH_OK, else the status of the first item
 * that is not (PMH_ERR_INVALID_ARG for a value outside the enum), or a
 * host-side error (NULL handle, n < 0, NULL set_status with n > 0;
 * PMH_ERR_CUDA).  A small device buffer stays with the handle.
 */
pmh_status pmh_sync_status(pmh_handle h, const int32_t *set_status, int64_t n, int64_t *counts, int64_t *first_bad,
                           void *stream);

/*
 * pmh_sketch_batch_host -- pmh_sketch_batch on HOST buffers: the same batch,
 * variants, precision, seed and results (identical values), with ids,
 * weights, offsets and the outputs in host memory.
 *
 * The call splits the sets into `chunks` contiguous ranges by work (the first
 * range gets half the share of the others; chunks <= 0: automatic, 4 for
 * batches of 2^22 elements or more, else 1) and pipelines them on internal
 * streams: host->device copy of a range's elements; the sketch of the range,
 * alternating between two compute streams so that one range's kernels fill
 * the SMs another range leaves idle; device->host copy of each variant
 * family's rows as soon as that family is done.  Copies overlap the kernels when the host
 * buffers are page-locked (cudaHostAlloc / cudaHostRegister / pinned tensors);
 * pageable buffers work but do not overlap.  It returns when every result is
 * in host memory.
 *
 *   offsets   host int64[num_sets + 1], non-decreasing, offsets[0] >= 0; the
 *             call reads ids / weights [0, offsets[num_sets]).
 *   out_ids   host uint64[num_variants * num_sets * m] (same layout as on the
 *             device); out_q, set_status optional (NULL).
 * Device workspace (a copy of the inputs and two chunks of outputs) stays
 * with the handle for later calls.  Errors: as pmh_sketch_batch, plus
 * PMH_ERR_INVALID_ARG for decreasing or negative offsets (checked on the
 * host).  Not for use while a stream capture is active on this thread.
 */
pmh_status pmh_sketch_batch_host(pmh_handle h, const uint64_t *ids, const double *weights, const int64_t *offsets,
                                 int64_t num_sets, uint32_t m, const int32_t *variants, int32_t num_variants,
                                 int32_t precision, uint64_t seed, uint64_t *out_ids, double *out_q,
                                 int32_t *set_status, int32_t chunks);

/*
 * pmh_last_host_span_ms -- device-side time of the most recent completed
 * pmh_sketch_batch_host call on `h`, from its first input copy to its last
 * output copy (CUDA events), and the number of ranges it used (chunks may be
 * NULL).  The host wall time of the call minus this span is time the device
 * waited for the host.  Errors: PMH_ERR_INVALID_ARG without such a call.
 */
pmh_status pmh_last_host_span_ms(pmh_handle h, float *ms, int32_t *chunks);

/*
 * pmh_sketch_batch_noalloc -- pmh_sketch_batch for callers that cannot
 * allocate GPU memory: code that runs under another runtime's fixed memory
 * budget, inside a framework that forbids cudaMalloc on its hot path, or
 * where an allocation could stall or fail at the worst moment.  The paper has
 * no counterpart; this is an interface of this library only.
 *
 * Same arguments and results as pmh_sketch_batch (without a handle: it runs
 * on the current device), computed by the same kernels, except that grid mode
 * is off: a set of 2^20 elements or more is sketched by one team instead of
 * the whole GPU (same result, far slower).  Its scratch memory (constant
 * tables, work queue, FP64 redo list, per-set statistics) is one fixed array
 * of about 6 MiB that every GPU holds for as long as the library is loaded;
 * the call itself allocates and frees no device memory and builds no CUDA
 * graph.  Limits: num_sets <= PMH_NOALLOC_MAX_SETS and
 * num_sets * num_variants <= PMH_NOALLOC_MAX_ITEMS; larger batches return
 * PMH_ERR_UNSUPPORTED (message in pmh_last_error(NULL)).  Each call resolves
 * the array's device address and uploads the tables of its m from a static
 * host buffer in stream order; because later calls rewrite that buffer, a
 * call made while `stream` is being captured into a CUDA graph returns
 * PMH_ERR_UNSUPPORTED.  Every call on a device shares the array: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and must
 * be ordered by the caller.
 */
#define PMH_NOALLOC_MAX_SETS 65536
#define PMH_NOALLOC_MAX_ITEMS 262144
pmh_status pmh_sketch_batch_noalloc(const uint64_t *ids, const double *weights, const int64_t *offsets,
                                    int64_t num_sets, uint32_t m, const int32_t *variants, int32_t num_variants,
                                    int32_t precision, uint64_t seed, uint64_t *out_ids, double *out_q,
                                    int32_t *set_status, uint64_t *counters, void *stream);

/*
 * Profiling.  pmh_set_profiling(h, 1) makes every later pmh_sketch_batch on
 * `h` record CUDA events on its stream before the work-queue build, between
 * the queue build (with the per-set statistics) and the sketch kernels (with
 * the prefilter pass of pmh_set_prefilter), and after them (each call its own
 * events from a ring of 256; profiled calls are launched directly, not from
 * a CUDA graph; calls during a stream capture are not profiled).
 * pmh_last_kernel_ms waits for the most recent call to finish and returns its
 * two intervals in milliseconds (queue build, sketch kernels); it returns
 * PMH_ERR_INVALID_ARG if that call was not profiled.
 * pmh_kernel_ms_history returns the same pair for up to `max_calls` most
 * recent profiled calls (oldest first) into host float arrays of that length
 * (either may be NULL), waits for the newest, and stores the number in *count.
 */
pmh_status pmh_set_profiling(pmh_handle h, int32_t enable);
pmh_status pmh_last_kernel_ms(pmh_handle h, float *queue_ms, float *sketch_ms);
pmh_status pmh_kernel_ms_history(pmh_handle h, int32_t max_calls, float *queue_ms, float *sketch_ms, int32_t *count);

/*
 * Team shapes of the persistent sketch kernel (no counterpart in the paper:
 * how GPU threads share one item).  A team of warps shares one signature in
 * shared memory and sketches one (set, variant) item at a time:
 *   PMH_SHAPE_WARP  4 warps per block, each warp its own team
 *   PMH_SHAPE_CTA8  8 warps per block, one team
 *   PMH_SHAPE_QUAD  4 warps per block, one team (register budget for 8 blocks/SM)
 *   PMH_SHAPE_PAIR  8 warps per block, teams of 2 warps
 *   PMH_SHAPE_QUAD8 8 warps per block, teams of 4 warps
 *   PMH_SHAPE_QUAD8L the same with the register budget for 5 blocks/SM
 * All shapes return identical results.
 *
 * pmh_set_team_shape(h, family, shape): family 1..4 (ProbMinHash1/1a, 2,
 * 3/3a, 4) or 0 for all; shape one of the above, or -1 to let the handle
 * choose.  A shape whose shared memory does not fit falls back to the default
 * rule (teams of 2 warps when 16 warps per SM fit, else warp teams, else CTA8;
 * else the shape with the most resident warps that fits).
 *
 * pmh_set_autotune(h, enable): with enable = 1 (the default), the first
 * pmh_sketch_batch for a new (m, precision, family, log2 of the item count)
 * runs the batch twice per shape on the caller's stream, waits for it, and
 * keeps the shape with the fastest trial per family for later calls; not during stream capture
 * (the default rule applies there).  enable = 0 uses the default rule;
 * enable = -1 also forgets the shapes chosen so far and keeps tuning on.
 *
 * pmh_last_team_shapes(h, shapes): host int32[4], the shape each family used
 * in the most recent call (-1 for families it did not have).
 * Errors: PMH_ERR_INVALID_ARG for a NULL handle or pointer or values out of range.
 */
#define PMH_SHAPE_WARP 0
#define PMH_SHAPE_CTA8 1
#define PMH_SHAPE_QUAD 2
#define PMH_SHAPE_PAIR 3
#define PMH_SHAPE_QUAD8 4
#define PMH_SHAPE_QUAD8L 5
pmh_status pmh_set_team_shape(pmh_handle h, int32_t family, int32_t shape);
pmh_status pmh_set_autotune(pmh_handle h, int32_t enable);
pmh_status pmh_last_team_shapes(pmh_handle h, int32_t *shapes);

/*
 * pmh_last_launches -- number of kernels the most recent pmh_sketch_batch on
 * `h` launched (queue build, statistics, per-family sketch kernels, with
 * PMH_FP32_RECHECK the per-family FP64 redo kernels (they return at once when
 * no item overflowed its contender log) and, when grid mode is on, its reset
 * kernel and per-family grid kernels).
 */
pmh_status pmh_last_launches(pmh_handle h, int32_t *launches);

/*
 * pmh_set_thresholds -- work-only tuning of later pmh_sketch_batch calls on `h`.
 * Results never depend on these values; only the amount of work does.
 *
 * The paper's algorithms generate each element's points in increasing order
 * and stop once a point exceeds the running maximum of the signature
 * (Sec. "ProbMinHash1", stop rule).  The GPU kernels first generate only the
 * points below a threshold T (first threshold round: T = m (ln m + t_c) / sum of weights,
 * which leaves a given component empty with probability about e^-t_c / m);
 * while a component is still empty they repeat with T x 4, and after `rounds`
 * finite rounds with T = infinity (the paper's unbounded loop).
 *
 *   t_c       finite; default 3.
 *   t_c_grid  the same constant for grid-mode items; default 8.
 *   rounds    0..64 finite rounds; default 5.
 *   grid_min  sets with at least grid_min elements are processed by all SMs
 *             together (grid mode; at most 16 such items per family and
 *             call, the rest as usual); <= 0 turns grid mode off.
 *             Default 2^20.
 * Errors: PMH_ERR_INVALID_ARG for NULL h, a non-finite t_c / t_c_grid or
 * rounds outside [0, 64].
 */
pmh_status pmh_set_thresholds(pmh_handle h, double t_c, double t_c_grid, int32_t rounds, int64_t grid_min);

/*
 * pmh_set_prefilter -- work-only option of later pmh_sketch_batch calls on
 * `h` (no counterpart in the paper: how the first threshold round of the
 * sketch kernels is fed).  Results never depend on it.
 *
 * The paper's loop evaluates every element's first point, and only some
 * elements continue (Sec. "ProbMinHash1": most elements of a large set stop
 * after one point).  With the prefilter on, one extra pass per call hashes the
 * elements of every set of list_factor * m (ln m + t_c) up to 262,144
 * elements once for all variants and keeps those whose first point can lie
 * below the first round's threshold T in some family (the sketch kernels'
 * own log-free test, with the smallest lower bound of any family); the first
 * round of each weighted variant of such a set then visits only these
 * elements.  A later round (rare) visits all elements again.  Binary-weight
 * variants and the rejection sampler do not use the lists (a call with no
 * other variant skips the pass).
 *
 *   list_factor  default 2.0; <= 0 turns the prefilter off.
 *
 * Memory: lists of 8 bytes per element of the call (16-byte entries for up
 * to half the elements of each set; a set with more survivors than that is
 * filtered in full) plus 8 bytes per set, kept in the handle.  The first
 * pmh_sketch_batch call on new (ids, weights, offsets, num_sets) arrays reads
 * offsets[0] and offsets[num_sets] back to size them, which waits for
 * `stream`; calls made during a stream capture before that read skip the
 * prefilter.  Later calls on the same arrays (the handle keeps the counts of
 * its 16 most recent batches) reuse the count: if the offsets
 * were rewritten with more elements in between, the sets that no longer fit
 * in the lists are filtered in full (same result, more work).  A call that
 * finds no device memory for the lists runs without them.
 * Errors: PMH_ERR_INVALID_ARG for NULL h or a non-finite list_factor.
 */
pmh_status pmh_set_prefilter(pmh_handle h, double list_factor);

/*
 * pmh_set_limits -- resource caps of later pmh_sketch_batch calls on `h`
 * (the iteration limits that keep the paper's loops finite, Sec.
 * Experiments).  Results of items that stay within them do not change.
 *
 *   cap_points      points one element may generate in warp-cooperative
 *                   expansion (sequences longer than the lane-sequential caps
 *                   of 32 points for ProbMinHash1/1a and 64 for ProbMinHash3/3a
 *                   go there); an element that needs more fails its item with
 *                   PMH_ERR_ITER_LIMIT.  0 = the default 64 m ln(m+1) + 4096.
 *                   ProbMinHash2/4 sequences have m points and no cap.
 *   max_contenders  FP32 candidate path: contender records kept per item (two
 *                   per near-margin event; -1 = the defaults, 64 per team and
 *                   1024 per grid-mode item; at most 1024).  An item whose log
 *                   overflows is not failed: it is sketched again by the FP64
 *                   kernel that follows its family's kernels in the same call
 *                   (counter PMH_CNT_REDO), with the same result as PMH_FP64.
 * Errors: PMH_ERR_INVALID_ARG for NULL h or max_contenders outside [-1, 1024].
 */
pmh_status pmh_set_limits(pmh_handle h, uint32_t cap_points, int32_t max_contenders);

/*
 * pmh_set_te_sampler -- how later pmh_sketch_batch calls on `h` draw the
 * truncated exponentials Exp(lambda;0,1) of ProbMinHash3/3a/4 (weighted
 * variants; the binary-weight ones draw uniforms either way).
 *   PMH_TE_INVERSION (default): -log1p(U expm1(-lambda)) / lambda, U from
 *     point i's value word (stream word 2i-2).
 *   PMH_TE_REJECTION: Algorithm "Fast generation of random values from
 *     Exp(lambda;0,1)" (Sec. Truncated Exponential Sampling): x = c1 U with
 *     c1 = (e^lambda - 1)/lambda from the same value word, returned when below
 *     1; otherwise the paper's rejection loop, whose uniforms are stream words
 *     2^40 + 256 (i-1) + j (attempt t: j = 2t, 2t+1), so that the draws do not
 *     depend on order or precision.  After 64 rejected attempts (probability
 *     below 2^-190) the inversion of the value word is used.
 * The two samplers give different (equally distributed) signatures; both
 * precisions give the same signature for either.  Errors: PMH_ERR_INVALID_ARG
 * for NULL h or another value.
 */
#define PMH_TE_INVERSION 0
#define PMH_TE_REJECTION 1
pmh_status pmh_set_te_sampler(pmh_handle h, int32_t sampler);

/*
 * pmh_bbit_reduce -- Algorithm "Reduction to a b-bit signature": component k
 * (0-based) of every signature keeps the least significant b bits of a hash
 * of the pair (z_k, k): mix(z_k ^ mix(mix(seed) + (k+1) phi)), mix the
 * SplitMix64 finalizer and phi = 0x9E3779B97F4A7C15.
 *   sigs    device uint64[num_sigs * m] (row-major winning ids)
 *   b       1, 2, 4, 8, 16, 32 or 64
 *   packed  device uint64[num_sigs * W], W = ceil(m b / 64): field k occupies
 *           bits (k b) mod 64 .. +b-1 of word (k b) / 64 of its row; unused high
 *           bits of a row's last word are zero.
 * pmh_bbit_allpairs -- for every pair of packed rows, the number of equal
 * b-bit fields into device uint16[num_sigs * num_sigs] (row-major; with
 * upper_only only b >= a is written).  Different elements collide with
 * probability 2^-b, so (count/m - 2^-b) / (1 - 2^-b) estimates J_P without
 * that bias (the paper notes that the plain estimator Eq. jaccard_estimator
 * is biased for b-bit signatures).
 * Both run asynchronously on `stream`.  Errors: PMH_ERR_INVALID_ARG (NULL
 * pointers, bad b, m < 1), PMH_ERR_UNSUPPORTED (m > 65535 or too many rows
 * for one all-pairs launch), PMH_ERR_CUDA.
 */
pmh_status pmh_bbit_reduce(pmh_handle h, const uint64_t *sigs, int64_t num_sigs, uint32_t m, uint32_t b, uint64_t seed,
                           uint64_t *packed, void *stream);
pmh_status pmh_bbit_allpairs(pmh_handle h, const uint64_t *packed, int64_t num_sigs, uint32_t m, uint32_t b,
                             int32_t upper_only, uint16_t *counts, void *stream);

/*
 * pmh_check_exp1 -- the FP32 Exp(1) variate of the candidate path, E(word) =
 * -ln(1 - U), U = (word >> 11) 2^-53 (the inversion of Sec. "ProbMinHash1",
 * exponential spacings), for each of n device words into device float out[n],
 * on `stream`.  For verification of its error bound against FP64; the sketch
 * kernels use the same inline function.  Errors: PMH_ERR_INVALID_ARG for
 * n < 0 or NULL pointers with n > 0, PMH_ERR_CUDA if the launch fails.
 */
pmh_status pmh_check_exp1(const uint64_t *words, int64_t n, float *out, void *stream);

/*
 * pmh_check_texp -- the FP32 truncated-exponential variate of the candidate
 * path, TE(word) = -log1p(U c) * inv with U = (word >> 11) 2^-53, for the FP32
 * constants c = expm1(-lambda) and inv = 1/lambda (Sec. "ProbMinHash3",
 * Exp(lambda;0,1) by inversion); same conventions and errors as
 * pmh_check_exp1.
 */
pmh_status pmh_check_texp(const uint64_t *words, int64_t n, float c, float inv, float *out, void *stream);

/*
 * pmh_estimate_jp -- numerators of the J_P estimator (Eq. jaccard_estimator)
 * for every pair of signatures: counts[a*num_sigs + b] = #{k : sigs[a][k] == sigs[b][k]}.
 *
 *   sigs      device uint64[num_sigs * m], row-major (one signature per row).
 *   num_sigs  >= 0;  m: 1 <= m <= 65535.
 *   upper_only 0: the full matrix is written.  1: only entries with a <= b are
 *             written (the rest of `counts` is left untouched).
 *   counts    device uint16[num_sigs * num_sigs].
 * Exact integer counts; J_P estimate = counts / m.  Errors: PMH_ERR_INVALID_ARG
 * (NULL pointers, num_sigs < 0), PMH_ERR_UNSUPPORTED (m > 65535, more than
 * 65535 tiles of 128 rows), PMH_ERR_CUDA.
 * pmh_estimate_allpairs is the same call under its earlier name.
 */
pmh_status pmh_estimate_jp(pmh_handle h, const uint64_t *sigs, int64_t num_sigs, uint32_t m, int32_t upper_only,
                           uint16_t *counts, void *stream);
pmh_status pmh_estimate_allpairs(pmh_handle h, const uint64_t *sigs, int64_t num_sigs, uint32_t m,
                                 int32_t upper_only, uint16_t *counts, void *stream);

/*
 * pmh_estimate_jp_block -- the same counts (Eq. jaccard_estimator) between the
 * rows of two signature tables, one block of the pair matrix:
 * counts[a * ld_counts + b] = #{k : sig_a[a][k] == sig_b[b][k]}.  Used to split
 * the all-pairs matrix into tiles (one or several per GPU).
 *   sig_a, sig_b device uint64[num_a * m], [num_b * m] row-major (may alias).
 *   counts    device uint16, num_a rows of ld_counts >= num_b entries.
 * Errors: PMH_ERR_INVALID_ARG (NULL pointers, negative sizes, ld_counts <
 * num_b), PMH_ERR_UNSUPPORTED (m > 65535, more than 65535 tiles of 128 rows
 * of sig_a), PMH_ERR_CUDA.
 */
pmh_status pmh_estimate_jp_block(pmh_handle h, const uint64_t *sig_a, int64_t num_a, const uint64_t *sig_b,
                                 int64_t num_b, uint32_t m, uint16_t *counts, int64_t ld_counts, void *stream);

/*
 * pmh_estimate_pairs -- the same count for listed pairs (Eq. jaccard_estimator):
 * counts[i] = #{k : sig_a[pairs_a[i]][k] == sig_b[pairs_b[i]][k]}.
 *   sig_a, sig_b  device uint64[* x m] row-major signature tables (may alias).
 *   pairs_a, pairs_b device int64[num_pairs] row indices (not checked).
 *   counts    device uint32[num_pairs].
 */
pmh_status pmh_estimate_pairs(pmh_handle h, const uint64_t *sig_a, const uint64_t *sig_b, const int64_t *pairs_a,
                              const int64_t *pairs_b, int64_t num_pairs, uint32_t m, uint32_t *counts,
                              void *stream);

/*
 * pmh_pminhash_batch -- Algorithm P-MinHash (the paper's reference method for
 * J_P, Sec. Probability Jaccard Similarity): for every element d with
 * w(d) > 0 and every component k, h_k(d) = Exp(1)/w(d) from word k (0-based)
 * of the element's stream (key mix(id ^ mix(seed)), word_k = mix(key + (k+1)
 * phi), Exp(1) = -log1p(-U)); component k keeps the lexicographically smallest
 * (h_k(d), d).  No early stop: n m hash values per set.  For comparison with
 * the ProbMinHash algorithms, which reach signatures of the same distribution
 * with far fewer values for large n.
 *   ids, weights, offsets, num_sets, m (1..PMH_MAX_M), seed: as pmh_sketch_batch.
 *   out_ids   device uint64[num_sets * m]; out_q device float64[same] or NULL
 *             (exact FP64 minima); set_status device int32[num_sets] or NULL.
 * Candidates are screened in FP32 and compared exactly in FP64, so the result
 * is that of an all-FP64 evaluation.  Empty sets: ids 0, q +inf.  Errors: as
 * pmh_sketch_batch (bad weights per set in set_status).  Asynchronous on
 * `stream`; a 4-byte device counter stays with the handle.
 */
pmh_status pmh_pminhash_batch(pmh_handle h, const uint64_t *ids, const double *weights, const int64_t *offsets,
                              int64_t num_sets, uint32_t m, uint64_t seed, uint64_t *out_ids, double *out_q,
                              int32_t *set_status, void *stream);

/*
 * pmh_merge -- signature of a union of disjoint sets from the signatures of
 * its parts: per component the lexicographic minimum of (q, id) over `parts`
 * partial signatures (Eq. signature_def; the minimum over a union is the
 * minimum of the parts' minima, and q_max only decreases).
 *   q, z      device float64 / uint64 [parts * m] (part-major); q >= 0 or +inf
 *             (component minima as pmh_sketch_batch writes them).
 *   out_q, out_z device [m].
 * Bit-exact with sketching the union when the parts were sketched with the
 * same (m, seed, variant family) and exact q (out_q).
 */
pmh_status pmh_merge(pmh_handle h, const double *q, const uint64_t *z, int64_t parts, uint32_t m, double *out_q,
                     uint64_t *out_z, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PMH_H_ */
