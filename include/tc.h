/*
 * tc.h -- C ABI of a GB300 (sm_103a) tensor-contraction engine.
 *
 * The operation is the two-operand contraction of Section 1 ("Tensor
 * Notation") of Peise, Fabregat-Traver and Bientinesi, "On the Performance
 * Prediction of BLAS-based Tensor Contractions":
 *
 *     C[f] = alpha * sum_{k contracted} A[f_A, k] * B[f_B, k] + beta * C[f]
 *
 * An index that appears in both inputs and not in C is contracted; an index
 * that appears in exactly one input and in C is free.  Beyond the paper's
 * notation, an index in A, B and C is a batch (Hadamard) index: C and both
 * inputs are indexed by it, nothing is summed over it, and in every
 * algorithm it is a sliced loop (never a kernel index).  Every algorithm the
 * library runs is one of the loop nests of Section 2 (slicing rules of
 * Table 1: a loop nest around one dot, axpy, gemv, ger or gemm kernel, with
 * copies where a matrix slice has no unit-stride dimension), or the fused
 * GETT kernel (algorithm 0), which has no counterpart in the paper.
 *
 * Conventions (not fixed by the paper):
 *   spec     "C=A,B" with one lower-case letter per index, e.g. "abc=ai,ibc".
 *   extents  one int64 per distinct index, in order of first appearance in
 *            the spec string read left to right ("abc=ai,ibc": a, b, c, i).
 *   strides  element strides, C modes then A modes then B modes, each in the
 *            spec's mode order; NULL means Fortran-contiguous storage, first
 *            index fastest (Section 1).  Strides must be >= 1.
 *   A, B, C  device pointers owned by the caller.  The library never frees
 *            them.  Element types by plan dtype:
 *              TC_F64      A, B, C double
 *              TC_F32      A, B, C float
 *              TC_TF32     A, B, C float (tensor cores, TF32 products)
 *              TC_BF16X3   A, B, C float (each input split in three BF16
 *                          slices on the tensor cores; see tc_plan_set_split)
 *              TC_TF32X3   A, B, C float (each input split in two TF32
 *                          words, hi = tf32(x), lo = tf32(x - hi); the
 *                          products hi.hi, hi.lo and lo.hi on the tensor
 *                          cores)
 *              TC_E4M3     A, B, C float (each input divided by a power
 *                          of two that brings its largest magnitude to at
 *                          most 448, rounded to FP8 E4M3, products on the
 *                          tensor cores (kind::f8f6f4), FP32 accumulation;
 *                          the fused GETT only, global-load path)
 *              TC_BF16     A, B __nv_bfloat16; C float
 *              TC_F16      A, B __half; C float
 *   alpha,   host pointers to one double (TC_F64) or one float (all other
 *   beta     dtypes).  beta == 0 writes C without reading it.
 *   stream   a cudaStream_t passed as void*; NULL is the legacy default
 *            stream.
 *
 * Errors: every call returns a tc_status.  Device work is asynchronous:
 * tc_execute reports argument and launch errors at once and device-side
 * timeouts through tc_plan_device_status after the stream is synchronised.
 * A plan is not thread-safe; use one plan per host thread.  A plan runs
 * on one stream at a time: tc_execute on another stream while the plan's
 * previous execute is still in flight is refused with
 * TC_ERROR_INVALID_ARGUMENT.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TC_SUCCESS = 0,
    TC_ERROR_INVALID_SPEC = 1,      /* malformed spec or index classes */
    TC_ERROR_INVALID_EXTENT = 2,    /* extent < 1 or product overflow */
    TC_ERROR_INVALID_STRIDE = 3,    /* stride < 1 or C self-overlap */
    TC_ERROR_UNSUPPORTED_DTYPE = 4, /* dtype not valid for this algorithm */
    TC_ERROR_INVALID_ALGORITHM = 5, /* id out of range */
    TC_ERROR_OUT_OF_MEMORY = 6,     /* workspace allocation failed */
    TC_ERROR_CUDA = 7,              /* a CUDA runtime call failed */
    TC_ERROR_TIMEOUT = 8,           /* a bounded device wait gave up */
    TC_ERROR_INVALID_ARGUMENT = 9,  /* NULL pointer, bad size, misuse */
    TC_ERROR_ADMISSION = 10         /* request does not fit the budget */
} tc_status;

typedef enum {
    TC_F64 = 0,
    TC_F32 = 1,
    TC_TF32 = 2,
    TC_BF16 = 3,
    TC_F16 = 4,
    TC_BF16X3 = 5,
    TC_TF32X3 = 6,
    TC_E4M3 = 7
} tc_dtype;

/* Kernels of Section 2 (BLAS-1: dot, axpy; BLAS-2: gemv, ger; BLAS-3:
 * gemm) plus the fused GETT of algorithm 0. */
typedef enum {
    TC_KERNEL_DOT = 0,
    TC_KERNEL_AXPY = 1,
    TC_KERNEL_GEMV = 2,
    TC_KERNEL_GER = 3,
    TC_KERNEL_GEMM = 4,
    TC_KERNEL_GETT = 5
} tc_kernel;

typedef struct tc_plan_s *tc_plan;

/* One algorithm.  Loop and index letters are those of the spec. */
typedef struct {
    int32_t id;               /* 0 = fused GETT; 1..n = Section 2 algorithms
                                 in enumeration order (kernels dot, axpy,
                                 gemv, ger, gemm; kernel-index choices with
                                 the free index of A outermost, then that of
                                 B, then the contracted one; loop orders in
                                 lexicographic order of first appearance) */
    char name[32];            /* NUL-terminated, e.g. "i'c-gemm" or "gett":
                                 sliced loops outermost first, an apostrophe
                                 after the loop holding a copy, then "-" and
                                 the kernel (Section 2, naming footnote) */
    int32_t kernel;           /* tc_kernel */
    int32_t n_loops;          /* number of sliced loops */
    char loops[8];            /* sliced indices, outermost first */
    int32_t n_kernel_indices;
    char kernel_indices[4];   /* by role: dot {k}; axpy {f}; gemv {f, k};
                                 ger {fA, fB}; gemm {fA, fB, k} */
    uint32_t copy_mask;       /* bit 0: A slice copied, bit 1: B, bit 2: C */
    int32_t copy_level[3];    /* A, B, C: position of the loop whose body
                                 holds the copy, -1 before every loop,
                                 -2 no copy */
    int32_t n_phases;         /* device-wide sequential phases: product of
                                 the contracted loops that enclose a free
                                 loop (1 for GETT) */
} tc_algorithm;

/* Parses the spec, classifies the indices, validates extents and strides
 * and enumerates the algorithms (Section 2, Table 1; batch indices are
 * sliced in all of them).  No device work and no device memory.  Rejects:
 * an index in one input only, a repeated index within an operand, more
 * than 8 modes per operand, extents < 1, strides < 1, and C strides under
 * which two C elements share an address.  *out is NULL on failure. */
tc_status tc_plan_create(tc_plan *out, const char *spec, const int64_t *extents,
                         const int64_t *strides, tc_dtype dtype);

/* Frees the plan and the device workspace it owns.  NULL is accepted. */
tc_status tc_plan_destroy(tc_plan plan);

/* Number of algorithms including GETT (ids 0 .. count-1). */
tc_status tc_algorithm_count(tc_plan plan, int32_t *count);

/* Copies up to capacity algorithm records into out (out may be NULL when
 * capacity is 0) and stores the total in *count. */
tc_status tc_enumerate_algorithms(tc_plan plan, tc_algorithm *out,
                                  int32_t capacity, int32_t *count);

/* Selects the algorithm tc_execute runs.  A new plan starts with GETT
 * (id 0) selected, or with the top-ranked algorithm once tc_predict has
 * ranked every candidate through tc_plan_select_best. */
tc_status tc_plan_select(tc_plan plan, int32_t alg_id);

/* The currently selected algorithm id. */
tc_status tc_plan_selected(tc_plan plan, int32_t *alg_id);

/* Bytes of device workspace the algorithm needs (copy buffers; for GETT,
 * id 0, the pre-converted input of tc_plan_set_gett_pack, else 0).  The
 * plan allocates it on the first tc_execute of that algorithm and keeps it
 * until tc_plan_destroy; call tc_execute once before capturing a CUDA
 * graph.  The workspace serves one execute at a time, so tc_execute
 * refuses a second stream while the plan's last execute is in flight
 * (below): give each stream its own plan. */
tc_status tc_algorithm_workspace(tc_plan plan, int32_t alg_id, size_t *bytes);

/* C = alpha * A.B + beta * C with the selected algorithm, enqueued on
 * stream.  Returns after the launches are enqueued.  When the plan's
 * previous tc_execute ran on a different stream and has not finished yet
 * (an event recorded after it is still pending), nothing is enqueued and
 * TC_ERROR_INVALID_ARGUMENT is returned: concurrent executes of one plan
 * would share its workspace.  Executes on the same stream queue behind one
 * another as usual.  While `stream` is capturing a CUDA graph the check is
 * skipped and nothing is recorded. */
tc_status tc_execute(tc_plan plan, const void *alpha, const void *A,
                     const void *B, const void *beta, void *C, void *stream);

/* tc_execute for callers that must not allocate device memory, such as
 * code running while another thread captures a CUDA graph in global
 * capture mode (where cudaMalloc fails), code that works inside a fixed
 * device-memory budget owned by its own allocator, or latency-critical
 * loops that cannot afford an allocation.  The paper has no counterpart.
 * Callers running beside another thread's global-mode capture must pass a
 * stream of their own created non-blocking: work enqueued on the legacy
 * default stream (stream NULL) during that capture invalidates it.
 *
 * Runs the selected loop-nest algorithm (ids >= 1, TC_F64 or TC_F32) like
 * tc_execute, but its copy scratch is a fixed 16 MiB array that every GPU
 * loading this library holds until the process exits; the plan allocates
 * nothing.  An algorithm whose copies need more than 16 MiB is refused with
 * TC_ERROR_INVALID_ARGUMENT (tc_algorithm_workspace gives the need); GETT
 * (id 0) is refused with TC_ERROR_INVALID_ALGORITHM.  The first call on a
 * device looks up the array's device address; make that call before any
 * stream capture.  All calls share the one array: calls whose work
 * overlaps on the GPU (other streams, other threads) race on it.  Every
 * scratch element is written before it is read, so nothing needs clearing
 * between calls. */
tc_status tc_execute_no_alloc(tc_plan plan, const void *alpha, const void *A,
                              const void *B, const void *beta, void *C, void *stream);

/* tc_execute for operands in host memory (no paper counterpart): the
 * call a host program makes end to end.  Enqueued on `stream`, in order:
 * copies of hA and hB (and of hC when beta != 0) into device buffers the
 * plan owns, the selected algorithm as tc_execute runs it, and the copy of
 * C back into hC.  Returns once everything is enqueued: synchronise the
 * stream before reading hC or changing hA / hB.  hA, hB, hC use the plan's
 * layouts (the strides given at tc_plan_create; each buffer spans
 * 1 + sum (extent - 1) * stride elements) and element types.  Pinned host
 * memory (cudaHostAlloc / cudaHostRegister) keeps the copies asynchronous;
 * pageable memory works, but its copies block the calling thread.  The
 * device buffers are allocated by the first call (do not make it during a
 * stream capture) and kept until tc_plan_destroy.  The one-stream-at-a-time
 * rule of tc_execute applies, and is checked before any copy is queued. */
tc_status tc_execute_host(tc_plan plan, const void *alpha, const void *hA, const void *hB,
                          const void *beta, void *hC, void *stream);

/* Reads and clears the plan's device status word (waits for the stream
 * the plan last ran on): TC_SUCCESS or TC_ERROR_TIMEOUT. */
tc_status tc_plan_device_status(tc_plan plan);

/* TC_BF16X3 plans: number of BF16 slice products kept per multiply,
 * 3 (weights 1, 2^-8), 6 (adds 2^-16, the default) or 9 (all).  Other
 * values give TC_ERROR_INVALID_ARGUMENT; other dtypes ignore the setting. */
tc_status tc_plan_set_split(tc_plan plan, int32_t products);

/* Tensor-core GETT tile width along N: 128 or 256 columns of C per tile
 * (the tile is 128 x width), or 0 to choose by N (256 when N >= 256).
 * Other values give TC_ERROR_INVALID_ARGUMENT. */
tc_status tc_plan_set_gett_tile(tc_plan plan, int32_t width);

/* Tensor-core GETT input path: 1 (default) streams each operand that a
 * TMA tensor map can describe through cp.async.bulk.tensor into a staging
 * ring; 0 loads every operand with ordinary global loads.  Results are the
 * same either way. */
tc_status tc_plan_set_gett_tma(tc_plan plan, int32_t enable);

/* Tensor-core GETT, FP32 inputs (TC_BF16X3, TC_TF32X3, TC_TF32) and, for
 * both inputs only, 16-bit ones (TC_BF16, TC_F16) and TC_E4M3:
 * pre-conversion of the smaller input, or of both.  With it, a pre-pass
 * kernel writes the input once into the plan's workspace as the converted
 * shared-memory images of its tiles (split-BF16 slices, TF32 words, the
 * 16-bit values or the scaled E4M3 bytes in the MMA's core-matrix layout,
 * zeros past the extents), and the GETT copies
 * them instead of loading and converting the input per tile; the K order
 * then follows the larger input alone.  mode 0: never; 1 (default): both
 * inputs for the compensated split form (K past the chunk of
 * tc_plan_set_compensation) and wherever M and N are both at least 1024,
 * when their images fit in 2 GiB, else (FP32 inputs) the smaller input
 * when it has at most 1/8 of the larger one's elements and its images fit
 * in 64 MiB; 2: the smaller input (FP32 inputs) whenever its images fit in
 * 64 MiB; 3: both inputs whenever their images fit in 2 GiB (else none),
 * each stage's two images then reach shared memory as two 1-D bulk copies
 * and no input is staged by TMA.  Other values give
 * TC_ERROR_INVALID_ARGUMENT.  The workspace is allocated by the first
 * execute that needs it (tc_algorithm_workspace(plan, 0) bounds it).  The
 * K order, and so the rounding of the sums, depends on whether an input is
 * pre-converted but not on which (modes 1-3 with a pre-converted input give
 * the same bits) nor on tc_plan_set_gett_tma.  With pre-conversion an
 * execute launches two kernels (pre-pass, GETT), three with both inputs. */
tc_status tc_plan_set_gett_pack(tc_plan plan, int32_t mode);

/* Tensor-core GETT, FP32-input kinds (TC_BF16X3, TC_TF32): CTA pairs.
 * With 1, and where the launch allows it (256-column tiles, no
 * compensated accumulation, more than 128 rows of M, every input staged by
 * TMA or pre-converted; or, for TC_BF16X3 with both inputs pre-converted
 * (tc_plan_set_gett_pack), any layout with more than 128 rows of M, on
 * 256-column tiles or compensated 128-column ones), clusters of two CTAs
 * share each MMA (tcgen05.mma.cta_group::2, M = 256): each CTA stages and
 * converts (or copies) its 128 rows of A and half of the tile's rows of B,
 * so a CTA moves half the B bytes per MMA; 0 (default) keeps one CTA per
 * tile.  Results are the same bits either way.  Other values give
 * TC_ERROR_INVALID_ARGUMENT. */
tc_status tc_plan_set_gett_pair(tc_plan plan, int32_t enable);

/* TC_BF16X3 and TC_TF32X3, tensor-core GETT without compensation: split
 * accumulators.  With 1 the weight-1 slice product (0,0) accumulates in one tensor-memory
 * accumulator and the smaller products in a second one, added once in the
 * epilogue: only K/16 FP32 roundings then act on the magnitude of the whole
 * sum instead of 6K/16, at the cost of not double-buffering the
 * accumulators.  0: one accumulator for every product.  -1 (default): split
 * when K > 64.  Other values give TC_ERROR_INVALID_ARGUMENT. */
tc_status tc_plan_set_split_accumulators(tc_plan plan, int32_t enable);

/* Failure-detection self-test (no paper counterpart).  Launches one CTA on
 * `stream` whose thread 0 waits on an mbarrier with the bounded wait every
 * kernel of this library uses, with limit_ns (0 < limit_ns <= 1e10) in place
 * of the kernels' 2 s; with signal != 0 a thread of another warp arrives
 * first.  Blocks until the kernel has finished.  Returns TC_ERROR_TIMEOUT
 * when the wait ran out (the kernel then returns normally and the context
 * stays usable), TC_SUCCESS when it was signalled, TC_ERROR_INVALID_ARGUMENT
 * for a limit out of range, TC_ERROR_CUDA on a launch or copy failure. */
tc_status tc_selftest_bounded_wait(int64_t limit_ns, int32_t signal, void *stream);

/* TC_BF16X3 and TC_TF32X3 plans, tensor-core GETT: compensated accumulation.  With a
 * chunk of c K elements (a positive multiple of 32) and K > c, each output
 * is summed on the tensor cores in FP32 over chunks of c contracted
 * positions, and the chunk sums are added into a float-float (hi, lo) pair
 * held in tensor memory by an error-free two-sum; the result is hi + lo.
 * The FP32 accumulation error then grows with c instead of with K.  Such
 * launches use 128 x 128 tiles whatever tc_plan_set_gett_tile says.
 * -1 (default) = 256; 0 = off (one FP32 accumulator across all of K).
 * Other values give TC_ERROR_INVALID_ARGUMENT; other dtypes and the loop
 * nests ignore the setting.  Beyond the paper, which computes in FP64. */
tc_status tc_plan_set_compensation(tc_plan plan, int32_t chunk);

/* 2 * product of all extents. */
tc_status tc_plan_flops(tc_plan plan, double *flops);

/* ---- Performance prediction (Section 3) ------------------------------
 *
 * The analysis runs at one of two granularities:
 *   0  the paper's: the algorithm's sliced loops around one BLAS call;
 *   1  the device's: the device-wide phases (contracted loops that enclose
 *      a free loop) around one phase launch.
 * Sizes are in units of elem_size bytes per element (pass 1 to count
 * elements, as the paper's worked example does); cache_size and line_size
 * use the same unit (the L2 and its 128-byte line on the device). */

typedef struct {
    int32_t kind;       /* 0 steady state (prefetch emulated, Section 3.3),
                           1 prefetch failure once per line (Section 3.4),
                           2 first iteration of loop `depth` (Section 3.5) */
    int32_t depth;      /* loop position of a first-iteration case, else -1 */
    int64_t count;      /* invocations this case stands for; the counts of
                           all cases sum to the product of the loop extents */
    int32_t omit;       /* 1 when the setup touches operands only */
    int32_t n_items;    /* length of the setup list */
} tc_pred_case;

typedef struct {
    int32_t kind;       /* 0 touch an operand slice, 1 remote region */
    int32_t operand;    /* 0 A, 1 B, 2 C; -1 for a remote region */
    int64_t size;       /* in the caller's unit */
} tc_setup_item;

/* Access distances (Section 3.2) of the kernel's A, B and C slices in the
 * steady state: for each, the summed size of the regions touched since its
 * previous access.  dist receives 3 values (A, B, C). */
tc_status tc_access_distances(tc_plan plan, int32_t alg_id, int32_t granularity,
                              int64_t elem_size, int64_t *dist);

/* The prediction cases of one algorithm (steady, prefetch failure, first
 * iterations), each with its invocation count and setup-list length. */
tc_status tc_prediction_cases(tc_plan plan, int32_t alg_id, int32_t granularity,
                              int64_t elem_size, int64_t cache_size, int64_t line_size,
                              tc_pred_case *out, int32_t capacity, int32_t *count);

/* The setup list of case `case_index` (Section 3.2): operands in order of
 * decreasing access distance, each followed by a remote region so that
 * what follows an operand sums to its distance, cut at the front to at
 * most 5/4 of cache_size. */
tc_status tc_setup_list(tc_plan plan, int32_t alg_id, int32_t granularity, int32_t case_index,
                        int64_t elem_size, int64_t cache_size, int64_t line_size,
                        tc_setup_item *out, int32_t capacity, int32_t *count);

/* Predicts the run time (seconds) of algorithms without running them
 * (Section 3 on the device): for each case of the device-granularity
 * analysis (first phase, steady phases) the setup list is replayed with
 * touch kernels and L2-sized remote reads, then one representative phase
 * runs over a few waves of its work, timed ten times with CUDA events; the
 * median, scaled to the whole phase and weighted by the case's count, sums
 * to the prediction.  The GETT runs a few waves of its real tiles.
 * alg_ids: n ids, or NULL for every algorithm (seconds then holds
 * tc_algorithm_count entries).  A, B, C: device buffers laid out as the plan
 * describes, or NULL for zero-filled scratch the call allocates and frees.
 * seconds[i] < 0 marks an algorithm that cannot run with the plan's dtype
 * (the loop nests run in FP64 and FP32 only).  Synchronises the stream.
 * The results stay in the plan for tc_plan_select_best. */
tc_status tc_predict(tc_plan plan, const int32_t *alg_ids, int32_t n, const void *A,
                     const void *B, void *C, double *seconds, void *stream);

/* Selects the algorithm with the smallest prediction of the last
 * tc_predict (ties: lower id) and stores its id in *best (may be NULL). */
tc_status tc_plan_select_best(tc_plan plan, int32_t *best);

/* Autotuner for the tensor-core GETT: predicts every tile configuration
 * -- tile width 128 or 256, TMA staging on or off, one or two CTAs per
 * tile (tc_plan_set_gett_pair), no input, the smaller input or both
 * pre-converted (tc_plan_set_gett_pack 0, 2 or 3); width, staging and
 * pairs give the same bits, pre-conversion can change the K order and so
 * the rounding (within the form's bound) -- with
 * the same micro-benchmark, and keeps the fastest in the plan, reporting
 * the width in *width and TMA in *tma (either may be NULL;
 * tc_plan_get_gett_config reads all four).  Results are cached per (spec,
 * extents, strides, dtype, split products, device); a cached plan key is
 * answered without running anything.  FP64/FP32 plans have nothing to tune
 * (width 0, tma 1).  Clears the plan's stored predictions. */
tc_status tc_autotune(tc_plan plan, const void *A, const void *B, void *C, void *stream,
                      int32_t *width, int32_t *tma);

/* The plan's tensor-core GETT settings: tile width (0: by N), TMA staging,
 * CTA pairs, pre-conversion mode; any pointer may be NULL. */
tc_status tc_plan_get_gett_config(tc_plan plan, int32_t *width, int32_t *tma, int32_t *pair,
                                  int32_t *pack);

/* Writes / merges the process-wide tuning cache as JSON lines, one per
 * key with its named integer choices ({"key": ..., "gett_tile": ...,
 * "gett_tma": ..., "gett_pair": ..., "gett_pack": ...} for plans,
 * {"key": ..., "batch_k_chunk": ..., "batch_tile_m": ...} for batch shape
 * classes), so that re-planning in a later process is free.  Loading keeps
 * every "name": integer pair; the tuners check the values they read. */
tc_status tc_tuning_cache_save(const char *path);
tc_status tc_tuning_cache_load(const char *path);

/* ---- Contraction chains: several kernels in one tree --------------------
 * Section 3.2: the access-distance method holds for trees with any
 * combination of loops and several kernels.  A chain "D=X,Y,Z" (one letter
 * a-z per index; extents in order of first appearance in the spec; dense
 * operands, first index fastest) computes every entry of D as the sum,
 * over the indices not in D, of the product of the three operands' entries;
 * every such index must appear in at least two operands.  It runs as two
 * pairwise contractions through an intermediate T, each a plan of this
 * library: one variant per pair contracted first (when both steps contract
 * an index), and for each a sliced form that loops one index of D carried
 * by the pair (not by the third operand) around both kernels, so that T
 * holds one slice.  T's modes: the pair's indices still needed, D's order
 * first, then the third operand's.  Host work only at creation. */
typedef struct tc_chain_s *tc_chain;

typedef struct {
    int32_t first[2];          /* operands contracted first (0 X, 1 Y, 2 Z) */
    int32_t third;
    char sliced;               /* index looped around both steps, 0: none */
    int64_t slices;            /* its extent (1 when not sliced) */
    int64_t workspace_bytes;   /* the intermediate (one slice) */
    double flops;              /* both steps, every slice */
    int32_t algorithm[2];      /* each step's selected algorithm id */
    double predicted_seconds;  /* (step 1 + step 2 predictions) x slices; < 0: none */
} tc_chain_variant;

/* dtype TC_F64, TC_F32 or an FP32-input tensor-core dtype (TC_TF32,
 * TC_BF16X3, TC_TF32X3; T is FP32).  Selects the variant with the fewest
 * flops (then the fewest slices).  Rejects specs that do not read "D=X,Y,Z",
 * indices outside a-z or repeated within an operand, an index outside D in
 * fewer than two operands, and chains with no valid variant. */
tc_status tc_chain_create(tc_chain *out, const char *spec, const int64_t *extents, tc_dtype dtype);
tc_status tc_chain_destroy(tc_chain chain);

/* Up to capacity variants into buf; their number into *count (may be NULL). */
tc_status tc_chain_variants(tc_chain chain, tc_chain_variant *buf, int32_t capacity, int32_t *count);

/* Largest intermediate in bytes that tc_chain_select(-1) may choose (-1: no
 * limit).  The limit covers the intermediate only: with a tensor-core
 * dtype a step's plan may also hold the pre-converted images of its inputs
 * (tc_plan_set_gett_pack's default), allocated by its first execute. */
tc_status tc_chain_set_workspace_limit(tc_chain chain, int64_t bytes);

/* Predicts every variant: for each step, tc_predict over every algorithm
 * (all_algorithms = 1) or over the fused GETT alone (0), keeping the
 * fastest; then selects as tc_chain_select(-1).  Runs micro-benchmarks on
 * stream with scratch operands; blocks until done. */
tc_status tc_chain_predict(tc_chain chain, int32_t all_algorithms, void *stream);

/* variant >= 0: that variant (TC_ERROR_INVALID_ARGUMENT if its T exceeds
 * the limit); -1: the smallest prediction if every variant has one, else
 * the fewest flops (then the fewest slices), among the variants within the
 * limit. */
tc_status tc_chain_select(tc_chain chain, int32_t variant);
tc_status tc_chain_selected(tc_chain chain, int32_t *variant);

/* D = alpha * X Y Z + beta * D on stream (device pointers; alpha/beta as
 * for the steps' dtype).  The intermediate is allocated on first use and
 * kept; step 1 runs with alpha 1, beta 0.  A plan's stream rule applies to
 * the chain: one stream at a time. */
tc_status tc_chain_execute(tc_chain chain, const void *alpha, const void *X, const void *Y,
                           const void *Z, const void *beta, void *D, void *stream);

/* Both steps' tc_plan_device_status (the selected variant). */
tc_status tc_chain_device_status(tc_chain chain);

/* ---- Batched form: many independent contractions, one launch ------------
 * No paper counterpart.  Every problem has the batch's spec and its own
 * extents, dense Fortran-ordered operands, and must reduce to a strided
 * GEMM: the free indices of A, the free indices of B and the contracted
 * indices each appear in the same order and contiguously in the operands
 * that carry them ("abc=ai,ibc" does).  One persistent kernel walks the
 * flattened tile list of all problems, largest problem first. */

typedef struct tc_batch_s *tc_batch;

/* count problems; extents holds count rows of one extent per index (in the
 * spec's order of first appearance).  dtype TC_F32 or TC_F64 (SIMT FMA
 * chains), or TC_BF16X3 (FP32 operands, split-BF16 with six slice products
 * on the tensor-core GETT kernel, 128-row tiles).  Host work only. */
tc_status tc_batch_create(tc_batch *out, const char *spec, int32_t count,
                          const int64_t *extents, tc_dtype dtype);
tc_status tc_batch_destroy(tc_batch batch);

/* Tile policy.  TC_F32 / TC_F64 tiles hold 4096 outputs, (8 << s) rows x
 * (512 >> s) columns for s = 0..4, and K runs in chunks of 8, 16 or 32:
 * 0 (fixed) 64 x 64 with chunks of 16; 1 (rule, the default) the smallest
 * tile height that covers the problem's M, with the largest chunk that
 * fits; 2 (autotuned) the choice of tc_batch_autotune for the problem's
 * shape class.  TC_BF16X3: 0 (fixed) tensor-core GETT tiles of 128 x 256;
 * 1 (rule) the split-BF16 stream kernel -- one MMA tile per 128 columns n
 * with all of M, for batches whose every problem has A, B and C dense
 * along m, k and m, K a multiple of 4 up to 32 and M up to 128 (with A
 * and B 16-byte aligned at execution; otherwise GETT tiles) -- else GETT
 * tiles 128 x w with the w in {128, 256} with the fewest padded columns
 * plus 64 per tile; 2 the autotuner's.  Policy 2 before tc_batch_autotune
 * is TC_ERROR_INVALID_ARGUMENT. */
tc_status tc_batch_set_tiles(tc_batch batch, int32_t policy);

/* Host arrays of count device pointers, in the caller's problem order. */
tc_status tc_batch_set_operands(tc_batch batch, void *const *A, void *const *B,
                                void *const *C);

/* Uploads the problem table (allocates it on first use).  tc_batch_execute
 * calls it when needed; call it yourself before capturing a CUDA graph, so
 * the captured work is the kernel alone. */
tc_status tc_batch_prepare(tc_batch batch);

/* C_q = alpha * A_q.B_q + beta * C_q for every problem q, enqueued on
 * stream: one launch, or one launch per problem when
 * one_launch_per_problem is 1 (for comparison).  alpha/beta point to
 * double (TC_F64) or float. */
tc_status tc_batch_execute(tc_batch batch, const void *alpha, const void *beta,
                           int32_t one_launch_per_problem, void *stream);

/* Total flops (2 M N K summed), tiles of the current policy and compulsory
 * bytes (A, B, C once each, beta = 0); any pointer may be NULL. */
tc_status tc_batch_info(tc_batch batch, double *flops, int64_t *tiles, int64_t *bytes);

/* One shape class of the batch autotuner (TC_F32 / TC_F64: problems with
 * the same ceil(log2 M), ceil(log2 K) and N bucket -- 0: N <= 256, 1:
 * N <= 2048, 2: larger; TC_BF16X3: the whole batch, classes -1). */
typedef struct {
    int32_t m_log2, k_log2, n_class;
    int32_t problems;     /* problems in the class */
    int32_t candidates;   /* configurations timed (0: answered from the tuning cache) */
    int32_t tile_m, tile_n, k_chunk;  /* the fastest configuration */
    int32_t kernel;       /* its kernel: 0 SIMT, 1 tensor-core GETT tiles, 2 split-BF16 stream */
    double seconds_best;  /* the class alone at that configuration (median; -1 if cached) */
    double seconds_rule;  /* ... at policy 1's configuration (-1 if cached) */
    double seconds_fixed; /* ... at policy 0's configuration (-1 if cached) */
} tc_batch_tuning;

/* Autotuner of the batched form (needs the operands).  TC_F32 / TC_F64:
 * for every shape class, times every (tile shape, K chunk) candidate on
 * the class's problems alone (one warm-up, median of reps launches on
 * stream), keeps the fastest, then times the whole batch with 2 and 3
 * pipeline stages; the class choices go to the tuning cache, and a class
 * found there is not timed.  TC_BF16X3: times the whole batch on GETT
 * tiles of width 128 and 256 and, where every problem suits it, on the
 * stream kernel.  Leaves policy 2 selected.  Every timed launch runs
 * with alpha = 1, beta = 0, so each C_q holds A_q.B_q afterwards.  Writes
 * up to capacity class rows to classes and the number of classes to
 * *n_classes (may be NULL).  Blocks until the timings are done. */
tc_status tc_batch_autotune(tc_batch batch, void *stream, int32_t reps, tc_batch_tuning *classes,
                            int32_t capacity, int32_t *n_classes);

/* The current policy, SIMT pipeline stages (TC_BF16X3: 0), split-BF16
 * tile width (SIMT: 0) and kernel (0 SIMT, 1 tensor-core GETT tiles, 2
 * split-BF16 stream); any pointer may be NULL. */
tc_status tc_batch_config(tc_batch batch, int32_t *policy, int32_t *stages, int32_t *tile_n,
                          int32_t *kernel);

/* Tile rows, columns and K chunk of problem `problem` (caller's order)
 * under the current policy. */
tc_status tc_batch_problem_tiles(tc_batch batch, int32_t problem, int32_t *tile_m,
                                 int32_t *tile_n, int32_t *k_chunk);

/* TC_BF16X3 batches: waits for the stream of the last execute, then reads
 * and clears the batch's device status word: TC_SUCCESS, or
 * TC_ERROR_TIMEOUT when a bounded wait in the kernel ran out (the kernel
 * then stopped early and C is incomplete).  Other dtypes: TC_SUCCESS. */
tc_status tc_batch_device_status(tc_batch batch);

/* ---- Serving: continuous batching of contraction requests ---------------
 * No paper counterpart.  A worker thread admits queued requests in arrival
 * order when a slot is free and their operands fit in the remaining device
 * budget (one allocation made at creation, carved first-fit).  Admitted
 * requests wait by batch class -- FP64, FP32 (SIMT GETT), TC_BF16X3 with
 * K <= 64, TC_BF16X3 with 64 < K <= 256 (split accumulators) -- and
 * whenever one of the server's streams is free, the class whose oldest
 * request has waited longest becomes ONE persistent batched launch over the
 * tiles of all its admitted requests (inputs copied in, one descriptor per
 * request, results copied out if asked, one completion event).  TC_BF16X3
 * with longer K (compensated) and the other tensor dtypes run one launch
 * each.  Requests that arrive while batches run form the next batches, and
 * batches on different streams overlap.  A request's class, K order and
 * tile shapes follow from the request alone, so its result is the same
 * alone and in any mix.  The server allocates at creation only: the budget,
 * and per stream a pinned and a device staging area for its batch tables
 * (256 descriptors, 2^20 tiles). */

typedef struct tc_server_s *tc_server;

typedef struct {
    int64_t completed, failed;
    int64_t admission_stalls;   /* times the queue head waited for memory */
    int64_t peak_inflight, queued;
    double flops_served;        /* sum of 2*prod(extents) over completed */
    double span_seconds;        /* first submission to last completion */
    double p50_seconds, p99_seconds, max_seconds;  /* submit -> result ready */
    int64_t batches;            /* launches made (a batch, or one solo request) */
    int64_t max_batch;          /* most requests in one launch */
} tc_server_report;

/* budget_bytes of device memory (allocated now), at most `slots` requests
 * in flight, `streams` CUDA streams (1..64).  Uses the current device. */
tc_status tc_server_create(tc_server *out, int64_t budget_bytes, int32_t slots,
                           int32_t streams);

/* Queues one request.  A, B: host inputs laid out densely (Fortran order),
 * in the dtype's element types (include/tc.h header comment); pinned memory
 * lets the copies run asynchronously.  C: host output or NULL to keep the
 * result only on the device until the request completes.  The caller keeps
 * the buffers alive until the request is done.  A request larger than the
 * whole budget is refused with TC_ERROR_ADMISSION; TC_E4M3 with
 * TC_ERROR_UNSUPPORTED_DTYPE. */
tc_status tc_server_submit(tc_server server, const char *spec, const int64_t *extents,
                           tc_dtype dtype, const void *A, const void *B, void *C,
                           int64_t *request_id);

/* Non-blocking: *done = 1 once finished (the return value is then the
 * request's status) and *latency its submit-to-ready seconds. */
tc_status tc_server_poll(tc_server server, int64_t request_id, int32_t *done, double *latency);

/* Blocks until the request finishes or timeout_s passes
 * (TC_ERROR_TIMEOUT). */
tc_status tc_server_wait(tc_server server, int64_t request_id, double timeout_s);

tc_status tc_server_stats(tc_server server, tc_server_report *out);

/* Finishes every queued request, then frees everything. */
tc_status tc_server_destroy(tc_server server);

/* Static description of a status code.  Never NULL. */
const char *tc_status_string(tc_status status);

/* Message of the last failing call on this host thread ("" if none). */
const char *tc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
