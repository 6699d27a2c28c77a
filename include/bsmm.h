/*
 * bsmm.h - block-sparse, irregularly tiled matrix product C = alpha*A*B + beta*C
 * on one GB300 (sm_103a).
 *
 * The operation (Calvin & Valeev, "Task-Based Algorithm for Matrix
 * Multiplication", SC15, Sec. 2.1 and Algorithm 1): the matrices are cut by
 * three tilings -- row blocks r[0..M), column blocks c[0..N), inner blocks
 * q[0..K) -- of arbitrary, nonuniform sizes (Sec. 3.2, data overdecomposition
 * into arbitrarily sized blocks; Sec. 4.1, nonuniform blocking). A and B store
 * only the tiles their masks mark nonzero (block sparsity, Sec. 1). The product
 * is the set of tile tasks
 *
 *     C_ij <- alpha * sum_{k ascending : a[i][k] and b[k][j]} A_ik B_kj + beta * C_ij
 *
 * over the nonzero triples (i,k,j) (the rank-k updates of Sec. 2.1, the alpha
 * of Algorithm 1; beta*C is the usual GEMM input term). The C tile set S_C is
 * the boolean product of the masks, united with an optional C mask.
 *
 * Storage conventions (all entry points):
 *   - Every stored tile is row-major and contiguous; its leading dimension is its
 *     column-block size. A tile of A is r_i x q_k, of B q_k x c_j, of C r_i x c_j.
 *   - Tiles live in caller-owned arenas (one double array per matrix). Offset
 *     tables are int64 element offsets into the arena, row-major over the tile
 *     grid (a_off: M x K, b_off: K x N, c_off: M x N), -1 for an absent tile.
 *     Offsets of present tiles must be even (every tile 16-byte aligned).
 *   - Block sizes are >= 0; a zero-size block is allowed.
 *   - beta == 0 never reads C (NaN already in C is ignored).
 *
 * Ownership: the caller owns A, B, C and the offset tables. A plan owns its
 * device task tables and its work buffers (the split modes' slice arenas)
 * until bsmm_destroy.
 *
 * Errors: every entry point returns a bsmm_status and never throws or aborts;
 * bsmm_last_error() gives a message for the calling thread. Kernels never trap:
 * bounded waits and checks set a device error word that bsmm_status_device
 * reads.
 *
 * Streams: entry points taking `stream` accept a cudaStream_t passed as void*
 * (NULL = the legacy default stream). They are asynchronous with respect to the
 * host unless stated otherwise, and never synchronise the device.
 */
#ifndef BSMM_H
#define BSMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsmm_plan_s* bsmm_plan_t;

typedef enum {
  BSMM_OK = 0,
  BSMM_ERR_INVALID = 1,      /* bad argument, layout, size or mask */
  BSMM_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  BSMM_ERR_NOMEM = 3,        /* host or device allocation failed */
  BSMM_ERR_TIMEOUT = 4,      /* a kernel's bounded wait ran out (device error word) */
  BSMM_ERR_UNSUPPORTED = 5,  /* a mode or size the library does not handle */
  BSMM_ERR_DEVICE = 6        /* a kernel check failed (device error word) */
} bsmm_status;

typedef enum {
  BSMM_FP64 = 0,        /* plain FP64 tile tasks */
  BSMM_SPLIT_BF16 = 1,  /* Ozaki-style slices stored as bfloat16, tcgen05 tensor cores */
  BSMM_SPLIT_FP16 = 2   /* the same slices stored as float16 */
} bsmm_mode;

typedef enum {
  BSMM_F64 = 0,  /* float64 arenas (every mode) */
  BSMM_F32 = 1,  /* float32 arenas (split modes; bsmm_execute_f32) */
  BSMM_C128 = 2  /* complex double arenas, (re, im) interleaved (split modes; bsmm_execute) */
} bsmm_elem;

typedef enum {
  BSMM_SCHED_FLOPS = 0,   /* order and pack work units by useful flop count */
  BSMM_SCHED_COSTS = 1,   /* by costs given through bsmm_plan_set_costs (e.g. the MLP) */
  BSMM_SCHED_NATURAL = 2  /* no reordering: units in row-major order, dealt round robin */
} bsmm_schedule;

typedef struct {
  int32_t mode;            /* bsmm_mode (default BSMM_FP64) */
  int32_t nslices;         /* split modes: slices per operand, 1..6 (default 6) */
  int32_t schedule;        /* bsmm_schedule (default BSMM_SCHED_FLOPS) */
  int32_t max_ctas;        /* persistent grid size cap; 0 = one per SM (times residency) */
  int32_t debug_checks;    /* 1 = kernels validate offsets against the plan */
  int32_t record_timings;  /* 1 = record per-unit start/end times (bsmm_plan_timings) */
  int32_t profile;         /* 1 = time each internal kernel with CUDA events (bsmm_plan_kernel_ms) */
  int32_t cluster;         /* split modes: CTAs per column-block group, 1, 2 or 4 (0 = 1):
                              the group's CTAs take the same 128-row block at the same time,
                              one 32-column block each, and share its A panel through L2
                              (each CTA loads its own operands). Groups of one suit sparse
                              masks best, where a neighbour's column block is often empty.
                              -1 = the planner's choice: 4, else 2, when the column blocks of
                              every group carry the same tensor-core work to within 0.5% (a
                              dense block pattern), else 1. Plans of one batch need equal
                              sizes, so a plan meant for a batch should fix it. */
  int32_t fp64_tile;       /* FP64 mode: sub-tile edge of a work unit, 32 or 64 (0 = 32) */
  int32_t stages;          /* split modes: depth of the shared-memory ring of 32-deep k chunks
                              (k panels in flight), 2..8 and within the 227 KB shared memory of
                              one CTA (0 = as many as fit next to the C staging buffer) */
  int32_t transa;          /* 1: the A arguments describe the K x M block matrix A' and the
                              product is C = alpha*A'^T*B + beta*C: a_mask and a_off are K x M
                              (row-major over (k,i)) and tile (k,i) is q_k x r_i row-major */
  int32_t transb;          /* 1: the B arguments describe the N x K block matrix B' and the
                              product is C = alpha*A*B'^T + beta*C: b_mask and b_off are N x K
                              and tile (j,k) is c_j x q_k row-major (Sec. 2.1: transposed
                              multiplies such as C = A B^T) */
  int32_t split_scale;     /* split modes: 0 = one power-of-two scale per tile (default);
                              1 = one per row of each A tile and per column of each B tile, for
                              tiles whose rows or columns span many binades (an all-zero row
                              or column takes no part in the maxima that set the accumulator's
                              unit) */
  int32_t ksplit;          /* split k (Sec. 3.2, Fig. 2: the rank-k updates of one C region
                              run as multiply tasks on consecutive pieces of its k-list, each
                              into a partial sum, then one reduction task adds the partials in
                              piece order and applies the epilogue):
                              0 = automatic in the split modes, whose results do not depend on
                                  the cut: a region is cut when the persistent grid would
                                  otherwise idle (few regions, or a region costlier than a
                                  fraction of a CTA's share of the work); no cut in FP64 mode,
                                  so that its rounding stays the plain definition's;
                             -1 = automatic in every mode (FP64 results then depend on the
                                  cut chosen for the machine, within the FP64 error bound);
                              1 = never;
                              n >= 2 = every region's k-list of length L is cut into
                                  n' = min(n, L) pieces, piece p taking list positions
                                  [floor(p L / n'), floor((p+1) L / n')).
                              The split modes' partial sums are exact integers, so their
                              results do not depend on the cut. In FP64 mode the partials
                              are FP64 sums added in piece order (each addition rounded), so
                              a cut region equals the plain result up to that rounding.
                              A region is a work unit's C region: an FP64 sub-tile of one C
                              tile, whose k-list is the tile's; or a split-mode 128-row block
                              times a group of `cluster` 32-column blocks, whose k-list is the
                              inner blocks where both have a stored tile. */
  int32_t elem;            /* bsmm_elem (default BSMM_F64). BSMM_F32 (split modes only; the
                              paper's tile kernel serves single- as well as double-precision
                              types, Sec. 4.3): A, B and C are float32 arenas, offsets count
                              float elements, and A and B tiles start on multiples of 4 (16
                              bytes; a misaligned tile is reported by the device status). The slices
                              and the exact sum are those of the float64 path (float32 values
                              are exact doubles); the sum is rounded once to float32 (ties to
                              even) and the epilogue runs in float32,
                              C = fl32(fl32(alpha*acc) + fl32(beta*C)). Execute with
                              bsmm_execute_f32, bsmm_execute_host or in a batch.
                              BSMM_C128 (split modes; transposed storage and split_scale
                              are taken as for float64): A, B
                              and C are complex double arenas passed to bsmm_execute as double
                              arrays of interleaved (re, im) pairs; offsets count complex
                              elements. Each tile takes one exponent over both parts; the
                              real and imaginary parts of the product are exact sums (of
                              Ar Br - Ai Bi and Ar Bi + Ai Br) rounded once each; alpha and
                              beta are real and scale each part. The tensor cores run the
                              equivalent real product [Ar, -Ai] x [[Br, Bi], [Bi, -Br]] (an
                              inner block of q complex elements is 2q real ones deep) and the
                              useful flop count is 8 r c q per nonzero triple. */
  int32_t store_warps;     /* split modes: the contraction kernel's form. 0 = automatic (with
                              store warps); 2 = with four C store warps (the C store of a
                              unit overlaps the next unit's accumulation); 1 = without (the
                              epilogue warps store). Results do not depend on it. An inner
                              block deeper than the exact FP32 accumulation depth (512 for 6
                              slices, more for fewer) is accumulated in several groups by a
                              form with store warps; with 1 such a plan is BSMM_ERR_UNSUPPORTED.
                              The whole inner dimension may hold up to 2^22 elements. */
  const char* model_path;  /* NULL or "" = no model. Otherwise the path of a cost-model file
                              written by bsmm_mlp_save: bsmm_plan loads it, predicts every work
                              unit's time with it on the GPU and packs the units by those
                              costs (schedule BSMM_SCHED_COSTS). A file that is missing,
                              unreadable, corrupt (checksum), or of another format or feature
                              version leaves the flop-count costs in place (the fallback);
                              bsmm_plan_cost_source tells which was used. The string is read
                              during bsmm_plan only. Results never depend on the schedule. */
} bsmm_options;

typedef enum {
  BSMM_COSTS_FLOPS = 0,  /* useful flop counts (the default, and the model file's fallback) */
  BSMM_COSTS_MODEL = 1,  /* predicted by the cost-model file of bsmm_options.model_path */
  BSMM_COSTS_GIVEN = 2   /* set by bsmm_plan_set_costs or bsmm_plan_predict_costs */
} bsmm_cost_source;

/* Fill *opt with the defaults above. */
void bsmm_options_default(bsmm_options* opt);

/*
 * Build a plan for one block-sparse product structure.
 * Computes S_C (boolean product of a_mask and b_mask, united with c_mask when
 * given), the C-tile-owned work units with their ascending k order, their costs
 * and their packing onto persistent CTAs, and uploads the task tables to the
 * current device. Host inputs only; they are copied, not retained.
 *   M, N, K          number of row, column and inner blocks (>= 0)
 *   row_sizes[M]     r_i >= 0;  col_sizes[N] c_j >= 0;  inner_sizes[K] q_k >= 0
 *   a_mask[M*K]      row-major, nonzero = tile A_ik stored
 *   b_mask[K*N]      row-major, nonzero = tile B_kj stored
 *   c_mask[M*N]      NULL, or extra C tiles to keep in S_C
 *   opt              NULL = defaults
 * Allocates device memory (task tables; slice arenas for the split modes).
 * Returns BSMM_ERR_INVALID for negative sizes or an unknown option value, and
 * BSMM_ERR_UNSUPPORTED for a split mode with more than 8192 inner blocks or more than
 * 2^22 inner elements in all (the 128-bit sums' headroom; a complex inner block of q
 * elements counts 2q), for a split mode with an inner block deeper than the exact FP32
 * accumulation depth (512 real lines for 6 slices) and store_warps = 1, and for
 * float32 or complex elements in FP64 mode.
 */
bsmm_status bsmm_plan(bsmm_plan_t* out, int32_t M, const int32_t* row_sizes, int32_t N,
                      const int32_t* col_sizes, int32_t K, const int32_t* inner_sizes,
                      const uint8_t* a_mask, const uint8_t* b_mask, const uint8_t* c_mask,
                      const bsmm_options* opt);

/*
 * Structure of a plan (host outputs; any pointer may be NULL):
 *   n_ctiles     |S_C|;  n_triples  number of nonzero (i,k,j) triples
 *   useful_flops sum over the triples of 2*r_i*c_j*q_k (8*r_i*c_j*q_k for complex
 *                elements; padding and slices not counted)
 *   c_mask_out   M*N bytes: S_C
 *   n_units      number of work units (each owned by one CTA, fixed k order)
 */
bsmm_status bsmm_plan_query(bsmm_plan_t plan, int64_t* n_ctiles, int64_t* n_triples,
                            double* useful_flops, uint8_t* c_mask_out, int64_t* n_units);

/*
 * Split k of a plan (see bsmm_options.ksplit; host outputs, any pointer may be NULL):
 *   n_regions   regions whose k-list was cut into pieces (each reduced by the extra
 *               reduction kernel that bsmm_execute then launches after the contraction)
 *   n_pieces    work units that are pieces of those regions (their sum over the regions)
 *   pieces      n_units entries: for each work unit, the number of pieces of its region
 *               (1 for a unit that finishes its region)
 */
bsmm_status bsmm_plan_ksplit(bsmm_plan_t plan, int64_t* n_regions, int64_t* n_pieces, int32_t* pieces);

/*
 * Per-unit cost features for the learned cost model (host output, row-major
 * n_units x BSMM_NFEATURES floats) and the unit's flop-count cost. Either pointer may
 * be NULL. With lg(x) = log2(1 + x), a unit's features are, in order: lg(rows),
 * lg(columns), lg(inner blocks in its k-list), lg(inner depth), lg(16-deep steps),
 * lg(useful flops), useful / padded flops, then for the split modes 1, s/6,
 * lg(row tiles), lg(column tiles), lg(32-deep chunks); for FP64 0, 0, 0, 0,
 * lg(16-deep steps). A piece of a cut k-list has the features of its own range. In the
 * split modes the k-list terms are those of the group's slowest CTA (the one with the
 * most 16-deep steps on its own column block's list; with groups of one CTA, the unit's
 * list), since a group costs what its slowest CTA does.
 */
#define BSMM_NFEATURES 12
bsmm_status bsmm_plan_features(bsmm_plan_t plan, float* features, double* flop_costs);

/*
 * Replace the unit costs used by BSMM_SCHED_COSTS and re-pack the units onto the
 * persistent CTAs (longest-processing-time order, greedy least-loaded CTA).
 * costs[n_units] host, > 0. The result bits do not change: only the order.
 */
bsmm_status bsmm_plan_set_costs(bsmm_plan_t plan, const double* costs);

/* Re-pack with an explicit persistent grid size (1..65535; 0 = default). */
bsmm_status bsmm_plan_set_ctas(bsmm_plan_t plan, int32_t ctas);

/*
 * Run the product on `stream` (device pointers):
 *   A, B       device arenas of FP64 tiles (for a plan with complex elements:
 *              interleaved (re, im) pairs, offsets counting complex elements);
 *              a_off (M*K), b_off (K*N) device int64
 *   C          device arena; c_off (M*N) device int64; every tile of S_C must be
 *              present in c_off (checked on the device when debug_checks is set)
 * Asynchronous; the plan's work buffers are reused, so two executes of the same
 * plan must not overlap on different streams.
 */
bsmm_status bsmm_execute(bsmm_plan_t plan, double alpha, const double* A, const int64_t* a_off,
                         const double* B, const int64_t* b_off, double beta, double* C,
                         const int64_t* c_off, void* stream);

/*
 * bsmm_execute for a plan built with elem = BSMM_F32: float32 arenas (offsets in float
 * elements; A and B tiles on multiples of 4), alpha and beta in float32. Same ownership, stream and error
 * behaviour as bsmm_execute; a plan built for float64 elements returns BSMM_ERR_INVALID,
 * and bsmm_execute returns BSMM_ERR_INVALID for a float32 plan.
 */
bsmm_status bsmm_execute_f32(bsmm_plan_t plan, float alpha, const float* A, const int64_t* a_off,
                             const float* B, const int64_t* b_off, float beta, float* C,
                             const int64_t* c_off, void* stream);

/*
 * Same as bsmm_execute (bsmm_execute_f32 for float32 elements) with HOST buffers:
 * copies A, B (and C when beta != 0) and the offset tables to device buffers the plan
 * keeps, runs the product's kernels on `stream`, copies C back, and returns once C is
 * on the host (bsmm_execute_host_async followed by bsmm_host_wait). The arenas hold the
 * plan's element type (bsmm_options.elem): float64, float32, or interleaved complex
 * doubles; a_elems, b_elems, c_elems = arena lengths in those elements. alpha and beta
 * are real (converted to float32 for float32 elements). Pinned host memory makes the
 * copies asynchronous.
 */
bsmm_status bsmm_execute_host(bsmm_plan_t plan, double alpha, const void* A, int64_t a_elems,
                              const int64_t* a_off, const void* B, int64_t b_elems,
                              const int64_t* b_off, double beta, void* C, int64_t c_elems,
                              const int64_t* c_off, void* stream);

/*
 * Host-buffer products in flight (Sec. 3.2: several iterations issued at once, further
 * ones as earlier ones retire, so that data movement of one overlaps the computation of
 * another). bsmm_execute_host_async enqueues one product with the arguments of
 * bsmm_execute_host and returns without waiting: the host-to-device copies run on a
 * copy stream of the plan, the kernels on `stream` (after the copies and after the plan's
 * previous host product), the copy of C back on a second copy stream. Product i uses
 * staging slot i % 2 of the plan (device buffers grown on demand), so the copies of
 * product i + 1 and the copy back of product i - 1 overlap product i's contraction; a
 * product whose slot must grow first waits for that slot's previous product.
 * Ownership: A, B, C and the offset tables stay the caller's and must stay valid and
 * unchanged (C unread) until bsmm_host_wait returns; with pinned memory the copies are
 * asynchronous, with pageable memory they may block the call. Errors: as
 * bsmm_execute_host for the arguments; a failed copy or launch returns BSMM_ERR_CUDA
 * after the plan's streams have been synchronised.
 * bsmm_host_wait: blocks until every host product enqueued on the plan has its C on
 * the host. BSMM_ERR_INVALID for a NULL plan, BSMM_ERR_CUDA if a copy or kernel failed.
 * Device-side error words are read by bsmm_status_device as for bsmm_execute.
 */
bsmm_status bsmm_execute_host_async(bsmm_plan_t plan, double alpha, const void* A, int64_t a_elems,
                                    const int64_t* a_off, const void* B, int64_t b_elems,
                                    const int64_t* b_off, double beta, void* C, int64_t c_elems,
                                    const int64_t* c_off, void* stream);
bsmm_status bsmm_host_wait(bsmm_plan_t plan);

/*
 * Batches: many independent products in one persistent launch. The task set of the
 * paper's Sec. 3.2 extended across products: the work units of every plan are
 * packed together (longest first onto the least-loaded CTA) so one contraction
 * launch runs them all.
 *
 * bsmm_batch_create: `count` plans, all with the same mode, slice count and cluster
 *   size, on one device. The plans must outlive the batch. Allocates device memory.
 *   In the split modes each plan may have its own element type (bsmm_options.elem).
 * bsmm_batch_set_args: per-product arguments as in bsmm_execute, given as host arrays
 *   of length `count` (alpha[i], beta[i], and DEVICE pointers A[i], a_off[i], ...). A[i],
 *   B[i] and C[i] point to arenas of plan i's element type (float64, float32, or
 *   interleaved complex doubles); alpha and beta are real (converted to float32 for
 *   float32 elements). Copied to the device synchronously; call again when any of them
 *   changes.
 * bsmm_batch_execute: issues the kernels of the whole batch on `stream`. FP64: one
 *   contraction launch. Split modes: the products are taken in waves whose slice
 *   workspaces fit in half of L2 (a larger product is a wave of its own); each wave
 *   issues its products' exponent and slicing kernels, then one contraction launch.
 *   Consecutive waves go to `stream` and to a second stream of the batch in turn (the
 *   second forked from `stream` before the first wave and joined back into it after the
 *   last, with events), so a wave's slicing overlaps the end of the previous wave's
 *   contraction; everything enqueued later on `stream` runs after the whole batch. It
 *   allocates, copies and synchronises nothing, so it can be captured into a CUDA
 *   graph and replayed. Products must not overlap in C.
 * bsmm_batch_query: units over the batch, summed useful flops, persistent bins (CTAs
 *   for FP64, clusters for the split modes); pointers may be NULL.
 * bsmm_batch_set_costs: costs[n_units] (> 0, units in plan order) and re-pack.
 * bsmm_batch_status_device: synchronise and return the batch's and the plans' device
 *   error words (cleared).
 */
typedef struct bsmm_batch_s* bsmm_batch_t;
bsmm_status bsmm_batch_create(bsmm_batch_t* out, int32_t count, const bsmm_plan_t* plans);
bsmm_status bsmm_batch_set_args(bsmm_batch_t batch, const double* alpha, const void* const* A,
                                const int64_t* const* a_off, const void* const* B,
                                const int64_t* const* b_off, const double* beta, void* const* C,
                                const int64_t* const* c_off);
bsmm_status bsmm_batch_execute(bsmm_batch_t batch, void* stream);
bsmm_status bsmm_batch_query(bsmm_batch_t batch, int64_t* n_units, double* useful_flops, int32_t* bins);

/* Number of kernels the batch's most recent bsmm_batch_execute launched (0 before the
 * first): per wave the products' slicing kernels and one contraction launch, plus one
 * split-k reduction per product that cut a k-list (FP64: one contraction launch). */
bsmm_status bsmm_batch_kernels(bsmm_batch_t batch, int32_t* kernels);
bsmm_status bsmm_batch_set_costs(bsmm_batch_t batch, const double* costs);
bsmm_status bsmm_batch_status_device(bsmm_batch_t batch, void* stream);
void bsmm_batch_destroy(bsmm_batch_t batch);

/*
 * The whole batch in one call (the same work as bsmm_batch_create, bsmm_batch_set_args
 * and bsmm_batch_execute): `count` plans (same rules as bsmm_batch_create) with their
 * per-product arguments as in bsmm_batch_set_args, launched on `stream`. The library
 * keeps the batch objects of its last 4 plan lists (keyed by the plans, never by
 * addresses that a later plan could reuse) with the arguments last uploaded to each:
 * the first call for a plan list creates the batch (allocation, synchronous uploads),
 * a call with new arguments uploads them after synchronising `stream` (the previous
 * launch's argument table is then no longer read), and a call with the plans and
 * arguments of the previous one only enqueues kernels, so such calls can be captured
 * into a CUDA graph once one call has set the batch up. Calls that overlap on
 * different streams with the same plan list race. The plans must outlive the calls;
 * a destroyed plan's entry is released when it becomes the least recently used.
 */
bsmm_status bsmm_execute_batch(int32_t count, const bsmm_plan_t* plans, const double* alpha, const void* const* A,
                               const int64_t* const* a_off, const void* const* B, const int64_t* const* b_off,
                               const double* beta, void* const* C, const int64_t* const* c_off, void* stream);

/*
 * Autotuning of a batch's launch shape. The paper has no counterpart (its tile kernel
 * is a library DGEMM); these pick, by measurement, the knobs that set the contraction's
 * work-unit shape and pipeline depth.
 *
 * bsmm_tune_point: one candidate. Split modes: `cluster` CTAs per column-block group
 *   (a work unit is 128 rows x 32*cluster columns), `stages`, the depth of the
 *   shared-memory ring (k panels in flight), and `store_warps`, the contraction kernel's
 *   form (as bsmm_options.store_warps: 0 = the planner's choice, 1 = without C store
 *   warps, 2 = with them). FP64 mode: `fp64_tile`, the sub-tile edge of a work unit (32
 *   or 64). Fields that do not apply to the mode must be 0.
 * bsmm_tune_space: the candidate list for a mode and slice count (split: cluster
 *   1, 2, 4 x every ring depth from 2 that fits one CTA's shared memory x both kernel
 *   forms; FP64: 32 and 64). Writes at most `cap` points to `out` (nullable) and their
 *   total to *count.
 * bsmm_batch_autotune: times the batch (bsmm_batch_set_args called before) under each
 *   candidate: every product is re-planned with that candidate's options (flop-count
 *   schedule; costs set earlier do not carry over), run once to warm up, then `reps`
 *   times (>= 1) between CUDA events on `stream`; the median is the candidate's time.
 *   Each run writes a scratch C of the caller's C extent, allocated here and freed on
 *   return, so the caller's C is not touched. The batch then keeps its products
 *   re-planned under the fastest candidate (it owns those plans; the plans given to
 *   bsmm_batch_create are left as they were) with the arguments already set. Those
 *   new plans share the slice workspace of the plans given to bsmm_batch_create, which
 *   must therefore still outlive the batch and must not run while the batch runs.
 *   chosen (nullable) receives the fastest candidate's index; ms (nullable, n entries)
 *   the median times in milliseconds, +infinity for a candidate that does not fit or
 *   whose plans are refused (e.g. the form without store warps for a batch with inner
 *   blocks deeper than the exact accumulation depth).
 *   Synchronises `stream`. Fails with BSMM_ERR_UNSUPPORTED when no candidate fits.
 */
typedef struct {
  int32_t cluster;    /* split modes: 1, 2 or 4 */
  int32_t stages;     /* split modes: 2..8 (0 = as many as fit) */
  int32_t fp64_tile;  /* FP64 mode: 32 or 64 */
  int32_t store_warps; /* split modes: 0, 1 or 2 (see bsmm_options.store_warps) */
} bsmm_tune_point;
bsmm_status bsmm_tune_space(int32_t mode, int32_t nslices, bsmm_tune_point* out, int32_t cap, int32_t* count);

/*
 * Host scheduling utilities: the planner's own packing and split-k choice, on host arrays
 * (no device needed).
 *
 * bsmm_schedule_lpt: longest-processing-time packing of n units with cost[n] (> 0) onto
 *   `bins` persistent CTAs (Sec. 3.2's task scheduler made static): units by descending
 *   cost (ties in unit order), each to the least-loaded bin (ties to the lowest bin); each
 *   bin then lists its units in ascending unit order. Outputs in CSR form: ptr[bins + 1]
 *   and units[n] (bin b runs units[ptr[b] .. ptr[b+1])), and, if makespan is not NULL,
 *   the largest bin load.
 * bsmm_schedule_pieces: how many pieces the planner cuts each of n units into (split k,
 *   Sec. 3.2 Fig. 2) given its cost[n] (> 0), its k-list length len[n] (>= 0), the bin
 *   count, the per-piece overhead charged in the simulation (in cost units) and the
 *   ksplit option (0 automatic, 1 never, >= 2 forced; see bsmm_options.ksplit).
 *   pieces[n] receives values in 1 .. max(1, len[i]).
 * Both return BSMM_ERR_INVALID for NULL arrays, n < 0, bins < 1, or a cost <= 0.
 */
bsmm_status bsmm_schedule_lpt(int64_t n, const double* cost, int32_t bins, int32_t* ptr, int32_t* units,
                              double* makespan);
bsmm_status bsmm_schedule_pieces(int64_t n, const double* cost, const int64_t* len, int32_t bins,
                                 double overhead, int32_t ksplit, int32_t* pieces);
bsmm_status bsmm_batch_autotune(bsmm_batch_t batch, int32_t n, const bsmm_tune_point* candidates, int32_t reps,
                                void* stream, int32_t* chosen, float* ms);

/*
 * bsmm_batch_autotune_cached: the tuning with a persistent cache. The cache is a JSON
 * file at cache_path (format "bsmm-tune", version 1, one entry per line) keyed by the GPU's
 * name, the mode and the slice count. When it holds an entry for this batch's key that is
 * still one of bsmm_tune_space's candidates, the batch is re-planned under it without any
 * timing (*from_cache = 1). Otherwise (no file, another format or version, no entry, a
 * stale candidate) the batch is tuned over the whole bsmm_tune_space with `reps` timed runs
 * per candidate (as bsmm_batch_autotune), and the fastest candidate and its time are
 * written into the file, other keys kept (*from_cache = 0). *chosen (nullable) receives
 * the candidate used. The file is replaced atomically; BSMM_ERR_INVALID when it cannot be
 * written.
 */
bsmm_status bsmm_batch_autotune_cached(bsmm_batch_t batch, const char* cache_path, int32_t reps, void* stream,
                                       bsmm_tune_point* chosen, int32_t* from_cache);

/*
 * Learned task-cost model. The paper tolerates the load variation of nonuniform
 * blocks (Sec. 4.4, Table 1) with many small tasks and a dynamic scheduler (Sec.
 * 3.2); here work units are packed statically onto persistent CTAs, so the packing
 * needs cost estimates. A small MLP (BSMM_NFEATURES inputs from bsmm_plan_features,
 * two tanh layers of 32, one output = log unit time) is trained on the GPU from
 * measured unit times (bsmm_plan_timings) and its predictions replace the flop-count
 * costs. Results never depend on it (only the order of the units).
 *
 * Parameters: one float vector of bsmm_mlp_num_params() entries, in this order:
 * W1[32][F], b1[32], W2[32][32], b2[32], w3[32], b3. Inputs are standardised with the
 * model's stored means/deviations and the output de-standardised (bsmm_mlp_set_norm,
 * or set from the data by bsmm_mlp_fit).
 *
 * bsmm_mlp_create      deterministic initialisation from `seed`; allocates device memory
 * bsmm_mlp_loss_grad   X[n x F], t[n] device (raw features, raw log times): mean squared
 *                      error of the standardised prediction and its gradient (host
 *                      outputs, grad may be NULL); synchronises `stream`
 * bsmm_mlp_fit         sets the standardisation from (X, t), then `steps` full-batch Adam
 *                      steps (beta1 0.9, beta2 0.999, eps 1e-8) at rate `lr`; reductions
 *                      run in a fixed order, so training is reproducible bit for bit;
 *                      *final_loss (host, may be NULL) after the last step
 * bsmm_mlp_predict     y[n] device = predicted log time for X (device), asynchronous
 * bsmm_plan_predict_costs  predicts every unit of `plan` and re-packs it with the
 *                      predicted times as costs (bsmm_plan_set_costs); synchronises
 */
typedef struct bsmm_mlp_s* bsmm_mlp_t;
bsmm_status bsmm_mlp_create(bsmm_mlp_t* out, uint64_t seed);
int32_t bsmm_mlp_num_params(void);
bsmm_status bsmm_mlp_set_params(bsmm_mlp_t mlp, const float* params, int64_t n);
bsmm_status bsmm_mlp_get_params(bsmm_mlp_t mlp, float* params, int64_t n);
bsmm_status bsmm_mlp_set_norm(bsmm_mlp_t mlp, const float* x_mean, const float* x_sd, float y_mean, float y_sd);
bsmm_status bsmm_mlp_get_norm(bsmm_mlp_t mlp, float* x_mean, float* x_sd, float* y_mean, float* y_sd);
bsmm_status bsmm_mlp_loss_grad(bsmm_mlp_t mlp, const float* X, const float* t, int64_t n, float* loss,
                               float* grad, void* stream);
bsmm_status bsmm_mlp_fit(bsmm_mlp_t mlp, const float* X, const float* t, int64_t n, int32_t steps, float lr,
                         float* final_loss, void* stream);
bsmm_status bsmm_mlp_predict(bsmm_mlp_t mlp, const float* X, int64_t n, float* y, void* stream);
bsmm_status bsmm_plan_predict_costs(bsmm_plan_t plan, bsmm_mlp_t mlp, void* stream);
/*
 * Cost-model files (the learned schedule's checkpoint). bsmm_mlp_save writes the
 * parameters and the standardisation of `mlp` to `path` (created or replaced); the
 * file is binary, little-endian: the 8 bytes "BSMMMLP\0", uint32 format version (1),
 * uint32 feature version (BSMM_FEATURE_VERSION: the order and meaning of the
 * bsmm_plan_features columns; 2 since the split modes' k-list terms are the slowest
 * CTA's of a group), uint32 F, uint32 hidden width, uint32 parameter count,
 * the float32 parameters, x means[F], x deviations[F], y mean, y deviation, then a
 * uint64 FNV-1a checksum of every byte before it. bsmm_mlp_load creates a model from
 * such a file (BSMM_ERR_INVALID for a missing or unreadable file, a bad checksum, or
 * another format, feature version or shape). Adam state is not saved.
 */
#define BSMM_FEATURE_VERSION 2
bsmm_status bsmm_mlp_save(bsmm_mlp_t mlp, const char* path);
bsmm_status bsmm_mlp_load(bsmm_mlp_t* out, const char* path);
/* Where the plan's current unit costs came from (bsmm_cost_source). */
bsmm_status bsmm_plan_cost_source(bsmm_plan_t plan, int32_t* source);

/*
 * The contraction launch the planner chose for a plan (host outputs; any may be NULL):
 * cluster = CTAs per column-block group (1, 2 or 4; bsmm_options.cluster = -1 resolved),
 * store_warps = 1 when the kernel form has C store warps, epi_walk = 1 when the epilogue
 * walks its own k lists for the accumulation groups (long k lists, 3 to 6 slices with
 * store warps) rather than taking the MMA warps' descriptors, stages = depth of the
 * shared-memory ring, ctas = persistent CTAs (FP64) or groups (split modes) of a launch.
 * FP64 plans report cluster 1, store_warps 0, epi_walk 0, stages 0. BSMM_ERR_INVALID for
 * a NULL plan.
 */
bsmm_status bsmm_plan_form(bsmm_plan_t plan, int32_t* cluster, int32_t* store_warps, int32_t* epi_walk,
                           int32_t* stages, int32_t* ctas);
void bsmm_mlp_destroy(bsmm_mlp_t mlp);

/*
 * Synchronise `stream` and return the plan's device error word as a status
 * (BSMM_OK, BSMM_ERR_TIMEOUT or BSMM_ERR_DEVICE), clearing it.
 */
bsmm_status bsmm_status_device(bsmm_plan_t plan, void* stream);

/*
 * Diagnostics for the kernels' bounded waits (no GPU fault, trap or hang): runs a one-block
 * kernel whose waits can never be satisfied (mbarriers that no thread arrives at). One
 * thread waits with a limit of limit_ns nanoseconds (1e6 .. 1e9), runs out, sets the error
 * word and the abort flag; two warps waiting with a 20x longer limit leave as soon as they
 * see the flag -- the timeout and abort protocol of the contraction kernel. Synchronises
 * the stream. Returns BSMM_ERR_TIMEOUT when the waits ran out as designed (the device and
 * the context stay usable), BSMM_OK if they did not, BSMM_ERR_INVALID for a limit out of
 * range, BSMM_ERR_CUDA when a CUDA call failed.
 */
bsmm_status bsmm_selftest_wait(int64_t limit_ns, void* stream);

/*
 * Per-unit timing records of the last execute with record_timings set:
 * start_ns[n_units], end_ns[n_units] (device %globaltimer, host outputs, either
 * may be NULL) and the CTA each unit ran on (cta[n_units], may be NULL). A split-mode
 * unit of a column-block group of several CTAs (bsmm_options.cluster) starts when the
 * group's first CTA starts it, and end_ns - start_ns is the longest time any CTA of the
 * group spent on it (the group's cost in the packing). Synchronises the device.
 */
bsmm_status bsmm_plan_timings(bsmm_plan_t plan, int64_t* start_ns, int64_t* end_ns, int32_t* cta);

/*
 * Device time of each internal kernel of a plan built with profile = 1, measured with
 * CUDA events recorded on the execute's stream around every launch: the mean over the
 * executes since the previous call of this function (the plan keeps the events of its
 * last 64 executes; with no execute since the previous call, the last execute's times
 * again). So a caller can run many executes without any synchronisation and read their
 * mean once afterwards. ms[max_n] host output (kernel order: split modes = exponents,
 * slicing, contraction[, split-k reduction]; FP64 = contraction[, reduction]);
 * *count = kernels per execute. Synchronises on the last event. BSMM_ERR_INVALID when
 * the averaged executes launched different kernel counts.
 */
bsmm_status bsmm_plan_kernel_ms(bsmm_plan_t plan, float* ms, int32_t max_n, int32_t* count);

/*
 * Diagnostics: arithmetic rates of the current GPU, measured. The FP64 ones are the
 * denominators of the FP64 path's roofline (the paper's tile kernel is an FP64 DGEMM,
 * Sec. 4.1); the INT8 one is the rate an integer variant of the split method could use.
 * Runs three kernels on every SM, three times each, on `stream` (the fastest pass
 * counts) and synchronises it. rates[3] host output: rates[0] = FP64 fused multiply-adds on the FP64
 * units, TFLOP/s (16 independent chains per thread); rates[1] = the FP64 tensor-core
 * instruction mma.sync m8n8k4, TFLOP/s; rates[2] = the INT8 tensor-core instruction
 * mma.sync m16n8k32 (s8 x s8 -> s32), TOP/s (sm_103a has no INT8 kind of tcgen05.mma).
 * Allocates and frees a small scratch buffer.
 */
bsmm_status bsmm_measure_rates(double* rates, void* stream);

/*
 * One dense tile task without any allocation (the paper has no counterpart: it is
 * an addition for callers that cannot allocate device memory where they need the
 * product -- for example code that runs while its allocator is locked or a graph
 * is being built around it, or a host that reserved all device memory up front).
 *
 * Computes C = alpha * A*B + beta * C for one m x k tile A, k x n tile B and m x n
 * tile C (row-major, contiguous, device pointers, 16-byte aligned) with the 6-or-
 * fewer-slice split-bfloat16 method of bsmm_execute: the same bits as a plan of the
 * 1 x 1 x 1 tiling (m), (n), (k) in BSMM_SPLIT_BF16 mode. beta == 0 does not read C;
 * k == 0 gives C = beta * C (A and B may then be NULL).
 * Limits: 0 <= m, n <= 256, 0 <= k <= 512, nslices in 1..6; anything else returns
 * BSMM_ERR_INVALID before anything runs (every k up to 512 is within the exact
 * accumulation depth of every slice count, so no depth is refused beyond that).
 *
 * Scratch: a file-scope device array of about 3.2 MB inside the library, held by
 * every GPU that loads the library until the process exits; no cudaMalloc,
 * cudaFree or other allocating call is made. Each call looks up the array's address
 * on the current device (cudaGetSymbolAddress); the first call on a device loads the
 * library's code there and should come before any stream capture. All calls share
 * the array and leave their contents in it, so calls that overlap on the GPU
 * (several streams or host threads) race: the caller must serialise them.
 * The call enqueues its kernels on `stream`, reads the device error word back from
 * the array on that stream and returns once the product is complete:
 * BSMM_ERR_DEVICE for a non-finite input element, BSMM_ERR_TIMEOUT when a kernel
 * wait ran out (C is then incomplete), BSMM_ERR_CUDA for a failed CUDA call.
 */
bsmm_status bsmm_split_tile_noalloc(int32_t m, int32_t n, int32_t k, int32_t nslices, double alpha,
                                    const double* A, const double* B, double beta, double* C, void* stream);

/* Thread-local message for the last failing call ("" if none). */
const char* bsmm_last_error(void);

/* Release a plan and its device memory. NULL-safe. */
void bsmm_destroy(bsmm_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* BSMM_H */
