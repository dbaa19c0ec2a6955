/*
 * sparsefusion.h - C ABI of the GB300 (sm_103a) sparse-fusion library.
 *
 * Sparse fusion (Cheshmi, Strout, Mehri Dehnavi, "Composing Loop-carried Dependence with
 * Other Loops", arXiv 2111.12238) runs two sparse kernels, at least one of which has
 * loop-carried dependences, as one parallel pass. An inspector (§2.2) builds a fused
 * schedule from the two kernels' dependence DAGs and the inter-kernel dependence matrix F;
 * an executor (§2.3, Figure 4) runs the fused schedule. This header exposes that
 * inspector-executor split (the driver of Figure 3b: intra_DAG, inter_DAG, compute_reuse,
 * scheduling, then fused_code) as plain C calls.
 *
 * Conventions for every call:
 *  - Array arguments are DEVICE pointers owned by the caller unless stated otherwise;
 *    they must stay valid until the stream work that uses them has finished.
 *  - CSR patterns: int32 rowptr[n_rows+1] with rowptr[0] = 0 and rowptr[n_rows] = nnz,
 *    int32 colidx[nnz] strictly ascending within each row. Lower-triangular operands
 *    (SpTRSV / SpIC0 patterns) hold only columns <= row and every row holds its diagonal
 *    as its LAST entry. nnz < 2^31.
 *  - Value arrays follow their pattern's CSR order. Dense blocks (right-hand sides,
 *    solutions) are n x k ROW-MAJOR (the k values of one row are contiguous).
 *  - Element type is chosen per call by sf_dtype: SF_F64 = double, SF_F32 = float.
 *  - Calls that launch device work are stream-ordered and asynchronous; `stream` is a
 *    cudaStream_t (NULL = legacy default stream). Device-side failures (a timed-out
 *    dependence wait, an incomplete-Cholesky breakdown, a non-finite pivot) are recorded
 *    in the schedule and reported by sf_schedule_check.
 *  - Errors never trap or abort: every call returns an sf_status; sf_last_error_detail
 *    gives a human-readable reason for the last failure on the calling thread.
 */
#ifndef SPARSEFUSION_H
#define SPARSEFUSION_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SF_OK = 0,
    SF_ERR_INVALID_ARG = 1,  /* a NULL pointer, size or option out of range          */
    SF_ERR_BAD_PATTERN = 2,  /* CSR pattern violates the conventions above           */
    SF_ERR_CUDA = 3,         /* a CUDA runtime call failed                            */
    SF_ERR_OOM = 4,          /* device allocation failed                              */
    SF_ERR_TIMEOUT = 5,      /* a dependence wait in a kernel exceeded its time limit */
    SF_ERR_BREAKDOWN = 6,    /* zero fill-in IC hit a non-positive pivot               */
    SF_ERR_NONFINITE = 7,    /* a diagonal entry used as divisor was zero             */
    SF_ERR_UNSUPPORTED = 8   /* the combination of pair / dtype / k is not provided   */
} sf_status;

/* The fused kernel pairs (Table 2 of the paper, restated in CSR form):
 *  SF_TRSV_SPMV  combination 4: x = L^-1 b (SpTRSV), then y = M x (SpMV). F = pattern(M).
 *  SF_IC0_TRSV   combination 5: L L^T ~ A by zero fill-in IC (SpIC0), then y = L^-1 b.
 *                F = I: row i of the solve waits for row i of the factor.
 *  SF_SPMV_TRSV  combination 2: r = b - A x_in (SpMV), then z = L^-1 r with L = tril(A)
 *                passed as its own CSR (one Gauss-Seidel half-sweep). F = I.
 *  SF_TRSV_TRSV  combination 1: x = L^-1 b, then z = L^-1 x with the same L. F = I.
 *  SF_ILU0_TRSV  combination 6: L U ~ A by zero fill-in ILU (SpILU0, row-oriented IKJ form on
 *                A's pattern, L unit lower), then y = L^-1 b. F = I. sf_inspect takes L =
 *                the pattern of tril(A) (the DAG) and M = A (square, every diagonal present,
 *                at most 256 entries per row).
 * Single-kernel schedules, the building blocks of the unfused two-launch path:
 *  SF_TRSV       x = L^-1 b alone.
 *  SF_IC0        the zero fill-in IC factor alone.                                      */
typedef enum {
    SF_TRSV_SPMV = 0,
    SF_IC0_TRSV = 1,
    SF_SPMV_TRSV = 2,
    SF_TRSV = 3,
    SF_IC0 = 4,
    SF_TRSV_TRSV = 5,
    SF_ILU0_TRSV = 6
} sf_pair;

typedef enum { SF_F64 = 0, SF_F32 = 1 } sf_dtype;

/* A CSR pattern (no values). rowptr / colidx are device pointers owned by the caller;
 * sf_inspect copies what it needs, so they may be freed once sf_inspect returns. */
typedef struct {
    int32_t n_rows;
    int32_t n_cols;
    int64_t nnz;
    const int32_t *rowptr;
    const int32_t *colidx;
} sf_csr;

/* Options; a zero-initialised struct selects every default. */
#define SF_WANT_ADJOINT 0x1u /* also build the transposed schedule used by sf_adjoint */
#define SF_EPOCH_FLAGS 0x2u  /* publish rows through per-row epoch flags even when k = 1
                                (by default a single right-hand side is published by its value:
                                the dependency vector is reset to an all-ones NaN pattern
                                before each launch and a consumer waits for its entry to change) */
#define SF_DYNAMIC_QUEUE 0x4u /* warps draw partitions from a ticket counter instead of the
                                default static round robin over a cooperative launch */
typedef struct {
    int64_t part_cost_target; /* C of the partition cut (§3.1 vertex cost); 0 = auto  */
    int32_t lanes_per_row;    /* lanes of a warp working on one row: 1..32 (pow2); 0 = auto */
    int32_t rhs_tile;         /* right-hand-side columns handled side by side; 0 = auto */
    int32_t g2_placement;     /* separated schedules (SpTRSV -> SpMV forward, SpMV -> SpTRSV
                                 adjoint): wavefront of the second kernel's vertices, which
                                 are sinks of the joint DAG (slack, §3.2.2). 0: earliest;
                                 -1: last wavefront; d > 0: delayed by d wavefronts (at most
                                 to the last). Ignored by paired schedules. */
    int32_t blocks_per_sm;    /* resident executor blocks per SM; 0 = occupancy limit  */
    uint64_t timeout_ns;      /* limit of one dependence wait on the GPU; 0 = 2 s    */
    uint32_t flags;           /* SF_WANT_ADJOINT | SF_EPOCH_FLAGS | SF_DYNAMIC_QUEUE  */
    int32_t team_lanes;       /* lanes of the unit that runs one partition: 8 or 32
                                 (several teams per warp); 0 = 32 */
    int32_t block_rows;       /* rows per block of the row-block executor; 0 = min(8192, n) */
    int32_t exec_mode;        /* 0 (automatic) and 1: partitions; 2: row blocks; 3: row blocks
                                 with warp-specialised loading (cp.async); 4: row blocks with
                                 packed records and bulk copies (2-4: k = 1 with value flags;
                                 the call fails when a block does not fit in shared memory);
                                 5: one CTA per instance (the whole system, or each instance
                                 of a batch) runs its SpTRSV level segment by level segment
                                 between CTA barriers, with x (and the order and L when they
                                 fit) in shared memory; the SpMV rows of a single system run
                                 on helper CTAs of the same cooperative launch, fed x by value
                                 (bounded waits), those of a batch on the instance's CTA after
                                 its solve (SF_TRSV_SPMV forward and SF_TRSV, k = 1;
                                 block_rows is then ignored).
                                 The autotuner chooses between them. */
} sf_options;

/* Opaque fused schedule (§3.1 "fused partitioning", the FusedSchedule of Figure 3b).
 * Owned by the library; device memory it holds is released by sf_schedule_destroy. */
typedef struct sf_schedule sf_schedule;

/* Inspector (§2.2, §3): build the fused schedule of `pair` on the GPU.
 *  L: the lower-triangular pattern (SpTRSV's matrix; tril(A) for SF_IC0_TRSV, SF_IC0 and
 *     SF_SPMV_TRSV). Square.
 *  M: SF_TRSV_SPMV: the SpMV operand (n x n); SF_SPMV_TRSV: A (n x n); otherwise NULL.
 * Builds the joint DAG (the SpTRSV DAG is the pattern of L, §2.2; F as listed for
 * sf_pair), its wavefront levels by parallel Kahn peeling, the linear order by
 * (level, kernel, row), and contiguous partitions of that order cut by vertex cost
 * (§3.1). Synchronises `stream` before returning. On success *out owns a new schedule;
 * on failure *out is NULL. The inspector's temporary device memory comes from a stream-ordered
 * memory pool of the library (one per device, created on first use), which keeps up to 1 GiB
 * of freed memory for later inspections instead of returning it to the driver. */
sf_status sf_inspect(sf_pair pair, const sf_csr *L, const sf_csr *M, const sf_options *opt,
                     void *stream, sf_schedule **out);

/* Batched inspector: `count` independent instances (host arrays Ls[count], Ms[count] of
 * patterns with device pointers; Ms may be NULL when the pair has no M) scheduled as one
 * block-diagonal system in a single queue ordered by (level, instance, row). Value
 * arrays and dense blocks passed to sf_execute / sf_adjoint for a batched schedule are
 * the instances' arrays concatenated in instance order. */
sf_status sf_inspect_batched(sf_pair pair, int32_t count, const sf_csr *Ls, const sf_csr *Ms,
                             const sf_options *opt, void *stream, sf_schedule **out);

/* Executor (§2.3): one persistent launch that runs the fused schedule.
 *  L_vals: SF_TRSV_SPMV, SF_SPMV_TRSV, SF_TRSV, SF_TRSV_TRSV: values of L; SF_IC0_TRSV, SF_IC0:
 *          the values of tril(A) to factor (input, not modified); SF_ILU0_TRSV: NULL.
 *          SF_SPMV_TRSV accepts NULL when L's pattern is tril(A)'s (checked at inspection) and
 *          SF_EPOCH_FLAGS is off: L = tril(A) is then read from A's rows (shared storage, one
 *          pass over A's row gives both r_i and the solve's sum).
 *  M_vals: SF_TRSV_SPMV: values of M; SF_SPMV_TRSV, SF_ILU0_TRSV: values of A; otherwise NULL.
 *  x_in:   SF_SPMV_TRSV only: the SpMV operand (n x k); otherwise NULL.
 *  b:      right-hand side (n x k); NULL for SF_IC0.
 *  y:      result (n x k): y = M L^-1 b, y = L^-1 b (IC0 or ILU0 factor L), z = L^-1 (b - A x_in),
 *          z = L^-1 L^-1 b for SF_TRSV_TRSV, or x = L^-1 b for SF_TRSV; NULL for SF_IC0.
 *  x_save: optional. SF_TRSV_SPMV, SF_TRSV_TRSV: receives the intermediate x = L^-1 b (n x k),
 *          needed by sf_adjoint. SF_IC0_TRSV / SF_IC0: receives the factor values on L's pattern
 *          (required for SF_IC0). SF_ILU0_TRSV: receives the factor on A's pattern (the strictly
 *          lower part of the unit lower L, then U with its diagonal). When NULL a library-owned
 *          buffer is used; it is allocated on the first call that needs it, so make one such
 *          call before capturing the stream into a CUDA graph.
 *  k:      number of right-hand sides, 1 <= k <= 1024. Unless SF_EPOCH_FLAGS was given, the
 *          vectors that carry the dependences (x_save or its library-owned stand-in for
 *          SF_TRSV_SPMV and SF_TRSV_TRSV, y for SF_TRSV, SF_SPMV_TRSV, SF_TRSV_TRSV, SF_IC0_TRSV
 *          and SF_ILU0_TRSV, the factor for the IC0 and ILU0 pairs) are first filled with the
 *          all-ones pattern on `stream` and every value is published by its own store; a
 *          result whose bits equal that pattern is stored as the canonical NaN instead (both
 *          are NaN). SF_ILU0_TRSV always publishes values this way.
 * Concurrent calls with the same schedule on different streams race; calls on one
 * stream are ordered. Returns after enqueueing the launch. */
sf_status sf_execute(const sf_schedule *sch, sf_dtype dt, int32_t k, const void *L_vals,
                     const void *M_vals, const void *x_in, const void *b, void *y, void *x_save,
                     void *stream);

/* Adjoint executor (not in the paper): gradients of the fused pair as one fused pass over
 * the transposed schedule (requires SF_WANT_ADJOINT at inspection).
 *  SF_TRSV_SPMV (y = M L^-1 b, x = L^-1 b): saved = x, gy = dL/dy. Computes u = M^T gy
 *    and lam = L^-T u; writes gb = lam, and when non-NULL gL_vals (pattern of L) with
 *    gL_ij = -sum_c lam_ic x_jc and gM_vals (pattern of M) with gM_ij = sum_c gy_ic x_jc.
 *    gx_in must be NULL.
 *  SF_SPMV_TRSV (z = L^-1 (b - A x_in)): saved = z, gy = dL/dz. Computes lam = L^-T gz;
 *    writes gb = lam, and when non-NULL gx_in = -A^T lam, gL_vals with gL_ij =
 *    -sum_c lam_ic z_jc, gM_vals (pattern of A) with gA_ij = -sum_c lam_ic x_in_jc.
 * Launches: the values of L^T and M^T (A^T) are first gathered into transposed order in
 * library-owned buffers, then the fused pass runs on the transposed schedule, then the value
 * gradients are written by a streaming pass over the entries of L and M (A).
 * Other pairs return SF_ERR_UNSUPPORTED. Same stream and ownership rules as sf_execute. */
sf_status sf_adjoint(const sf_schedule *sch, sf_dtype dt, int32_t k, const void *L_vals,
                     const void *M_vals, const void *x_in, const void *saved, const void *gy,
                     void *gb, void *gx_in, void *gL_vals, void *gM_vals, void *stream);

/* Plain SpMV building block of the unfused path: y = M x (b == NULL) or y = b - M x.
 * M is n_rows x n_cols; x is n_cols x k, b and y are n_rows x k. Asynchronous. */
sf_status sf_spmv(sf_dtype dt, int32_t k, const sf_csr *M, const void *M_vals, const void *x,
                  const void *b, void *y, void *stream);

/* Synchronises `stream`, then reports (and clears) the first device-side failure recorded
 * by executions of this schedule: SF_ERR_TIMEOUT, SF_ERR_BREAKDOWN or SF_ERR_NONFINITE;
 * *row (may be NULL) receives the row involved, or -1. */
sf_status sf_schedule_check(const sf_schedule *sch, void *stream, int32_t *row);

/* Host-side validity check of the schedule (§3.2: every intra- and inter-kernel
 * dependence must be honoured): copies the order, partitions and patterns to the host
 * and checks that the order is a permutation of the joint DAG's vertices, that every DAG
 * and F edge points forward in it, and that the partitions are contiguous and cover it.
 * Checks the adjoint schedule too when present. Synchronous. SF_OK when valid,
 * SF_ERR_BAD_PATTERN otherwise. */
sf_status sf_validate(const sf_schedule *sch);

/* Depth (number of wavefronts of the joint DAG), number of partitions and number of
 * joint-DAG vertices of the forward schedule. Host memory outputs; any may be NULL. */
sf_status sf_schedule_info(const sf_schedule *sch, int32_t *depth, int32_t *n_parts,
                           int64_t *n_items);

/* Extended description of a schedule. */
typedef struct {
    int32_t pair, n, k_hint, instances;
    int32_t depth, n_parts;            /* forward schedule */
    int64_t n_items;
    int32_t adj_depth, adj_n_parts;    /* adjoint schedule, 0 when absent */
    int64_t adj_n_items;
    int32_t lanes_per_row, rhs_tile;
    int64_t part_cost_target, adj_part_cost_target;
    int32_t packing;                   /* 0 separated, 1 interleaved (paired rows) */
    int32_t blocks_per_sm;             /* 0 = occupancy limit */
    int32_t epoch_flags;               /* 1 when SF_EPOCH_FLAGS is in effect */
    int32_t dynamic_queue;             /* 1 when SF_DYNAMIC_QUEUE is in effect */
    double reuse_ratio;                /* Table 2 / §2.2 reuse ratio of the pair */
    double inspect_ms;                 /* wall time of the inspector call */
    int64_t wide_cost, adj_wide_cost;  /* vertices of cost above this run on a whole warp in a
                                          partition of their own (0: none) */
    int64_t cost_total, adj_cost_total; /* sum of the vertex costs c(v) of each schedule */
    int32_t adj_lanes_per_row, reserved2;
    int32_t team_lanes, adj_team_lanes;
    int32_t block_rows, n_blocks, adj_block_rows, adj_n_blocks;
    int32_t exec_mode, adj_exec_mode, block_lanes, adj_block_lanes;
    int32_t block_segments, adj_block_segments;   /* level segments of the row-block order */
    int32_t block_threads, adj_block_threads;     /* threads per row-block CTA */
    int32_t parts_class0, adj_parts_class0;       /* separated schedules: partitions whose first
                                                     vertex is a first-kernel row (class 0; 0 for
                                                     paired schedules) */
    int32_t split_pct, adj_split_pct;             /* see sf_schedule_set_split */
    int32_t g2_placement, adj_g2_placement;       /* see sf_options.g2_placement */
    int32_t min_blocks, adj_min_blocks;           /* see sf_schedule_set_occupancy */
    int64_t ic0_pairs;                 /* IC0 schedules: intersection pairs listed by the
                                          inspector (-1: too many, not listed); else 0 */
    int32_t ic0_use_pairs, reserved3;  /* 1 when the factor reads the listed pairs */
    int64_t slice_cost, adj_slice_cost;   /* see sf_schedule_set_slices (0: off) */
    int32_t slice_units, adj_slice_units; /* queue units with split rows (0: no row split) */
    int32_t max_slices, adj_max_slices;   /* most slices of one row */
    int32_t fwd_rhs_tile, adj_rhs_tile;   /* right-hand-side tile of each direction (0: automatic) */
} sf_info;
sf_status sf_schedule_query(const sf_schedule *sch, sf_info *info);

/* Copies one schedule to HOST buffers for inspection and tests. which = 0 forward,
 * 1 adjoint. level[n_items] (wavefront of each vertex, vertex v = kernel*n + row),
 * order[n_items] (row | kernel << 31 in execution order), part_ptr[n_parts+1];
 * any pointer may be NULL. Synchronous. */
sf_status sf_schedule_export(const sf_schedule *sch, int32_t which, int32_t *level,
                             int32_t *order, int32_t *part_ptr);

/* Changes launch parameters of both directions without re-inspecting (the partition cut
 * stays as it was; see sf_schedule_recut): lanes_per_row (1..32, pow2), rhs_tile
 * (1..lanes_per_row, pow2) and blocks_per_sm (>= 1); 0 keeps the current value.
 * epoch_flags: 1 always publishes through epoch flags, 0 uses value flags when k = 1,
 * -1 keeps the current setting. */
sf_status sf_schedule_set_launch(sf_schedule *sch, int32_t lanes_per_row, int32_t rhs_tile,
                                 int32_t blocks_per_sm, int32_t epoch_flags);

/* Re-cuts the partitions (§3.1 coarsening) of the forward (which = 0), adjoint (1) or both
 * (-1) schedules for a new cost target (0 = automatic) and, when non-zero, a new lane count
 * per row and per team (8 or 32); levels and order are kept. Synchronises `stream` before and after; no launch
 * of this schedule may be pending on another stream. Used by autotuning. */
sf_status sf_schedule_recut(sf_schedule *sch, int32_t which, int64_t part_cost_target,
                            int32_t lanes_per_row, int32_t team_lanes, void *stream);

/* Re-places the second kernel's vertices of the forward (0), adjoint (1) or both (-1)
 * separated schedules (g2_placement as in sf_options) and rebuilds their order, partition
 * cut (same cost target) and row-block order; the earliest levels are kept from inspection.
 * Paired schedules are left as they are. Synchronises `stream` before and after. */
sf_status sf_schedule_replace(sf_schedule *sch, int32_t which, int32_t g2_placement, void *stream);

/* Row-block executor (k = 1 with value flags, exec_mode 2): blocks of B consecutive rows
 * (in decreasing row order for the adjoint), each run by one CTA that keeps the block's
 * values in shared memory, so dependences inside a block never leave the SM; the CTA runs
 * one level segment at a time between barriers. A pre-pass computes each row's
 * independent part and 1 / L_ii, so first-kernel rows finish as (c - sum) * (1 / L_ii)
 * (one rounding more than a division). Rebuilds the block
 * order of the forward (0), adjoint (1) or both (-1) schedules for block_rows rows
 * (0 keeps the current size, or takes the automatic size when leaving exec_mode 5), sets
 * exec_mode (-1 keeps; 0 automatic, 1 partitions, 2 row blocks, 3 warp-specialised row
 * blocks, 4 row blocks with packed records, built here, 5 the single-CTA executor: one block
 * per instance, which needs block_rows = 0) and the row-block lanes per row (1, 2, 4 or 32;
 * 0 keeps; exec_modes 3 and 4 run one consumer thread per row). For exec_mode 5 the last
 * argument is the number of CTAs sharing an SM instead (1, 2 or 4, of 1024, 512 or 256
 * threads and an equal share of the SM's shared memory; 0 automatic: 1 when every instance
 * has an SM of its own, else 2). The single-CTA executor scales the diagonal by its
 * reciprocal when L is staged in shared memory (one rounding more than a division), and
 * divides otherwise. Synchronises `stream` before and after. */
sf_status sf_schedule_reblock(sf_schedule *sch, int32_t which, int32_t block_rows, int32_t exec_mode,
                              int32_t lanes_per_row, void *stream);

/* Number of kernel launches one sf_execute (which = 0) or one sf_adjoint with both value
 * gradients (which = 1) makes with k right-hand sides in the schedule's current launch shape
 * (pre-passes, gathers and gradient passes included). Host only. */
sf_status sf_schedule_launches(const sf_schedule *sch, int32_t which, int32_t k, int32_t *count);

/* Timing hook: the next launches of the forward (0) or adjoint (1) schedule record ev_start
 * (a cudaEvent_t) on the launch stream right before the fused executor kernel and ev_stop
 * right after it (pre-passes, gathers and gradient passes fall outside), so a caller can
 * time the executor kernel alone with cudaEventElapsedTime. Both NULL stops the recording.
 * The events stay owned by the caller and must outlive the launches. No GPU work. */
sf_status sf_schedule_set_exec_events(sf_schedule *sch, int32_t which, void *ev_start, void *ev_stop);

/* Register budget of the partition executor's kernels for the forward (0), adjoint (1) or
 * both (-1) schedules: min_blocks 1 (or 0, the default) lets the kernels keep all the
 * registers they want, which suits schedules bound by their dependence chain; 3 selects
 * variants compiled for three (four for IC0) resident 256-thread blocks per SM, which suits
 * schedules bound by the number of rows in flight (many independent instances, wide
 * wavefronts). The variants exist for value-flag launches (k = 1) with 1, 2 or 4 lanes per
 * row and 32-lane teams, and for IC0 launches with 32 lanes per row. 2 selects variants for
 * two resident blocks (128 registers) of value-flag launches with 16 or 32 lanes per row (many
 * right-hand sides): twice the teams, each further ahead of the dependence chain. Other
 * launches use the default kernels. No GPU work. */
sf_status sf_schedule_set_occupancy(sf_schedule *sch, int32_t which, int32_t min_blocks);

/* IC0 schedules (SF_IC0_TRSV, SF_IC0; §2.1 up-looking zero-fill factor): entry (i, j) of
 * the factor subtracts sum_{k<j} L_ik L_jk over the columns k that rows i and j share. The
 * inspector lists those columns once per entry as pairs of entry positions (8 bytes per
 * pair, kept with the schedule) unless there are more than 4 nnz(L) + 2^20 of them. use = 1
 * (the default when listed) makes the executor read the pairs; with use = 0 it finds the
 * common columns by binary search on every call. SF_ERR_UNSUPPORTED for other pairs, or
 * for use = 1 when nothing was listed. No GPU work. */
sf_status sf_schedule_set_ic0_pairs(sf_schedule *sch, int32_t use);

/* Partition classes of the separated schedules (SpTRSV -> SpMV forward, SpMV -> SpTRSV
 * adjoint): with class0_pct in 1..99 that percent of the executor's teams run the partitions
 * whose first vertex is a first-kernel row (the solve chain), the other teams run the
 * partitions that open with a second-kernel row (sinks of the joint DAG), each class round
 * robin in partition order, so second-kernel rows never occupy a team the chain waits for.
 * 0 (the default) runs one class. Applies to the forward (0), adjoint (1) or both (-1)
 * schedules; paired schedules ignore it. No GPU work. */
sf_status sf_schedule_set_split(sf_schedule *sch, int32_t which, int32_t class0_pct);

/* Execution-time split of long rows (§3.1 vertex cost c(v) used to balance the load of the
 * executor, not only of partitions): in the forward (which = 0), adjoint (1) or both (-1)
 * schedules, every SpTRSV row, SpMV -> SpTRSV row or transposed solve row (adjoints) whose cost
 * exceeds cost_per_slice gets a partition of its own (the partitions are re-cut with the same
 * cost target; levels and order are unchanged) and runs as m = ceil(cost / cost_per_slice)
 * slices (at most 32) on m teams: each slice streams a contiguous chunk of the row's entries
 * as their inputs arrive, m - 1 helpers store partial sums (library scratch of m - 1 values per
 * right-hand side, published by value), the owner slice (queued after its helpers; its chunk,
 * the latest columns, is half as long) adds them in slice order and finishes the row. Applies
 * to launches that publish through values (k = 1, or 16 or more lanes per row) of the
 * partition executor; other launches run rows whole. 0 turns it off (default). Synchronises
 * `stream`; no launch of this schedule may be pending on another stream. */
sf_status sf_schedule_set_slices(sf_schedule *sch, int32_t which, int64_t cost_per_slice, void *stream);

/* Right-hand-side tile of the forward (0), adjoint (1) or both (-1) schedules: the columns of
 * the k right-hand sides that the lanes of a row handle side by side (a power of two up to
 * 32; rows then get at least that many lanes); 0 returns to the schedule's tile (the
 * rhs_tile option or sf_schedule_set_launch; automatic when that is 0, the power of two at or
 * above k, at most 32). Chosen per direction by the autotuner. No GPU work. */
sf_status sf_schedule_set_rhs_tile(sf_schedule *sch, int32_t which, int32_t rhs_tile);

/* Packing of the forward pass of an SF_SPMV_TRSV schedule (§3.2.3): 1 interleaved (default;
 * each paired row computes r_i = b_i - A_i x_in in registers, then its solve row), 0 separated
 * (the SpMV vertices first: every group of the partition executor computes r_i for its share
 * of the rows, in increasing row order, before it takes partitions, and publishes it by value
 * in a buffer of n x k values the library owns; the solve rows, split over teams or not, then
 * wait for their r_i and walk L's strict part only). Separated packing needs a value-flag
 * launch (k = 1, or 16 or more lanes per row) of the partition executor on its one- or
 * two-block kernels (sf_schedule_set_occupancy 1 or 2); other launches return
 * SF_ERR_UNSUPPORTED. The levels and order are the same for both. Other pairs:
 * SF_ERR_UNSUPPORTED. sf_schedule_info reports the choice in `packing`. No GPU work. */
sf_status sf_schedule_set_packing(sf_schedule *sch, int32_t packing);

/* Copies a row-block schedule to HOST buffers: order[n_items] (row | kernel << 31, sorted
 * by (block, level, kernel, row)), block_ptr[n_blocks+1], seg_ptr[block_segments+1] (first
 * position of every level segment: a maximal run of positions with the same block and
 * level, run by one CTA between two barriers) and block_seg[n_blocks+1] (first segment of
 * every block). Any pointer may be NULL. Synchronous. */
sf_status sf_schedule_export_blocks(const sf_schedule *sch, int32_t which, int32_t *order,
                                    int32_t *block_ptr, int32_t *seg_ptr, int32_t *block_seg);

/* Sets the time limit of one dependence wait (0 = 2 s). */
sf_status sf_schedule_set_timeout(sf_schedule *sch, uint64_t timeout_ns);

/* Testing hook: swaps two entries of the forward order (positions q1 and q2) on the
 * device, in the partition order and in the row-block order, producing a schedule that may
 * violate a dependence. An execution of such a
 * schedule ends through the bounded dependence wait with SF_ERR_TIMEOUT reported by
 * sf_schedule_check, never by a hang. */
sf_status sf_schedule_debug_swap(sf_schedule *sch, int64_t q1, int64_t q2);

void sf_schedule_destroy(sf_schedule *sch);

/* Allocation-free fused SpTRSV -> SpMV, y = M L^-1 b with one right-hand side (k = 1).
 *
 * The paper has no counterpart: this entry point serves callers that must not allocate device
 * memory at the point of the call - code that runs inside a custom allocator's own callbacks,
 * applications whose device memory is all handed out in advance by their own pool or budget,
 * and latency-critical loops that cannot wait for the device-wide synchronisation an
 * allocation can imply. It needs no inspector schedule (and so allocates nothing): rows run in
 * their natural order (all SpTRSV rows, then all SpMV rows), which is a valid order of the
 * joint DAG because L is lower triangular, and the intermediate x plus the launch state live
 * in a fixed device array compiled into the library.
 *
 *  L, M:   patterns as for sf_inspect with SF_TRSV_SPMV (n x n, n = L.n_rows); device
 *          pointers, caller-owned. They are checked on the GPU at every call.
 *  L_vals, M_vals, b (n x 1) inputs and y (n x 1) output: device pointers, caller-owned.
 *  n must not exceed SF_NOALLOC_MAX_ROWS (larger sizes return SF_ERR_INVALID_ARG).
 * Scratch: one array of SF_NOALLOC_SCRATCH_BYTES bytes per device, held by every GPU that
 * loads the library until the process exits. The first call on a device (and the first after
 * the device's context was reset) looks up that array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture. Every call clears the
 * part of the array it uses, but all calls share the one array: calls whose executions overlap
 * on the GPU (other streams, other host threads) race and give wrong results; serialise them.
 * The call is stream-ordered and then synchronises `stream` to report the outcome:
 * SF_ERR_BAD_PATTERN, SF_ERR_TIMEOUT or SF_ERR_NONFINITE (a zero diagonal of L) as for the
 * scheduled path. */
#define SF_NOALLOC_MAX_ROWS 1048576
#define SF_NOALLOC_SCRATCH_BYTES (256 + 8 * SF_NOALLOC_MAX_ROWS)
sf_status sf_trsv_spmv_noalloc(sf_dtype dt, const sf_csr *L, const sf_csr *M, const void *L_vals,
                               const void *M_vals, const void *b, void *y, void *stream);

/* Measurement helpers for the roofline of the executor (the paper has no counterpart; they
 * compute nothing of the method). Both are asynchronous on `stream`; the caller times them with
 * CUDA events.
 *  sf_bench_fma: the FMA rate of the GPU in the given element type: blocks x 256 threads, each
 *    running 8 independent chains of `iters` fused multiply-adds, i.e. blocks * 256 * 16 * iters
 *    flops. sink: device buffer of >= 256 elements (not written).
 *  sf_bench_hop: the latency of handing one value between two SMs through L2 (one relaxed
 *    store, one polling relaxed load), `hops` (even, >= 2) times in alternation by two resident
 *    blocks. word: one zeroed device uint32; out: two zeroed device uint64, out[0] receives the
 *    elapsed ns, out[1] = 1 when a poll gave up after 1 s (never a hang). */
sf_status sf_bench_fma(sf_dtype dt, int32_t blocks, int32_t iters, void *sink, void *stream);
sf_status sf_bench_hop(int32_t hops, void *word, void *out, void *stream);

const char *sf_status_string(sf_status s);

/* Copies the thread-local description of the last failure into buf (NUL-terminated). */
sf_status sf_last_error_detail(char *buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* SPARSEFUSION_H */
