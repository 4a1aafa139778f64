/*
 * lbspmv.h -- load-balanced CSR sparse matrix-vector multiply for NVIDIA GB300 (sm_103a).
 *
 * The method is the atom/tile/tile-set load-balancing model of "GPU Load Balancing"
 * (M. Osama, 2022): a work atom is a nonzero, a work tile is a row, the tile set is the
 * matrix (Ch.3 Sec. "Terminology"; Ch.4 Sec. "Input from Sparse Data Structures").  SpMV
 * runs under one of three schedule families:
 *   - thread-mapped: one row per thread (Ch.3 Sec. "Thread-Mapped"; Listing lst:spmv);
 *   - group-mapped: a group of threads (4..32 lanes, a warp, or a block) per set of rows,
 *     with a prefix sum of row lengths and a binary search atom -> row (Ch.3 Sec.
 *     "Group-Mapped", Alg. alg:group-mapped; Ch.4 Sec. "Group-level load balancing");
 *   - merge-path (work-oriented): rows + nonzeros split evenly, a 2-D diagonal search per
 *     split, partial rows carried out and fixed up afterwards (Ch.3 Sec. "Work-Oriented",
 *     Alg. alg:work-oriented; Ch.4 Sec. "Merge-path load balancing").
 *
 * Conventions for every call below.
 *   - All array arguments are DEVICE pointers owned by the caller unless a parameter says
 *     "host".  The library never frees caller memory.  Any alignment is accepted.
 *   - Indices are int32: row_offsets[m+1] (row_offsets[0] == 0, non-decreasing,
 *     row_offsets[m] == nnz), col_idx[nnz] in [0, n).  Values are FP32, BF16 or FP16
 *     (lb_dtype); x, y, g and dx are FP32; the values gradient dvalues is FP32 or, where a
 *     call takes its type (dvdt), BF16/FP16 rounded to nearest even from the FP32 product
 *     (the storage an autograd engine expects for 16-bit values); accumulation is FP32.
 *   - y is OVERWRITTEN: y = A x (no beta).  Empty rows give 0.  m == 0 is a no-op;
 *     nnz == 0 gives y = 0.
 *   - Work is stream-ordered on `stream` (0 = the legacy default stream).  No call
 *     synchronizes the device except the ones documented as copying results to the host.
 *     lb_spmv_planned, lb_spmv_t, lb_spmv_dvalues and lb_spmv_batched allocate nothing and
 *     never synchronize.
 *   - Argument errors are reported before any GPU work as LB_ERR_INVALID_ARG; CUDA errors
 *     as LB_ERR_CUDA.  Pointers must be aligned to their element type.  Kernels never trap
 *     and never wait on a flag or on other warps or CTAs, so none can hang; a kernel that
 *     meets a tile only malformed offsets produce skips it and records LB_ERR_BAD_MATRIX in
 *     a device error word read by lb_device_error().
 *   - Matrix contents are not checked by the SpMV calls; lb_validate_csr checks them.
 *   - No C++ exception crosses this interface.
 */
#ifndef LBSPMV_H
#define LBSPMV_H

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LB_OK = 0,
    LB_ERR_INVALID_ARG = -1, /* bad size, null pointer, unknown enum, plan of the wrong kind */
    LB_ERR_BAD_MATRIX = -2,  /* malformed matrix contents (found by a check or a kernel) */
    LB_ERR_UNSUPPORTED = -3, /* valid request this library does not implement */
    LB_ERR_NO_MEMORY = -4,   /* a plan or workspace allocation failed */
    LB_ERR_CUDA = -5,        /* a CUDA runtime call failed */
    LB_ERR_TIMEOUT = -6,     /* reserved: no kernel of this library waits on a signal */
    LB_ERR_TOO_LARGE = -7,   /* the request exceeds a fixed-size static workspace */
    LB_ERR_OUT_OF_RANGE = -8 /* range-checked build only: an index read from the inputs
                                (a column, a row, a position) lies outside its array */
} lb_status;

typedef enum {
    LB_SCHED_AUTO = 0,          /* merge-path unless (min(m, n) < 500 and nnz < 10000) */
    LB_SCHED_THREAD_MAPPED = 1, /* Ch.3 Sec. "Thread-Mapped"; Listing lst:thread-mapped */
    LB_SCHED_WARP_MAPPED = 2,   /* group-mapped with a 32-lane group (Ch.4 "Warp- and block-level") */
    LB_SCHED_BLOCK_MAPPED = 3,  /* group-mapped with the whole block as the group */
    LB_SCHED_GROUP_MAPPED = 4,  /* group-mapped, group_size in {4, 8, 16, 32} */
    LB_SCHED_MERGE_PATH = 5,    /* work-oriented merge-path (Alg. alg:work-oriented) */
    LB_SCHED_NONZERO_SPLIT = 6  /* work-oriented, nonzeros only (Ch.3 "Work-Oriented"); plans only */
} lb_schedule;

typedef enum { LB_F32 = 0, LB_BF16 = 1, LB_F16 = 2 } lb_dtype;

/* Launch shape of a schedule; 0 selects the default.
 *   merge-path:   (threads, items_per_thread) in {(128, 16), (256, 8), (256, 16), (384, 8),
 *                 (512, 8)}, default (256, 8): CTAs of `threads` threads whose warps each
 *                 work one tile at a time of 32 * items_per_thread - 8 work items (rows +
 *                 nonzeros); the plan's block-level passes (SpMM beyond the warp kernels,
 *                 the transpose) use tiles of threads * items_per_thread - 8 items;
 *   block-mapped: threads in {128, 256} (the group is the block);
 *   group-mapped: group_size in {4, 8, 16, 32}. */
typedef struct {
    int threads;
    int items_per_thread;
    int group_size;
} lb_tuning;

typedef struct lb_plan lb_plan;
typedef struct lb_batched_plan lb_batched_plan;

/* Human-readable name of a status code (static storage). */
const char *lb_status_string(lb_status s);

/* Library version, major * 10000 + minor * 100 + patch. */
int lb_version(void);

/*
 * y = A x for a CSR matrix, in one call: the dissertation's kernel signature
 * spmv(rows, cols, nnz, offsets, indices, values, x, y) (Listing lst:spmv) plus a value
 * type and a stream.  The schedule is chosen by the rule of Ch.4 Sec. "Improved Performance
 * Response" (merge-path unless min(m, n) < 500 and nnz < 10000; then group- or thread-mapped
 * by the mean row length).  Merge-path recomputes its partition every call and takes its
 * workspace with cudaMallocAsync / cudaFreeAsync on `stream`.
 */
lb_status lb_spmv(int m, int n, int nnz, const int *row_offsets, const int *col_idx,
                  const void *values, lb_dtype vdt, const float *x, float *y, cudaStream_t stream);

/*
 * lb_spmv_static: y = A x like lb_spmv, but with NO device allocation.  The dissertation has
 * no counterpart; this is an interface for callers that must not allocate: a process whose
 * device memory is already reserved by another allocator (a framework's caching allocator,
 * or an arena sized to the card), where lb_spmv's cudaMallocAsync workspace can fail with
 * out-of-memory; latency-bound loops where an allocation may block on the pool or driver; or
 * code that has promised its host framework to allocate only through that framework.
 *
 * Schedule: always merge-path with the (256, 8) launch shape (tiles of
 * LB_SPMV_STATIC_TILE_ITEMS work items), whatever the matrix size.
 * Workspace: a file-scope __device__ array inside the library, one per device, holding the
 * partition and carry arrays of at most LB_SPMV_STATIC_MAX_TILES tiles (8 MiB).  So
 * m + nnz must be at most LB_SPMV_STATIC_MAX_TILES * LB_SPMV_STATIC_TILE_ITEMS
 * (130,023,424); larger requests return LB_ERR_TOO_LARGE before any GPU work.
 * Set-up: the FIRST call on each device (with that device current) looks up the array's
 * device address (cudaGetSymbolAddress), caches it, and does the merge-path kernel's
 * host-side set-up (shared-memory carveout, occupancy) for all three value types; make that
 * first call before any stream capture.  Later calls only enqueue one small memset (the
 * carry rows are filled with -1 every call) and the partition, merge-path and fixup kernels
 * on `stream`.
 * Concurrency: every call on one device shares the one workspace, so calls that overlap in
 * time (on different streams, or from several host threads without stream ordering between
 * them) RACE and give wrong results.  Calls ordered on one stream are safe.
 * Arguments, results and other errors are as for lb_spmv.
 */
#define LB_SPMV_STATIC_MAX_TILES 524288
#define LB_SPMV_STATIC_TILE_ITEMS 248
lb_status lb_spmv_static(int m, int n, int nnz, const int *row_offsets, const int *col_idx,
                         const void *values, lb_dtype vdt, const float *x, float *y,
                         cudaStream_t stream);

/*
 * Merge-path partition (Alg. alg:work-oriented, "2DSearch"; Ch.4 Sec. "Merge-path load
 * balancing").  Row ends R_r (key row_offsets[r+1]) are merged with nonzero indices N_k
 * (key k), R_r before N_k when row_offsets[r+1] <= k.  For tile boundaries
 * d_c = min(c * tile_items, m + nnz), c = 0..G with G = ceil((m + nnz) / tile_items), writes
 * tile_row[c] = #{r : r + row_offsets[r+1] < d_c} (row ends before d_c) and
 * tile_nz[c] = d_c - tile_row[c] (nonzeros before d_c).  tile_row and tile_nz are device
 * arrays of G + 1 ints.  Bit-exact; no allocation.  A tile_items so small that G reaches
 * 2^31 - 1 returns LB_ERR_INVALID_ARG.
 */
lb_status lb_partition(int m, int nnz, const int *row_offsets, int tile_items, int *tile_row,
                       int *tile_nz, cudaStream_t stream);

/* Number of tiles G for lb_partition (host arithmetic only). */
int lb_num_tiles(int m, int nnz, int tile_items);

/*
 * Build a plan for one sparsity structure.  The plan copies row_offsets (device, m + 1
 * ints), resolves LB_SCHED_AUTO, and for merge-path computes the partition once and owns
 * the carry buffers, so lb_spmv_planned allocates nothing.  `t` may be NULL.  The work is
 * enqueued on `stream`; the plan is usable on any stream ordered after it.
 */
lb_status lb_plan_create(int m, int n, int nnz, const int *row_offsets, lb_schedule s,
                         const lb_tuning *t, cudaStream_t stream, lb_plan **out);

/*
 * Resolved schedule and launch shape of a plan; any output pointer may be NULL.  num_tiles and
 * tile_items describe the LB_TILES_ROWS tile set (below).
 */
lb_status lb_plan_info(const lb_plan *p, lb_schedule *s, lb_tuning *t, int *num_tiles,
                       int *tile_items);

/*
 * A plan's tile sets, each a merge-path partition (Alg. alg:work-oriented) of its own tile
 * size:
 *   LB_TILES_ROWS        tiles of threads * items_per_thread - 8 work items, walked by the
 *                        block-level passes over the forward partition (dvalues gathering x,
 *                        the transpose and SpMM); every plan;
 *   LB_TILES_TRANSPOSED  warp tiles (248 work items) of the transposed product's merge path
 *                        over the CSC view; after lb_plan_build_transpose;
 *   LB_TILES_MERGE       warp tiles (32 * items_per_thread - 8 work items; 248 for schedules
 *                        other than merge-path) of the merge-path forward and of the CSR-order
 *                        backward pass; every plan with m > 0.
 * lb_plan_tiles gives a set's tile count and size; LB_ERR_INVALID_ARG for a set the plan
 * does not hold.
 */
#define LB_TILES_ROWS 0
#define LB_TILES_TRANSPOSED 1
#define LB_TILES_MERGE 2
lb_status lb_plan_tiles(const lb_plan *p, int which, int *num_tiles, int *tile_items);

/*
 * Copy one of a plan's tile sets (`which`, above) to HOST arrays of num_tiles + 1 ints
 * (synchronizes the device).  With tile_row == NULL only *num_tiles is written.
 */
lb_status lb_plan_partition(const lb_plan *p, int which, int *tile_row, int *tile_nz,
                            int *num_tiles);

/* y = A x with a plan (no allocation, no synchronization; CUDA-graph capturable). */
lb_status lb_spmv_planned(const lb_plan *p, const int *col_idx, const void *values, lb_dtype vdt,
                          const float *x, float *y, cudaStream_t stream);

/*
 * Build the CSC view of the plan's matrix, once (after checking offsets and column range as
 * lb_validate_csr does; LB_ERR_BAD_MATRIX if they fail): col_offsets[n+1], row_idx[nnz] and
 * perm[nnz] (perm[p] = the CSR index of CSC entry p) by a stable transpose (entries of a
 * column keep increasing CSR index), plus the merge-path partition of the transposed
 * matrix.  The framework's atom/tile view covers CSC as it covers CSR (Ch.4 Sec.
 * "Implementing Sparse Data Structures"; "Merge-path load balancing": any format with an
 * atoms-per-tile count).  Deterministic; allocates plan memory and temporary workspace.
 */
lb_status lb_plan_build_transpose(lb_plan *p, const int *col_idx, cudaStream_t stream);

/* Copy the CSC view to HOST arrays (n + 1, nnz, nnz ints); synchronizes the device. */
lb_status lb_plan_transpose(const lb_plan *p, int *col_offsets, int *row_idx, int *perm);

/*
 * dx = A^T g (backward of y = A x with respect to x) over the CSC view, in two passes.  First,
 * one streaming pass over the nonzeros in CSR order forms the scaled values v[k] * g[row(k)]
 * (row(k) from the forward partition) and writes them into L2-sized buckets of CSC order
 * (plan memory, 4 bytes per nonzero).  Then a merge-path pass over the CSC view (tiles =
 * columns, atoms = CSC entries) sums, per column, the scaled values gathered from the bucket
 * being worked on, and the fixup adds the carries.  The summation order (CSC order within a
 * column) and the product rounding are fixed, so dx is deterministic.  Requires
 * lb_plan_build_transpose.  g: m floats, dx: n floats (overwritten).  Not safe to run
 * concurrently with another lb_spmv_t / lb_spmv_backward on the same plan (shared scratch).
 *
 * CSC input.  A matrix A (m x n) given in CSC form (col_offsets[n+1], row_idx[nnz], values in
 * CSC order) is A^T in CSR form.  A plan created from col_offsets with n_cols = m, with
 * lb_plan_build_transpose(plan, row_idx), computes y = A x as lb_spmv_t(plan, values, x, y):
 * merge-path over A's rows in the CSC view (Ch.4: merge-path over any format with an
 * atoms-per-tile count; CSC as a format in Sec. "Implementing Sparse Data Structures").
 */
lb_status lb_spmv_t(const lb_plan *p, const void *values, lb_dtype vdt, const float *g, float *dx,
                    cudaStream_t stream);

/*
 * dvalues[k] = g[row(k)] * x[col_idx[k]] (backward of y = A x with respect to the values),
 * one coalesced pass over the nonzeros; row(k) comes from the plan's merge-path partition
 * (each tile stages its row ends and searches them).  Merge-path plans only.  dvalues: nnz
 * elements of dvdt (LB_F32, LB_BF16 or LB_F16: the FP32 product rounded to nearest even).
 */
lb_status lb_spmv_dvalues(const lb_plan *p, const int *col_idx, const float *g, const float *x,
                          void *dvalues, lb_dtype dvdt, cudaStream_t stream);

/*
 * y = A x with a merge-path plan (as lb_spmv_planned), also saving the gathered operand of
 * every nonzero: x_gathered[k] = x[col_idx[k]] (device, nnz floats, overwritten).  The values
 * gradient dvalues[k] = g[row(k)] * x[col_idx[k]] needs exactly these, so
 * lb_spmv_dvalues_gathered can form it by streaming them back instead of gathering x again.
 * Costs 4 bytes per nonzero of coalesced stores.  LB_ERR_UNSUPPORTED for plans whose schedule
 * is not merge-path.  No allocation, no synchronization.
 */
lb_status lb_spmv_planned_save(const lb_plan *p, const int *col_idx, const void *values, lb_dtype vdt,
                               const float *x, float *y, float *x_gathered, cudaStream_t stream);

/*
 * dvalues[k] = g[row(k)] * x_gathered[k] with x_gathered from lb_spmv_planned_save (the same
 * values as lb_spmv_dvalues, bit for bit); row(k) from the plan's forward partition.
 * dvalues: nnz elements of dvdt, as lb_spmv_dvalues.
 */
lb_status lb_spmv_dvalues_gathered(const lb_plan *p, const float *g, const float *x_gathered, void *dvalues,
                                   lb_dtype dvdt, cudaStream_t stream);

/*
 * Both gradients of y = A x in one go: dvalues[k] = g[row(k)] * x_gathered[k] (x_gathered from
 * lb_spmv_planned_save) is formed in the same CSR-order pass that prepares the scaled values
 * for dx = A^T g (see lb_spmv_t), so the backward is two passes over the nonzeros instead of
 * three.  Results equal lb_spmv_t's dx and lb_spmv_dvalues_gathered's dvalues bit for bit.
 * Requires lb_plan_build_transpose; dx (n floats) and dvalues (nnz elements of dvdt: LB_F32,
 * or vdt itself for 16-bit values) are overwritten; any other dvdt is LB_ERR_INVALID_ARG.
 */
lb_status lb_spmv_backward(const lb_plan *p, const void *values, lb_dtype vdt, const float *g,
                           const float *x_gathered, float *dx, void *dvalues, lb_dtype dvdt,
                           cudaStream_t stream);

/*
 * The backward without a CSC view, and not bit-reproducible: one streaming pass over the
 * nonzeros in CSR order (the forward partition, as in lb_spmv_backward's first pass) adds
 * every v[k] * g[row(k)] into dx[col_idx[k]] with a float reduction in L2, and, when dvalues
 * is given, writes dvalues[k] = g[row(k)] * x_gathered[k] (bit-exact, as lb_spmv_backward).
 * The additions into a column arrive in no fixed order, so dx can differ in its last bits from
 * run to run; it stays within the FP32 bound of the transposed product (per column
 * 1e-5 * sum_i |a_ij| |g_i|).  The dissertation computes no backward; this is the
 * atomic-scatter alternative to the transposed SpMV of lb_spmv_backward, for callers that
 * trade reproducibility for one pass and no CSC plan memory.
 * col_idx: nnz ints; values: nnz of vdt; g: m floats; x_gathered: nnz floats from
 * lb_spmv_planned_save (may be NULL when dvalues is NULL); dx: n floats, overwritten (zeroed,
 * then accumulated); dvalues: nnz elements of dvdt (LB_F32, or vdt itself for 16-bit values)
 * or NULL.  Needs only the plan's forward partition.
 */
lb_status lb_spmv_backward_scatter(const lb_plan *p, const int *col_idx, const void *values, lb_dtype vdt,
                                   const float *g, const float *x_gathered, float *dx, void *dvalues,
                                   lb_dtype dvdt, cudaStream_t stream);

/*
 * SpMM: C = A B with B dense (n x kc, row-major, FP32) and C (m x kc, row-major, FP32,
 * overwritten), over merge-path tiles of the plan's matrix: the dissertation's SpMV with a loop
 * over the columns of B (Ch.4 Sec. "Application Space", the SpMM listing).  kc = 8 or 16 with B
 * and C 32-byte aligned: 248-item warp tiles, each nonzero gathering 8 columns of B's row in
 * one 32-byte load per chunk; kc <= 4: the same warp tiles with 16-byte (or scalar) gathers;
 * other kc: the plan's block tiles, 16-byte vectors of B per thread (scalar loads when
 * kc % 4 != 0 or B, C are not 16-byte aligned).  Rows split across tiles are completed by a
 * fixup of kc-wide carries in tile order, so C is deterministic.  On the block tiles, plans
 * whose tiles exceed 2048 work items give LB_ERR_UNSUPPORTED.  The first call (and any call
 * with more columns or tiles than before) allocates the plan's carry buffer (G * (kc + 1) * 4
 * bytes), and the first warp-tile call on a plan whose own tiles are not 248 items allocates
 * and builds a partition of its own; later calls allocate nothing.
 */
lb_status lb_spmm_planned(lb_plan *p, const int *col_idx, const void *values, lb_dtype vdt, int kc,
                          const float *B, float *C, cudaStream_t stream);

void lb_plan_destroy(lb_plan *p);

/*
 * Plan for `count` independent CSR matrices run as one block-diagonal matrix (the
 * "sets of sets" extension of Ch.6 Sec. "Multi-GPU Load Balancing": merge-path keeps its
 * structure one level up).  h_m, h_n, h_nnz: HOST arrays of `count` sizes.
 * row_offsets_concat (device) concatenates each matrix's own offsets (m_i + 1 entries,
 * each starting at 0).  The plan materializes the block-diagonal row offsets and one
 * global merge-path partition over sum(m_i + nnz_i).  Schedules:
 *   LB_SCHED_MERGE_PATH (and LB_SCHED_AUTO): the global merge path, one persistent launch
 *     plus the fixup; t picks its launch shape.
 *   LB_SCHED_THREAD_MAPPED: a row per lane over the block-diagonal matrix (Ch.3 Sec.
 *     "Thread-Mapped"), rows longer than 32 nonzeros summed by the lane's whole warp (the
 *     group-mapped remedy, Ch.3 Sec. "Group-Mapped"); one launch, no carries.  Suited to
 *     batches of mostly very short rows; t must be NULL or zero.
 * Other schedules return LB_ERR_UNSUPPORTED.  The autotuner (lb_tune_batched) measures both
 * for a batch's shape class.
 */
lb_status lb_batched_plan_create(int count, const int *h_m, const int *h_n, const int *h_nnz,
                                 const int *row_offsets_concat, lb_schedule s, const lb_tuning *t,
                                 cudaStream_t stream, lb_batched_plan **out);

/* Launch shape, number of tiles and work items per tile of a batched plan (any output may
 * be NULL). */
lb_status lb_batched_plan_info(const lb_batched_plan *p, lb_tuning *t, int *num_tiles, int *tile_items);

/* The schedule a batched plan runs (LB_SCHED_MERGE_PATH or LB_SCHED_THREAD_MAPPED). */
lb_status lb_batched_plan_schedule(const lb_batched_plan *p, lb_schedule *s);

/* Copy the global partition to HOST arrays of num_tiles + 1 ints (synchronizes). */
lb_status lb_batched_plan_partition(const lb_batched_plan *p, int *tile_row, int *tile_nz,
                                    int *num_tiles);

/*
 * y_i = A_i x_i for every matrix of the plan in ONE persistent launch plus the fixup (one
 * launch and no fixup under the thread-mapped schedule).
 * col_idx_concat holds local column indices; values_concat, x_concat (sum n_i floats) and
 * y_concat (sum m_i floats) are concatenated in matrix order.  No allocation.
 */
lb_status lb_spmv_batched(const lb_batched_plan *p, const int *col_idx_concat,
                          const void *values_concat, lb_dtype vdt, const float *x_concat,
                          float *y_concat, cudaStream_t stream);

void lb_batched_plan_destroy(lb_batched_plan *p);

/*
 * Autotuner timing core.  The dissertation chooses a schedule by a fixed size rule (Ch.4 Sec.
 * "Improved Performance Response"); lb_tune measures instead.  Every candidate schedule and
 * launch shape this library implements (merge-path at each shape, thread-mapped, warp-mapped,
 * group-mapped with 4, 8 and 16 lanes, block-mapped with 128 and 256 threads) builds a plan
 * and runs y = A x `reps` times on `stream`, timed by CUDA events after one untimed call.
 * Results (schedule, resolved tuning, mean milliseconds) are written sorted fastest first,
 * at most `capacity` of them; *count receives how many.  y (m floats, device) is scratch
 * and is left holding A x.  Creates and destroys plans (allocates) and synchronizes the
 * stream.  lb_tune_candidates() is the number of candidates.
 */
typedef struct {
    lb_schedule schedule;
    lb_tuning tuning;
    float ms;
} lb_tune_result;

int lb_tune_candidates(void);

lb_status lb_tune(int m, int n, int nnz, const int *row_offsets, const int *col_idx, const void *values,
                  lb_dtype vdt, const float *x, float *y, int reps, lb_tune_result *results, int capacity,
                  int *count, cudaStream_t stream);

/*
 * The same for a batch (arguments as for lb_batched_plan_create and lb_spmv_batched): the
 * thread-mapped batch schedule and the block-diagonal merge path at every launch shape,
 * timed.
 */
lb_status lb_tune_batched(int count, const int *h_m, const int *h_n, const int *h_nnz,
                          const int *row_offsets_concat, const int *col_idx_concat, const void *values_concat,
                          lb_dtype vdt, const float *x_concat, float *y_concat, int reps,
                          lb_tune_result *results, int capacity, int *count_out, cudaStream_t stream);

/*
 * Single-source shortest paths over a directed graph in CSR form (vertex u's out-edges are
 * u -> col_idx[k], k in [row_offsets[u], row_offsets[u+1]), n vertices), expressed on the
 * load-balancing schedules as in Ch.4 Sec. "Application Space" (the SSSP listing): the
 * frontier's edges are the atoms, split evenly over the threads; relaxing an edge lowers the
 * neighbour's distance with an atomic minimum and puts the neighbour on the next frontier when
 * it dropped; the host iterates until the frontier is empty.  With weights the frontier is
 * split by distance (near-far, Davidson et al., IPDPS 2014): neighbours whose new distance
 * reaches the split point are set aside and join a later frontier when the split point
 * advances (by delta = mean weight * 8 / mean degree).  weights: nnz non-negative FP32 values,
 * or NULL for unit weights (dist = BFS level, one level per iteration).  dist (n floats,
 * device) receives the distances (+inf when unreachable); *iterations (host) the number of
 * frontier iterations.  FP32 sums: each distance is the minimum over paths of the FP32 sum
 * along the path, whatever the order of relaxation.  Allocates its workspace (about 24 bytes
 * per vertex) and synchronizes `stream` once per iteration and once per advance of the split
 * point.  Negative weights are not supported.
 */
lb_status lb_sssp(int n, int nnz, const int *row_offsets, const int *col_idx, const float *weights,
                  int source, float *dist, int *iterations, cudaStream_t stream);

/*
 * Measured ceilings of the current GPU for the roofline of these kernels (no counterpart in
 * the dissertation): the rate of random 4-byte gathers from an L2-resident 16 MB vector
 * (every gather is its own 32-byte sector request from an SM to L2, the limit of SpMV with
 * scattered columns), and streaming read and copy bandwidth over 1 GiB buffers.  Each is the
 * best of three timed runs after a warm-up.  Allocates about 2 GiB temporarily and
 * synchronizes `stream`.
 */
typedef struct {
    double gathers_per_s; /* random 4-byte gathers (sector requests) per second */
    double read_GBps;     /* streaming read, 1e9 bytes per second */
    double copy_GBps;     /* streaming copy, bytes read + written, 1e9 bytes per second */
} lb_calibration;

lb_status lb_calibrate(lb_calibration *out, cudaStream_t stream);

/*
 * COO input (the framework's COO view of a sparse matrix, Ch.4 Sec. "Implementing Sparse Data
 * Structures"): for a COO matrix sorted by row (row_idx[nnz], device), write its CSR row
 * offsets row_offsets[m + 1] (device): row_offsets[r] = #{k : row_idx[k] < r}.  Then
 * (row_offsets, col_idx, values) is the same matrix in CSR form and every call above applies.
 * A check writes a bit mask to the device int *d_status: 1 a row index outside [0, m), 2 the
 * rows decrease somewhere (0 = valid; the offsets mean nothing otherwise).  No allocation.
 */
lb_status lb_coo_row_offsets(int m, int nnz, const int *row_idx, int *row_offsets, int *d_status,
                             cudaStream_t stream);

/*
 * Check a CSR matrix on the device and write a bit mask to the device int *d_status
 * (0 = valid): 1 row_offsets[0] != 0; 2 row_offsets decreasing somewhere; 4
 * row_offsets[m] != nnz; 8 a column index outside [0, n); 16 (only with check_sorted)
 * columns of a row not strictly increasing.  Never traps.
 */
lb_status lb_validate_csr(int m, int n, int nnz, const int *row_offsets, const int *col_idx,
                          int check_sorted, int *d_status, cudaStream_t stream);

/*
 * Read the current device's error word into *status; clear it when `clear` is nonzero.
 * Synchronizes the device.  LB_OK, or the last error a kernel recorded: LB_ERR_BAD_MATRIX (a
 * merge-path tile held more work than a tile can, or reached outside the arrays, which only
 * malformed row offsets produce; that tile was skipped).  LB_ERR_TIMEOUT is reserved: no
 * kernel of this library waits, so none records it.
 */
lb_status lb_device_error(int *status, int clear);

/*
 * Profiling aid: while set (non-NULL), every merge-path SpMV call (lb_spmv, lb_spmv_planned,
 * lb_spmv_planned_save, lb_spmv_t, lb_spmv_backward, lb_spmv_batched) records `before` right
 * before and `after` right after its merge-path kernel on the call's stream.  Process-wide, not thread-safe; pass
 * NULLs to stop.
 */
lb_status lb_set_profile_events(cudaEvent_t before, cudaEvent_t after);

/*
 * Test support for the out-of-memory paths (no counterpart in the dissertation; the paper
 * has no allocation).  Every device allocation the library makes (plan arrays, CSC views,
 * the workspace of lb_spmv, lb_validate_csr's status word, SSSP's frontier, calibration
 * buffers) goes through one counter.
 *   lb_debug_fail_allocations_after(count): the next `count` allocations proceed and every
 *     later one fails as if the device were full, so the call reports LB_ERR_NO_MEMORY and
 *     releases what it had allocated; count < 0 removes the limit (the default).
 *     Process-wide.
 *   lb_debug_live_allocations(): the library's device allocations currently held (plans not
 *     yet destroyed, workspaces whose stream-ordered free has not been issued).
 */
void lb_debug_fail_allocations_after(int count);
long long lb_debug_live_allocations(void);

#ifdef __cplusplus
}
#endif

#endif /* LBSPMV_H */
