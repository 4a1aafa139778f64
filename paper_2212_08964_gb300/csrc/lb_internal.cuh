// lb_internal.cuh -- shared device helpers and launcher declarations for liblbspmv (sm_103a).
//
// No kernel of the library waits on a flag, a barrier of other warps or another CTA: every
// warp-tiled kernel runs its warps independently, and the block-level passes use only
// __syncthreads.  So no kernel can hang on a signal that never comes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbspmv.h"

#include <nvtx3/nvToolsExt.h>

namespace lb {

// ------------------------------------------------------------------------------------------
// Range checks.  In the range-checked build (LB_CHECKED, liblbspmv_checked.so) every index a
// kernel reads from its inputs (a column, a row, a position) is tested against the array it
// addresses before the access; a violation skips the access and records LB_ERR_OUT_OF_RANGE
// in the device error word.  The build stands in for a memory checker.  In the normal build
// the tests compile away and the inputs are trusted (lb_validate_csr checks them).
#ifdef LB_CHECKED
}  // namespace lb
extern __device__ int g_lb_device_error;
namespace lb {
__device__ __forceinline__ bool in_range(long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicExch(&g_lb_device_error, static_cast<int>(LB_ERR_OUT_OF_RANGE));
    return false;
}
#define LB_IN_RANGE(i, n) ::lb::in_range((i), (n))
#else
#define LB_IN_RANGE(i, n) true
#endif

// ------------------------------------------------------------------------------------------
// Value types: stored as FP32, BF16 or FP16, always widened to FP32 in registers.

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

// Neumaier's compensated addition: s + c carries the running sum with an error bound that
// does not grow with the number of terms.
__device__ __forceinline__ void kbn_add(float &s, float &c, float v) {
    float t = s + v;
    if (fabsf(s) >= fabsf(v))
        c += (s - t) + v;
    else
        c += (v - t) + s;
    s = t;
}

// ------------------------------------------------------------------------------------------
// PTX wrappers.

// L2 eviction-priority policy for cache hints: streamed arrays are marked evict-first so that
// the gathered vector stays resident in L2.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// ------------------------------------------------------------------------------------------
// Kernel argument blocks.

// Merge-path SpMV over one tile set.  "Rows" are the tiles of the set (CSR rows, or CSC
// columns for the transposed product) and "atoms" its nonzeros.
struct MergeArgs {
    int num_tiles;        // G
    int num_rows;         // rows of the set (y has this many entries)
    int num_atoms;        // atoms of the set (entries of idx, and of val or perm)
    const int *tile_row;  // [G+1] row ends consumed before each tile boundary
    const int *tile_nz;   // [G+1] atoms consumed before each tile boundary
    const int *row_end;   // row_end[r] = offset one past the last atom of row r (offsets + 1)
    const int *idx;       // gather index per atom (column index; CSC row index when transposed)
    const void *val;      // values, per atom (unused by the gather-sum product)
    const float *x;       // gathered dense vector
    long long x_len;      // its length (the range-checked build tests every gather against it)
    float *y;             // output, one entry per row
    int *carry_row;       // [G] row left open at the end of each tile
    float *carry_val;     // [G] that row's partial sum inside the tile
    const int *mat_nz_base;   // batched: [K+1] first nonzero of each matrix
    const int *mat_col_base;  // batched: [K] offset of each matrix's x inside x_concat
    const int *tile_mat;      // batched: [G+1] matrix holding each tile's first nonzero
    float *xg;                // plain only, may be null: xg[k] = x[idx[k]] is saved for every atom
    int *err;                 // device error word
    int vec_vals;             // val has the same 32-byte phase as idx (FP32) or 16-byte phase (16-bit)
    int vec_xg;               // xg has the same 32-byte phase as idx
};

// Work items per merge-path tile of the warp-tiled kernel: 32 lanes x `ipt` slots, less 8
// kept for the lead of a tile's first nonzero past a 32-byte boundary.
__host__ __device__ constexpr int merge_tile_items(int ipt) { return 32 * ipt - 8; }

// The alignment flags of MergeArgs, from the arrays' addresses.
void set_merge_alignment(MergeArgs &a, size_t value_bytes);

// kPlain: y[r] = sum of val[k] * x[idx[k]] over row r.  kBatched: the same over a batch, with
// per-matrix column bases.  kGatherSum: y[r] = sum of x[idx[k]] (no values; the transposed
// product gathers its precomputed scaled values this way).
enum MergeMode { kPlain = 0, kBatched = 1, kGatherSum = 2 };

// Launch the persistent merge-path kernel (one wave of resident CTAs over the warp tiles of
// `a`, which come from a partition with merge_tile_items(ipt) items per tile) followed by the
// fixup kernel.  `ev_before` / `ev_after` (may be null) are recorded around the main kernel.
cudaError_t launch_merge_spmv(lb_dtype vdt, int mode, int threads, int ipt, const MergeArgs &a,
                              cudaStream_t stream, cudaEvent_t ev_before, cudaEvent_t ev_after);
cudaError_t launch_merge_f32(int mode, int threads, int ipt, const MergeArgs &a, cudaStream_t s,
                             cudaEvent_t eb, cudaEvent_t ea);
cudaError_t launch_merge_bf16(int mode, int threads, int ipt, const MergeArgs &a, cudaStream_t s,
                              cudaEvent_t eb, cudaEvent_t ea);
cudaError_t launch_merge_f16(int mode, int threads, int ipt, const MergeArgs &a, cudaStream_t s,
                             cudaEvent_t eb, cudaEvent_t ea);

// The host-side set-up of the plain merge-path product of one value type and shape (done by
// the first launch otherwise).
cudaError_t prepare_merge_f32(int threads, int ipt);
cudaError_t prepare_merge_bf16(int threads, int ipt);
cudaError_t prepare_merge_f16(int threads, int ipt);

// Fixup: y[r] += sum of the carries of row r, for every carry row r < num_rows.
cudaError_t launch_fixup(int num_tiles, int num_rows, const int *carry_row, const float *carry_val,
                         float *y, cudaStream_t stream);

// Merge-path partition of `offsets` (m + 1 entries) into tiles of tile_items work items.
cudaError_t launch_partition(int m, long long nnz, const int *offsets, int tile_items, int *tile_row,
                             int *tile_nz, cudaStream_t stream);

// Thread-, group- and block-mapped schedules.
cudaError_t launch_mapped(lb_schedule s, const lb_tuning &t, lb_dtype vdt, int m, int n, int nnz, const int *ro,
                          const int *ci, const void *v, const float *x, float *y, cudaStream_t stream);

// dvalues over the forward block tiles, gathering x: dv[k] = g[row(k)] * x[ci[k]], stored as
// dvdt (FP32, or BF16/FP16 rounded to nearest even).
cudaError_t launch_dvalues(int num_tiles, int tile_items, const int *tile_row, const int *tile_nz,
                           const int *row_end, const int *ci, const float *g, const float *x, int n, void *dv,
                           lb_dtype dvdt, cudaStream_t stream);

// Stable CSR -> CSC transpose (deterministic LSD radix sort by column).
struct TransposeOut {
    int *col_offsets;  // [n+1]
    int *row_idx;      // [nnz]
    int *perm;         // [nnz]
};
cudaError_t build_transpose(int m, int n, int nnz, const int *ro, const int *ci, int num_tiles,
                            int tile_items, const int *tile_row, const int *tile_nz, TransposeOut out,
                            cudaStream_t stream);

// L2-sized buckets for bringing CSR-ordered data into CSC order (see lb_transpose.cu).
// log2 of the bucket size in CSC entries; one bucket means no bucketing is needed.
int value_bucket_shift(long long nnz);
// bucket_pos[k] (position of CSR entry k in bucket order) and bucket_perm[p] (position in
// bucket order of the entry CSC entry p needs), from perm.
cudaError_t build_value_buckets(int nnz, int shift, const int *perm, int *bucket_pos, int *bucket_perm,
                                cudaStream_t stream);
// One streaming pass over the nonzeros in CSR order, over the forward's warp tiles (merge-path
// tiles of merge_tile_items(8) or (16) items): the scaled values pv[pos(k)] = values[k] *
// g[row(k)] with pos = bucket_pos (identity when null), when pv is given, and
// dv[k] = g[row(k)] * xg[k] when xg and dv are given (FP32, or the 16-bit values' type vdt
// when dv_narrow).
cudaError_t launch_csr_backward(lb_dtype vdt, int num_tiles, int tile_items, int m, int nnz, const int *tile_row,
                                const int *tile_nz, const int *row_end, const float *g, const void *values,
                                const int *bucket_pos, float *pv, const float *xg, void *dv, bool dv_narrow,
                                cudaStream_t stream);

// rowid[k] = the row of nonzero k, over the forward block tiles.
cudaError_t launch_tile_row_ids(int num_tiles, int tile_items, const int *tile_row, const int *tile_nz,
                                const int *row_end, int *rowid, cudaStream_t stream);
// The same pass adding v[k] * g[row(k)] into dx[col_idx[k]] with float reductions (dx zeroed
// by the caller; not bit-reproducible), and dv[k] = g[row(k)] * xg[k] when dv is given.
cudaError_t launch_csr_backward_scatter(lb_dtype vdt, int num_tiles, int tile_items, int m, int n, int nnz,
                                        const int *tile_row,
                                        const int *tile_nz, const int *row_end, const float *g, const void *values,
                                        const int *ci, float *dx, const float *xg, void *dv, bool dv_narrow,
                                        cudaStream_t stream);

// Batched-plan helpers.
// Thread-mapped SpMV over a batch's block-diagonal matrix (rows longer than a few nonzeros
// summed by the warp); every row is complete when the kernel ends (no fixup).
cudaError_t launch_batched_rows(lb_dtype vdt, long long rows, const int *ro, const int *ci, const void *val,
                                const float *x, long long x_len, float *y, int kc, const int *mat_row_base,
                                const int *mat_col_base, int G, const int *tile_row, cudaStream_t stream);
cudaError_t launch_block_diag_offsets(int count, const int *ro_pos, const int *row_base, const int *nz_base,
                                      const int *ro_concat, int total_rows, int *ro_global, cudaStream_t stream);
cudaError_t launch_tile_matrix(int num_tiles, const int *tile_nz, int count, const int *mat_nz_base,
                               int *tile_mat, cudaStream_t stream);

// SpMM C = A B (B dense n x kc row-major, C m x kc), then the fixup of the carries
// (carry_row[G], carry_val[G * kc]).  The wide and warp kernels run over warp tiles of
// spmm_warp_tile_items() items (a tile that fails the tile check records LB_ERR_BAD_MATRIX in
// err): the wide kernel where spmm_wide_ok holds (kc = 8 or 16, B, C and the carries 32-byte
// aligned), the warp kernel for kc <= 4.  Otherwise: the block kernel over block tiles of at
// most 2048 items.
int spmm_warp_tile_items();
bool spmm_wide_ok(int kc, const float *B, const float *C);
cudaError_t launch_spmm_wide(lb_dtype vdt, int G, int m, int n, int nnz, int kc, const int *tile_row,
                             const int *tile_nz, const int *row_end, const int *ci, const void *values, const float *B,
                             float *C, int *carry_row, float *carry_val, int *err, cudaStream_t st);
cudaError_t launch_spmm_warp(lb_dtype vdt, int G, int m, int n, int nnz, int kc, const int *tile_row,
                             const int *tile_nz, const int *row_end, const int *ci, const void *values, const float *B,
                             float *C, int *carry_row, float *carry_val, int *err, cudaStream_t st);
cudaError_t launch_spmm_block(lb_dtype vdt, int G, int m, int n, int kc, int tile_items, const int *tile_row,
                              const int *tile_nz, const int *row_end, const int *ci, const void *values,
                              const float *B, float *C, int *carry_row, float *carry_val, cudaStream_t st);

// Nonzero splitting: tiles of nzsplit_tile_nonzeros() nonzeros; first_row / last_row[G] hold
// the rows of each tile's first and last nonzero; the SpMV clears y, writes rows with nonzeros
// and fixes up 2 * G carries.
int nzsplit_tile_nonzeros();
cudaError_t launch_nz_partition(int G, int m, int nnz, const int *ro, int *first_row, int *last_row,
                                cudaStream_t st);
cudaError_t launch_nzsplit(lb_dtype vdt, int G, int m, int n, int nnz, const int *first_row, const int *last_row,
                           const int *ro, const int *ci, const void *values, const float *x, float *y,
                           int *carry_row, float *carry_val, cudaStream_t st);

// Single-source shortest paths over a CSR graph (w null: unit weights); allocates its
// workspace with cudaMallocAsync and synchronizes the stream once per iteration.
cudaError_t run_sssp(int n, int nnz, const int *ro, const int *ci, const float *w, int source, float *dist,
                     int *iterations, cudaStream_t st);

// Row offsets (m + 1) of a row-sorted COO matrix; *d_status gets 1 (row out of range) | 2
// (rows decrease) | 0.
cudaError_t launch_coo_offsets(int m, int nnz, const int *row_idx, int *row_offsets, int *d_status,
                               cudaStream_t stream);

cudaError_t launch_validate(int m, int n, int nnz, const int *ro, const int *ci, int check_sorted,
                            int *d_status, cudaStream_t stream);

// Exclusive scan of n ints (in place allowed); `sums` holds scan_scratch_ints(n) ints.
cudaError_t exclusive_scan(const int *in, int *out, long long n, int *sums, cudaStream_t st);
long long scan_scratch_ints(long long n);

// Device properties of the current device (cached).
int current_sm_count();

// An NVTX range around a public call, named after it: visible on profiler timelines, and
// nearly free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define LB_NVTX_RANGE() ::lb::NvtxRange lb_nvtx_range_(__func__)

// Every device allocation of the library goes through these four calls.  They count the live
// allocations and, for tests of the out-of-memory paths, fail on demand as if the device
// were full (lb_debug_fail_allocations_after in the C ABI).
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);
cudaError_t dev_free(void *p);
cudaError_t dev_free_async(void *p, cudaStream_t st);
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t st) {
    return dev_malloc_async(reinterpret_cast<void **>(p), bytes, st);
}

// Device address of the current device's error word (looked up once per device), or nullptr.
int *device_error_ptr();

}  // namespace lb
