// lb_api.cu -- the C ABI of liblbspmv (declared in include/lbspmv.h).
//
// Host-side only: argument checks, plan objects, schedule selection and kernel dispatch.
// Every step of the computation runs in this library's kernels.
#include <atomic>
#include <climits>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "lb_internal.cuh"

using namespace lb;

// Device error word (per device; a kernel that skips a malformed tile writes here).
__device__ int g_lb_device_error = 0;

// ------------------------------------------------------------------------------------------
// Device allocations: counted, and failed on demand for tests of the out-of-memory paths.

namespace {
std::atomic<long long> g_live_allocs{0};
std::atomic<long long> g_alloc_budget{-1};  // allocations left before failures start; -1: no limit

bool take_allocation() {
    long long b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) return false;
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) return true;
    }
    return true;
}
}  // namespace

namespace lb {
cudaError_t dev_malloc(void **p, size_t bytes) {
    *p = nullptr;
    if (!take_allocation()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ++g_live_allocs;
    return e;
}
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (!take_allocation()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) ++g_live_allocs;
    return e;
}
cudaError_t dev_free(void *p) {
    if (!p) return cudaSuccess;
    --g_live_allocs;
    return cudaFree(p);
}
cudaError_t dev_free_async(void *p, cudaStream_t st) {
    if (!p) return cudaSuccess;
    --g_live_allocs;
    return cudaFreeAsync(p, st);
}
}  // namespace lb

extern "C" void lb_debug_fail_allocations_after(int count) { g_alloc_budget.store(count < 0 ? -1 : count); }

extern "C" long long lb_debug_live_allocations(void) { return g_live_allocs.load(); }

namespace {

constexpr int kMaxDevices = 64;
constexpr int kDefaultThreads = 256;
constexpr int kDefaultIpt = 8;

cudaEvent_t g_ev_before = nullptr;
cudaEvent_t g_ev_after = nullptr;

int *device_error_word() {
    static int *ptrs[kMaxDevices] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    if (ptrs[dev]) return ptrs[dev];
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lb_device_error) != cudaSuccess) return nullptr;
        ptrs[dev] = static_cast<int *>(p);
    }
    return ptrs[dev];
}

bool merge_shape_ok(int threads, int ipt) {
    static const int shapes[][2] = {{128, 16}, {256, 8}, {256, 16}, {384, 8}, {512, 8}};
    for (const auto &s : shapes)
        if (s[0] == threads && s[1] == ipt) return true;
    return false;
}

bool dtype_ok(lb_dtype d) { return d == LB_F32 || d == LB_BF16 || d == LB_F16; }

bool sched_ok(lb_schedule s) { return s >= LB_SCHED_AUTO && s <= LB_SCHED_NONZERO_SPLIT; }

// Resolve a requested schedule and tuning into concrete values, or report an invalid request.
bool resolve(int m, int n, int nnz, lb_schedule s, const lb_tuning *t, lb_schedule *out_s, lb_tuning *out_t) {
    lb_tuning r = t ? *t : lb_tuning{0, 0, 0};
    if (s == LB_SCHED_AUTO) {
        // Ch.4 Sec. "Improved Performance Response": merge-path unless rows or columns are below
        // alpha = 500 and the nonzeros below beta = 10000; then thread- or group-mapped.  The
        // paper leaves the choice between those two open; short rows go to thread-mapped, longer
        // ones to the smallest group covering the mean row length.
        const long long mn = m < n ? m : n;
        if (mn < 500 && nnz < 10000) {
            const double mean = m > 0 ? static_cast<double>(nnz) / m : 0.0;
            if (mean <= 4.0) {
                s = LB_SCHED_THREAD_MAPPED;
            } else {
                int g = 4;
                while (g < 32 && g < mean) g <<= 1;
                s = LB_SCHED_GROUP_MAPPED;
                r.group_size = g;
            }
        } else {
            s = LB_SCHED_MERGE_PATH;
        }
    }
    switch (s) {
        case LB_SCHED_MERGE_PATH:
            if (r.threads == 0) r.threads = kDefaultThreads;
            if (r.items_per_thread == 0) r.items_per_thread = kDefaultIpt;
            if (!merge_shape_ok(r.threads, r.items_per_thread)) return false;
            break;
        case LB_SCHED_THREAD_MAPPED:
            break;
        case LB_SCHED_WARP_MAPPED:
            r.group_size = 32;
            break;
        case LB_SCHED_BLOCK_MAPPED:
            if (r.threads == 0) r.threads = 256;
            if (r.threads != 128 && r.threads != 256) return false;
            break;
        case LB_SCHED_GROUP_MAPPED:
            if (r.group_size == 0) r.group_size = 32;
            if (r.group_size != 4 && r.group_size != 8 && r.group_size != 16 && r.group_size != 32) return false;
            break;
        case LB_SCHED_NONZERO_SPLIT:
            r = lb_tuning{0, 0, 0};  // fixed: 256 threads x 8 nonzeros per tile
            break;
        default:
            return false;
    }
    *out_s = s;
    *out_t = r;
    return true;
}

lb_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return LB_OK;
    if (e == cudaErrorMemoryAllocation) return LB_ERR_NO_MEMORY;
    return LB_ERR_CUDA;
}

bool sizes_ok(int m, int n, int nnz) {
    if (m < 0 || n < 0 || nnz < 0) return false;
    if (m == 0 && nnz != 0) return false;
    if (n == 0 && nnz != 0) return false;
    return true;
}

// Work items per tile of the block-level passes over the forward partition (the CSR-order
// backward pass, dvalues, the transpose and SpMM): threads * items_per_thread slots, less 8.
int cta_tile_items(int threads, int ipt) { return threads * ipt - 8; }

size_t value_bytes(lb_dtype d) { return d == LB_F32 ? 4 : 2; }

// Pointers must be aligned to their element type (the kernels use vector accesses).
bool aligned(const void *p, size_t bytes) { return (reinterpret_cast<uintptr_t>(p) & (bytes - 1)) == 0; }

int num_tiles_of(long long m, long long nnz, int tile_items) {
    const long long W = m + nnz;
    return static_cast<int>((W + tile_items - 1) / tile_items);
}

template <typename P>
cudaError_t dmalloc(P **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return dev_malloc(reinterpret_cast<void **>(p), count * sizeof(P));
}

}  // namespace

int *lb::device_error_ptr() { return device_error_word(); }

struct lb_plan {
    int device = -1;
    int m = 0, n = 0, nnz = 0;
    lb_schedule sched = LB_SCHED_MERGE_PATH;
    lb_tuning tune = {0, 0, 0};
    int tile_items = 0;
    int G = 0;
    int *ro = nullptr;
    int *tile_row = nullptr, *tile_nz = nullptr, *carry_row = nullptr;
    float *carry_val = nullptr;
    // Warp tiles (merge_tile_items(items_per_thread) items): the merge-path forward and the
    // per-nonzero passes of the backward.
    int wG = 0, w_tile_items = 0;
    int *w_tile_row = nullptr, *w_tile_nz = nullptr, *w_carry_row = nullptr;
    float *w_carry_val = nullptr;
    bool has_t = false;
    int Gt = 0, t_tile_items = 0;  // warp tiles of the transposed (gather-sum) product
    int *co = nullptr, *ri = nullptr, *perm = nullptr;
    int *t_tile_row = nullptr, *t_tile_nz = nullptr, *t_carry_row = nullptr;
    float *t_carry_val = nullptr;
    int bucket_shift = 0;  // 0: one L2-sized bucket (CSR order, gathered through perm)
    int *bucket_pos = nullptr, *bucket_perm = nullptr;
    float *pv = nullptr;  // per call: values[k] * g[row(k)] in bucket order (nnz floats)
    // Nonzero splitting (that schedule only): rows of each tile's first and last nonzero, and
    // two carries per tile.
    int G_nz = 0;
    int *nz_first = nullptr, *nz_last = nullptr, *nz_carry_row = nullptr;
    float *nz_carry_val = nullptr;
    // SpMM carries, allocated on first use and grown with the number of columns.
    int *mm_carry_row = nullptr;
    float *mm_carry_val = nullptr;
    long long mm_cols = 0;
    long long mm_carry_tiles = 0;
    // SpMM's 248-item warp tiles, for plans whose warp tiles have another size (made on first use).
    int *mm_tile_row = nullptr, *mm_tile_nz = nullptr;
    int mmG = 0;
};

struct lb_batched_plan {
    int device = -1;
    int count = 0, kc = 0;
    long long total_rows = 0, total_cols = 0, total_nnz = 0;
    lb_schedule sched = LB_SCHED_MERGE_PATH;
    lb_tuning tune = {0, 0, 0};
    int tile_items = 0;
    int G = 0;
    int *ro_g = nullptr, *mat_nz_base = nullptr, *mat_col_base = nullptr, *mat_row_base = nullptr;
    int *tile_row = nullptr, *tile_nz = nullptr, *tile_mat = nullptr, *carry_row = nullptr;
    float *carry_val = nullptr;
};

static void release_transpose(lb_plan *p) {
    int **ints[] = {&p->co, &p->ri, &p->perm, &p->t_tile_row, &p->t_tile_nz, &p->t_carry_row, &p->bucket_pos,
                    &p->bucket_perm};
    for (int **q : ints) {
        if (*q) dev_free(*q);
        *q = nullptr;
    }
    if (p->t_carry_val) dev_free(p->t_carry_val);
    p->t_carry_val = nullptr;
    if (p->pv) dev_free(p->pv);
    p->pv = nullptr;
    p->bucket_shift = 0;
}

static void free_plan_arrays(lb_plan *p) {
    release_transpose(p);
    int *nz_ints[] = {p->nz_first, p->nz_last, p->nz_carry_row};
    for (int *q : nz_ints)
        if (q) dev_free(q);
    if (p->nz_carry_val) dev_free(p->nz_carry_val);
    p->nz_first = p->nz_last = p->nz_carry_row = nullptr;
    p->nz_carry_val = nullptr;
    if (p->mm_carry_row) dev_free(p->mm_carry_row);
    if (p->mm_carry_val) dev_free(p->mm_carry_val);
    if (p->mm_tile_row) dev_free(p->mm_tile_row);
    if (p->mm_tile_nz) dev_free(p->mm_tile_nz);
    p->mm_tile_row = p->mm_tile_nz = nullptr;
    p->mmG = 0;
    p->mm_carry_row = nullptr;
    p->mm_carry_val = nullptr;
    p->mm_cols = 0;
    p->mm_carry_tiles = 0;
    int *ints[] = {p->ro, p->tile_row, p->tile_nz, p->carry_row, p->w_tile_row, p->w_tile_nz, p->w_carry_row};
    for (int *q : ints)
        if (q) dev_free(q);
    if (p->carry_val) dev_free(p->carry_val);
    if (p->w_carry_val) dev_free(p->w_carry_val);
}

static bool on_device(int dev) {
    int cur = -1;
    return cudaGetDevice(&cur) == cudaSuccess && cur == dev;
}

extern "C" {

const char *lb_status_string(lb_status s) {
    switch (s) {
        case LB_OK:
            return "LB_OK";
        case LB_ERR_INVALID_ARG:
            return "LB_ERR_INVALID_ARG: invalid argument";
        case LB_ERR_BAD_MATRIX:
            return "LB_ERR_BAD_MATRIX: malformed matrix";
        case LB_ERR_UNSUPPORTED:
            return "LB_ERR_UNSUPPORTED: not supported by this library";
        case LB_ERR_NO_MEMORY:
            return "LB_ERR_NO_MEMORY: device allocation failed";
        case LB_ERR_CUDA:
            return "LB_ERR_CUDA: CUDA runtime error";
        case LB_ERR_TIMEOUT:
            return "LB_ERR_TIMEOUT: reserved (no kernel of this library waits)";
        case LB_ERR_TOO_LARGE:
            return "LB_ERR_TOO_LARGE: the matrix exceeds the fixed static workspace";
        case LB_ERR_OUT_OF_RANGE:
            return "LB_ERR_OUT_OF_RANGE: an index read from the inputs lies outside its array (checked build)";
    }
    return "unknown lb_status";
}

int lb_version(void) { return 10000; }

int lb_num_tiles(int m, int nnz, int tile_items) {
    if (m < 0 || nnz < 0 || tile_items <= 0) return -1;
    return num_tiles_of(m, nnz, tile_items);
}

lb_status lb_set_profile_events(cudaEvent_t before, cudaEvent_t after) {
    g_ev_before = before;
    g_ev_after = after;
    return LB_OK;
}

lb_status lb_partition(int m, int nnz, const int *row_offsets, int tile_items, int *tile_row, int *tile_nz,
                       cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (m < 0 || nnz < 0 || tile_items <= 0 || (m == 0 && nnz != 0)) return LB_ERR_INVALID_ARG;
    if (!row_offsets || !tile_row || !tile_nz) return LB_ERR_INVALID_ARG;
    if ((static_cast<long long>(m) + nnz + tile_items - 1) / tile_items >= INT_MAX) return LB_ERR_INVALID_ARG;
    return from_cuda(launch_partition(m, nnz, row_offsets, tile_items, tile_row, tile_nz, stream));
}

lb_status lb_spmv(int m, int n, int nnz, const int *row_offsets, const int *col_idx, const void *values,
                  lb_dtype vdt, const float *x, float *y, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!sizes_ok(m, n, nnz) || !dtype_ok(vdt)) return LB_ERR_INVALID_ARG;
    if (m == 0) return LB_OK;
    if (!row_offsets || !y) return LB_ERR_INVALID_ARG;
    if (nnz > 0 && (!col_idx || !values || !x)) return LB_ERR_INVALID_ARG;
    if (nnz == 0) return from_cuda(cudaMemsetAsync(y, 0, static_cast<size_t>(m) * sizeof(float), stream));
    lb_schedule s;
    lb_tuning t;
    if (!resolve(m, n, nnz, LB_SCHED_AUTO, nullptr, &s, &t)) return LB_ERR_INVALID_ARG;
    if (s != LB_SCHED_MERGE_PATH) return from_cuda(launch_mapped(s, t, vdt, m, n, nnz, row_offsets, col_idx, values, x, y, stream));
    if (!aligned(col_idx, 4) || !aligned(values, value_bytes(vdt)) || !aligned(x, 4) || !aligned(y, 4))
        return LB_ERR_INVALID_ARG;
    int *err = device_error_word();
    if (!err) return LB_ERR_CUDA;
    const int T = merge_tile_items(t.items_per_thread);
    const int G = num_tiles_of(m, nnz, T);
    // Workspace: tile_row[G+1], tile_nz[G+1], carry_row[G], carry_val[G].
    const size_t bytes = (2 * (static_cast<size_t>(G) + 1) + static_cast<size_t>(G)) * sizeof(int) +
                         static_cast<size_t>(G) * sizeof(float);
    void *ws = nullptr;
    cudaError_t e = dev_malloc_async(&ws, bytes, stream);
    if (e != cudaSuccess) return from_cuda(e);
    int *tile_row = static_cast<int *>(ws);
    int *tile_nz = tile_row + G + 1;
    int *carry_row = tile_nz + G + 1;
    float *carry_val = reinterpret_cast<float *>(carry_row + G);
    e = launch_partition(m, nnz, row_offsets, T, tile_row, tile_nz, stream);
    if (e == cudaSuccess) {
        MergeArgs a{};
        a.num_tiles = G;
        a.num_rows = m;
        a.num_atoms = nnz;
        a.tile_row = tile_row;
        a.tile_nz = tile_nz;
        a.row_end = row_offsets + 1;
        a.idx = col_idx;
        a.val = values;
        a.x = x;
        a.x_len = n;
        a.y = y;
        a.carry_row = carry_row;
        a.carry_val = carry_val;
        a.err = err;
        set_merge_alignment(a, value_bytes(vdt));
        e = launch_merge_spmv(vdt, kPlain, t.threads, t.items_per_thread, a, stream, g_ev_before, g_ev_after);
    }
    cudaError_t e2 = dev_free_async(ws, stream);
    return from_cuda(e != cudaSuccess ? e : e2);
}

// The merge-path forward of a plan over its warp tiles (x_gathered may be null).
static lb_status planned_forward(const lb_plan *p, const int *col_idx, const void *values, lb_dtype vdt,
                                 const float *x, float *y, float *x_gathered, cudaStream_t stream) {
    if (!aligned(col_idx, 4) || !aligned(values, value_bytes(vdt)) || !aligned(x, 4) || !aligned(y, 4))
        return LB_ERR_INVALID_ARG;
    int *err = device_error_word();
    if (!err) return LB_ERR_CUDA;
    MergeArgs a{};
    a.num_tiles = p->wG;
    a.num_rows = p->m;
    a.num_atoms = p->nnz;
    a.tile_row = p->w_tile_row;
    a.tile_nz = p->w_tile_nz;
    a.row_end = p->ro + 1;
    a.idx = col_idx;
    a.val = values;
    a.x = x;
    a.x_len = p->n;
    a.y = y;
    a.carry_row = p->w_carry_row;
    a.carry_val = p->w_carry_val;
    a.xg = x_gathered;
    a.err = err;
    set_merge_alignment(a, value_bytes(vdt));
    return from_cuda(launch_merge_spmv(vdt, kPlain, p->tune.threads, p->tune.items_per_thread, a, stream, g_ev_before,
                                       g_ev_after));
}

lb_status lb_plan_create(int m, int n, int nnz, const int *row_offsets, lb_schedule s, const lb_tuning *t,
                         cudaStream_t stream, lb_plan **out) {
    LB_NVTX_RANGE();
    if (!out) return LB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!sizes_ok(m, n, nnz) || !sched_ok(s)) return LB_ERR_INVALID_ARG;
    if (!row_offsets && m > 0) return LB_ERR_INVALID_ARG;
    lb_plan *p = new (std::nothrow) lb_plan();
    if (!p) return LB_ERR_NO_MEMORY;
    if (!resolve(m, n, nnz, s, t, &p->sched, &p->tune)) {
        delete p;
        return LB_ERR_INVALID_ARG;
    }
    cudaGetDevice(&p->device);
    p->m = m;
    p->n = n;
    p->nnz = nnz;
    // The forward partition is built for every schedule (dvalues and the transpose use it).
    const int threads = p->sched == LB_SCHED_MERGE_PATH ? p->tune.threads : kDefaultThreads;
    const int ipt = p->sched == LB_SCHED_MERGE_PATH ? p->tune.items_per_thread : kDefaultIpt;
    p->tile_items = cta_tile_items(threads, ipt);
    p->G = num_tiles_of(m, nnz, p->tile_items);
    cudaError_t e = cudaSuccess;
    if ((e = dmalloc(&p->ro, static_cast<size_t>(m) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->tile_row, static_cast<size_t>(p->G) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->tile_nz, static_cast<size_t>(p->G) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->carry_row, static_cast<size_t>(p->G))) != cudaSuccess ||
        (e = dmalloc(&p->carry_val, static_cast<size_t>(p->G))) != cudaSuccess) {
        free_plan_arrays(p);
        delete p;
        return from_cuda(e);
    }
    if (m > 0) {
        e = cudaMemcpyAsync(p->ro, row_offsets, (static_cast<size_t>(m) + 1) * sizeof(int), cudaMemcpyDeviceToDevice,
                            stream);
        if (e == cudaSuccess) e = launch_partition(m, nnz, p->ro, p->tile_items, p->tile_row, p->tile_nz, stream);
    } else {
        int zero[2] = {0, 0};
        e = cudaMemcpy(p->ro, zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->tile_row, zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->tile_nz, zero, sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && m > 0) {
        // Every plan holds the warp tiles: the merge-path forward runs over them, and so do the
        // per-nonzero passes of the backward (the shape's items per lane, else 8).
        p->w_tile_items = merge_tile_items(p->sched == LB_SCHED_MERGE_PATH ? p->tune.items_per_thread : kDefaultIpt);
        p->wG = num_tiles_of(m, nnz, p->w_tile_items);
        const size_t g = static_cast<size_t>(p->wG);
        if ((e = dmalloc(&p->w_tile_row, g + 1)) == cudaSuccess && (e = dmalloc(&p->w_tile_nz, g + 1)) == cudaSuccess &&
            (e = dmalloc(&p->w_carry_row, g)) == cudaSuccess && (e = dmalloc(&p->w_carry_val, g)) == cudaSuccess)
            e = launch_partition(m, nnz, p->ro, p->w_tile_items, p->w_tile_row, p->w_tile_nz, stream);
    }
    if (e == cudaSuccess && p->sched == LB_SCHED_NONZERO_SPLIT && nnz > 0) {
        const int T = nzsplit_tile_nonzeros();
        p->G_nz = static_cast<int>((static_cast<long long>(nnz) + T - 1) / T);
        const size_t g = static_cast<size_t>(p->G_nz);
        if ((e = dmalloc(&p->nz_first, g)) == cudaSuccess && (e = dmalloc(&p->nz_last, g)) == cudaSuccess &&
            (e = dmalloc(&p->nz_carry_row, 2 * g)) == cudaSuccess && (e = dmalloc(&p->nz_carry_val, 2 * g)) == cudaSuccess)
            e = launch_nz_partition(p->G_nz, m, nnz, p->ro, p->nz_first, p->nz_last, stream);
    }
    if (e != cudaSuccess) {
        free_plan_arrays(p);
        delete p;
        return from_cuda(e);
    }
    *out = p;
    return LB_OK;
}

lb_status lb_plan_info(const lb_plan *p, lb_schedule *s, lb_tuning *t, int *num_tiles, int *tile_items) {
    if (!p) return LB_ERR_INVALID_ARG;
    if (s) *s = p->sched;
    if (t) *t = p->tune;
    if (num_tiles) *num_tiles = p->G;
    if (tile_items) *tile_items = p->tile_items;
    return LB_OK;
}

// The plan's tile sets: LB_TILES_ROWS (block tiles of the passes over the forward partition),
// LB_TILES_TRANSPOSED (warp tiles of the transposed product), LB_TILES_MERGE (warp tiles of
// the merge-path forward).
static bool plan_tiles(const lb_plan *p, int which, int *G, int *items, const int **tr, const int **tn) {
    switch (which) {
        case LB_TILES_ROWS:
            *G = p->G, *items = p->tile_items, *tr = p->tile_row, *tn = p->tile_nz;
            return true;
        case LB_TILES_TRANSPOSED:
            if (!p->has_t) return false;
            *G = p->Gt, *items = p->t_tile_items, *tr = p->t_tile_row, *tn = p->t_tile_nz;
            return true;
        case LB_TILES_MERGE:
            if (!p->w_tile_row) return false;
            *G = p->wG, *items = p->w_tile_items, *tr = p->w_tile_row, *tn = p->w_tile_nz;
            return true;
        default:
            return false;
    }
}

lb_status lb_plan_tiles(const lb_plan *p, int which, int *num_tiles, int *tile_items) {
    int G = 0, items = 0;
    const int *tr = nullptr, *tn = nullptr;
    if (!p || !plan_tiles(p, which, &G, &items, &tr, &tn)) return LB_ERR_INVALID_ARG;
    if (num_tiles) *num_tiles = G;
    if (tile_items) *tile_items = items;
    return LB_OK;
}

lb_status lb_plan_partition(const lb_plan *p, int which, int *tile_row, int *tile_nz, int *num_tiles) {
    int G = 0, items = 0;
    const int *tr = nullptr, *tn = nullptr;
    if (!p || !num_tiles || !plan_tiles(p, which, &G, &items, &tr, &tn)) return LB_ERR_INVALID_ARG;
    *num_tiles = G;
    if (!tile_row) return LB_OK;
    if (!tile_nz) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    const size_t bytes = (static_cast<size_t>(G) + 1) * sizeof(int);
    if (e == cudaSuccess) e = cudaMemcpy(tile_row, tr, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(tile_nz, tn, bytes, cudaMemcpyDeviceToHost);
    return from_cuda(e);
}

lb_status lb_spmv_planned(const lb_plan *p, const int *col_idx, const void *values, lb_dtype vdt, const float *x,
                          float *y, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p || !dtype_ok(vdt)) return LB_ERR_INVALID_ARG;
    if (p->m == 0) return LB_OK;
    if (!y || (p->nnz > 0 && (!col_idx || !values || !x))) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    if (p->nnz == 0) return from_cuda(cudaMemsetAsync(y, 0, static_cast<size_t>(p->m) * sizeof(float), stream));
    if (p->sched == LB_SCHED_NONZERO_SPLIT)
        return from_cuda(launch_nzsplit(vdt, p->G_nz, p->m, p->n, p->nnz, p->nz_first, p->nz_last, p->ro, col_idx, values, x,
                                        y, p->nz_carry_row, p->nz_carry_val, stream));
    if (p->sched != LB_SCHED_MERGE_PATH)
        return from_cuda(launch_mapped(p->sched, p->tune, vdt, p->m, p->n, p->nnz, p->ro, col_idx, values, x, y, stream));
    return planned_forward(p, col_idx, values, vdt, x, y, nullptr, stream);
}

lb_status lb_spmv_planned_save(const lb_plan *p, const int *col_idx, const void *values, lb_dtype vdt,
                               const float *x, float *y, float *x_gathered, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p || !dtype_ok(vdt)) return LB_ERR_INVALID_ARG;
    if (p->sched != LB_SCHED_MERGE_PATH) return LB_ERR_UNSUPPORTED;
    if (p->m == 0) return LB_OK;
    if (!y || (p->nnz > 0 && (!col_idx || !values || !x || !x_gathered))) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    if (p->nnz == 0) return from_cuda(cudaMemsetAsync(y, 0, static_cast<size_t>(p->m) * sizeof(float), stream));
    if (!aligned(x_gathered, 4)) return LB_ERR_INVALID_ARG;
    return planned_forward(p, col_idx, values, vdt, x, y, x_gathered, stream);
}

lb_status lb_plan_build_transpose(lb_plan *p, const int *col_idx, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p) return LB_ERR_INVALID_ARG;
    if (p->nnz > 0 && !col_idx) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    if (p->has_t) return LB_OK;
    const int n = p->n, nnz = p->nnz;
    cudaError_t e = cudaSuccess;
    // The counting pass indexes by column, so the structure is checked first (one sync; the
    // transpose is built once per structure).
    {
        int *d_status = nullptr, h_status = 0;
        if ((e = dev_malloc_async(reinterpret_cast<void **>(&d_status), sizeof(int), stream)) != cudaSuccess)
            return from_cuda(e);
        e = launch_validate(p->m, n, nnz, p->ro, col_idx, 0, d_status, stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, stream);
        dev_free_async(d_status, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return from_cuda(e);
        if (h_status != 0) return LB_ERR_BAD_MATRIX;
    }
    p->t_tile_items = merge_tile_items(kDefaultIpt);
    p->Gt = num_tiles_of(n, nnz, p->t_tile_items);
    if ((e = dmalloc(&p->co, static_cast<size_t>(n) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->ri, static_cast<size_t>(nnz))) != cudaSuccess ||
        (e = dmalloc(&p->perm, static_cast<size_t>(nnz))) != cudaSuccess ||
        (e = dmalloc(&p->t_tile_row, static_cast<size_t>(p->Gt) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->t_tile_nz, static_cast<size_t>(p->Gt) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->t_carry_row, static_cast<size_t>(p->Gt))) != cudaSuccess ||
        (e = dmalloc(&p->t_carry_val, static_cast<size_t>(p->Gt))) != cudaSuccess) {
        release_transpose(p);
        return from_cuda(e);
    }
    TransposeOut out{p->co, p->ri, p->perm};
    e = build_transpose(p->m, n, nnz, p->ro, col_idx, p->G, p->tile_items, p->tile_row, p->tile_nz, out, stream);
    if (e == cudaSuccess && nnz > 0) {
        e = dmalloc(&p->pv, static_cast<size_t>(nnz));
        const int shift = value_bucket_shift(nnz);
        if (e == cudaSuccess && ((static_cast<long long>(nnz) - 1) >> shift) > 0) {  // more than one bucket
            p->bucket_shift = shift;
            if ((e = dmalloc(&p->bucket_pos, static_cast<size_t>(nnz))) == cudaSuccess &&
                (e = dmalloc(&p->bucket_perm, static_cast<size_t>(nnz))) == cudaSuccess)
                e = build_value_buckets(nnz, shift, p->perm, p->bucket_pos, p->bucket_perm, stream);
        }
    }
    if (e == cudaSuccess) {
        if (n > 0) {
            e = launch_partition(n, nnz, p->co, p->t_tile_items, p->t_tile_row, p->t_tile_nz, stream);
        } else {
            e = cudaMemsetAsync(p->t_tile_row, 0, sizeof(int), stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->t_tile_nz, 0, sizeof(int), stream);
        }
    }
    if (e != cudaSuccess) {
        release_transpose(p);
        return from_cuda(e);
    }
    p->has_t = true;
    return LB_OK;
}

lb_status lb_plan_transpose(const lb_plan *p, int *col_offsets, int *row_idx, int *perm) {
    if (!p || !p->has_t || !col_offsets || (p->nnz > 0 && (!row_idx || !perm))) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(col_offsets, p->co, (static_cast<size_t>(p->n) + 1) * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && p->nnz > 0)
        e = cudaMemcpy(row_idx, p->ri, static_cast<size_t>(p->nnz) * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && p->nnz > 0)
        e = cudaMemcpy(perm, p->perm, static_cast<size_t>(p->nnz) * sizeof(int), cudaMemcpyDeviceToHost);
    return from_cuda(e);
}

// dx = A^T g in two passes over the plan's CSC view: the scaled values v[k] * g[row(k)] in CSR
// order into L2-sized buckets of CSC order (with dvalues alongside when asked), then the
// merge-path gather-sum over the columns.
static lb_status transposed_product(const lb_plan *p, const void *values, lb_dtype vdt, const float *g,
                                    const float *x_gathered, float *dx, void *dvalues, bool dv_narrow,
                                    cudaStream_t stream) {
    int *err = device_error_word();
    if (!err) return LB_ERR_CUDA;
    cudaError_t e = launch_csr_backward(vdt, p->wG, p->w_tile_items, p->m, p->nnz, p->w_tile_row, p->w_tile_nz,
                                        p->ro + 1, g, values, p->bucket_pos, p->pv, x_gathered, dvalues, dv_narrow,
                                        stream);
    if (e != cudaSuccess) return from_cuda(e);
    MergeArgs a{};
    a.num_tiles = p->Gt;
    a.num_rows = p->n;
    a.num_atoms = p->nnz;
    a.tile_row = p->t_tile_row;
    a.tile_nz = p->t_tile_nz;
    a.row_end = p->co + 1;
    a.idx = p->bucket_shift > 0 ? p->bucket_perm : p->perm;
    a.x = p->pv;
    a.x_len = p->nnz;
    a.y = dx;
    a.carry_row = p->t_carry_row;
    a.carry_val = p->t_carry_val;
    a.err = err;
    set_merge_alignment(a, 0);
    // The gather-sum streams only its positions, whatever the plan's forward shape: it always
    // runs the default (256, 8) shape over the transposed warp tiles.
    return from_cuda(
        launch_merge_spmv(LB_F32, kGatherSum, kDefaultThreads, kDefaultIpt, a, stream, g_ev_before, g_ev_after));
}

lb_status lb_spmv_t(const lb_plan *p, const void *values, lb_dtype vdt, const float *g, float *dx,
                    cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p || !p->has_t || !dtype_ok(vdt)) return LB_ERR_INVALID_ARG;
    if (p->n == 0) return LB_OK;
    if (!dx || (p->nnz > 0 && (!values || !g))) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    if (p->nnz == 0) return from_cuda(cudaMemsetAsync(dx, 0, static_cast<size_t>(p->n) * sizeof(float), stream));
    return transposed_product(p, values, vdt, g, nullptr, dx, nullptr, false, stream);
}

lb_status lb_spmv_backward(const lb_plan *p, const void *values, lb_dtype vdt, const float *g,
                           const float *x_gathered, float *dx, void *dvalues, lb_dtype dvdt, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p || !p->has_t || !dtype_ok(vdt) || !dx || !dvalues) return LB_ERR_INVALID_ARG;
    if (dvdt != LB_F32 && dvdt != vdt) return LB_ERR_INVALID_ARG;
    if (p->nnz > 0 && (!values || !g || !x_gathered)) return LB_ERR_INVALID_ARG;
    if (!aligned(dvalues, value_bytes(dvdt))) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    if (p->n == 0) return LB_OK;
    if (p->nnz == 0) return from_cuda(cudaMemsetAsync(dx, 0, static_cast<size_t>(p->n) * sizeof(float), stream));
    return transposed_product(p, values, vdt, g, x_gathered, dx, dvalues, dvdt != LB_F32, stream);
}

lb_status lb_spmv_backward_scatter(const lb_plan *p, const int *col_idx, const void *values, lb_dtype vdt,
                                   const float *g, const float *x_gathered, float *dx, void *dvalues, lb_dtype dvdt,
                                   cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p || !dtype_ok(vdt) || !dx) return LB_ERR_INVALID_ARG;
    if (dvdt != LB_F32 && dvdt != vdt) return LB_ERR_INVALID_ARG;
    if (dvalues && !aligned(dvalues, value_bytes(dvdt))) return LB_ERR_INVALID_ARG;
    if (p->nnz > 0 && (!col_idx || !values || !g || (dvalues && !x_gathered))) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    if (p->n == 0) return LB_OK;
    cudaError_t e = cudaMemsetAsync(dx, 0, static_cast<size_t>(p->n) * sizeof(float), stream);
    if (e != cudaSuccess || p->nnz == 0) return from_cuda(e);
    return from_cuda(launch_csr_backward_scatter(vdt, p->wG, p->w_tile_items, p->m, p->n, p->nnz, p->w_tile_row,
                                                 p->w_tile_nz, p->ro + 1, g, values, col_idx, dx, x_gathered, dvalues,
                                                 dvdt != LB_F32, stream));
}

lb_status lb_spmv_dvalues(const lb_plan *p, const int *col_idx, const float *g, const float *x, void *dvalues,
                          lb_dtype dvdt, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p || !dtype_ok(dvdt)) return LB_ERR_INVALID_ARG;
    if (p->nnz == 0) return LB_OK;
    if (!col_idx || !g || !x || !dvalues || !aligned(dvalues, value_bytes(dvdt))) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    return from_cuda(launch_dvalues(p->G, p->tile_items, p->tile_row, p->tile_nz, p->ro + 1, col_idx, g, x, p->n,
                                    dvalues, dvdt, stream));
}

lb_status lb_spmv_dvalues_gathered(const lb_plan *p, const float *g, const float *x_gathered, void *dvalues,
                                   lb_dtype dvdt, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p || !dtype_ok(dvdt)) return LB_ERR_INVALID_ARG;
    if (p->nnz == 0) return LB_OK;
    if (!g || !x_gathered || !dvalues || !aligned(dvalues, value_bytes(dvdt))) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    // The pass's value type only selects the gradient's storage here (no values are read).
    return from_cuda(launch_csr_backward(dvdt, p->wG, p->w_tile_items, p->m, p->nnz, p->w_tile_row, p->w_tile_nz,
                                         p->ro + 1, g, nullptr, nullptr, nullptr, x_gathered, dvalues, dvdt != LB_F32,
                                         stream));
}

lb_status lb_spmm_planned(lb_plan *p, const int *col_idx, const void *values, lb_dtype vdt, int kc, const float *B,
                          float *C, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p || !dtype_ok(vdt) || kc < 0) return LB_ERR_INVALID_ARG;
    if (p->m == 0 || kc == 0) return LB_OK;
    if (!C || (p->nnz > 0 && (!col_idx || !values || !B))) return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    const size_t c_bytes = static_cast<size_t>(p->m) * static_cast<size_t>(kc) * sizeof(float);
    if (p->nnz == 0) return from_cuda(cudaMemsetAsync(C, 0, c_bytes, stream));
    if (!aligned(col_idx, 4) || !aligned(values, value_bytes(vdt)) || !aligned(B, 4) || !aligned(C, 4))
        return LB_ERR_INVALID_ARG;
    int *err = device_error_word();
    if (!err) return LB_ERR_CUDA;
    // B of 8 or 16 columns, 32-byte aligned: the wide warp-tiled kernel (8 columns of B's row
    // per gather); kc <= 4: the warp-tiled kernel.  Both run over 248-item warp tiles (the
    // plan's own when they have that size, else a partition of its own, made on the first call
    // that needs it).  Other B: the block kernel over the plan's block tiles.
    const bool wide = spmm_wide_ok(kc, B, C);
    const bool warp = wide || kc <= 4;
    const int *tr = p->tile_row, *tn = p->tile_nz;
    int G = p->G;
    if (warp) {
        const int T = spmm_warp_tile_items();
        tr = p->w_tile_row, tn = p->w_tile_nz, G = p->wG;
        if (p->w_tile_items != T) {
            if (!p->mm_tile_row) {
                const int g = num_tiles_of(p->m, p->nnz, T);
                cudaError_t e = dmalloc(&p->mm_tile_row, static_cast<size_t>(g) + 1);
                if (e == cudaSuccess) e = dmalloc(&p->mm_tile_nz, static_cast<size_t>(g) + 1);
                if (e == cudaSuccess) e = launch_partition(p->m, p->nnz, p->ro, T, p->mm_tile_row, p->mm_tile_nz, stream);
                if (e != cudaSuccess) {
                    if (p->mm_tile_row) dev_free(p->mm_tile_row);
                    if (p->mm_tile_nz) dev_free(p->mm_tile_nz);
                    p->mm_tile_row = p->mm_tile_nz = nullptr;
                    return from_cuda(e);
                }
                p->mmG = g;
            }
            tr = p->mm_tile_row, tn = p->mm_tile_nz, G = p->mmG;
        }
    } else if (p->tile_items > 2048) {
        return LB_ERR_UNSUPPORTED;  // the block kernel stages tiles of up to 2048 items
    }
    if (kc > p->mm_cols || G > p->mm_carry_tiles) {
        // Carries for G tiles of kc columns; reallocated only when either grows.
        const long long cols = kc > p->mm_cols ? kc : p->mm_cols;
        const long long tiles = G > p->mm_carry_tiles ? G : p->mm_carry_tiles;
        if (p->mm_carry_row) dev_free(p->mm_carry_row);
        if (p->mm_carry_val) dev_free(p->mm_carry_val);
        p->mm_carry_row = nullptr;
        p->mm_carry_val = nullptr;
        p->mm_cols = 0;
        p->mm_carry_tiles = 0;
        cudaError_t e = dmalloc(&p->mm_carry_row, static_cast<size_t>(tiles));
        if (e == cudaSuccess) e = dmalloc(&p->mm_carry_val, static_cast<size_t>(tiles) * static_cast<size_t>(cols));
        if (e != cudaSuccess) return from_cuda(e);
        p->mm_cols = cols;
        p->mm_carry_tiles = tiles;
    }
    if (wide)
        return from_cuda(launch_spmm_wide(vdt, G, p->m, p->n, p->nnz, kc, tr, tn, p->ro + 1, col_idx, values, B, C,
                                          p->mm_carry_row, p->mm_carry_val, err, stream));
    if (warp)
        return from_cuda(launch_spmm_warp(vdt, G, p->m, p->n, p->nnz, kc, tr, tn, p->ro + 1, col_idx, values, B, C,
                                          p->mm_carry_row, p->mm_carry_val, err, stream));
    return from_cuda(launch_spmm_block(vdt, G, p->m, p->n, kc, p->tile_items, tr, tn, p->ro + 1, col_idx, values, B, C,
                                       p->mm_carry_row, p->mm_carry_val, stream));
}

void lb_plan_destroy(lb_plan *p) {
    if (!p) return;
    free_plan_arrays(p);
    delete p;
}

lb_status lb_batched_plan_create(int count, const int *h_m, const int *h_n, const int *h_nnz,
                                 const int *row_offsets_concat, lb_schedule s, const lb_tuning *t,
                                 cudaStream_t stream, lb_batched_plan **out) {
    LB_NVTX_RANGE();
    if (!out) return LB_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 0 || (count > 0 && (!h_m || !h_n || !h_nnz))) return LB_ERR_INVALID_ARG;
    if (!sched_ok(s)) return LB_ERR_INVALID_ARG;
    if (s != LB_SCHED_AUTO && s != LB_SCHED_MERGE_PATH && s != LB_SCHED_THREAD_MAPPED) return LB_ERR_UNSUPPORTED;
    lb_tuning r = t ? *t : lb_tuning{0, 0, 0};
    if (s == LB_SCHED_THREAD_MAPPED) {
        if (r.threads != 0 && r.threads != kDefaultThreads) return LB_ERR_INVALID_ARG;
        r = lb_tuning{0, 0, 0};  // the partition below still uses the default merge tiles
    }
    if (r.threads == 0) r.threads = kDefaultThreads;
    if (r.items_per_thread == 0) r.items_per_thread = kDefaultIpt;
    if (!merge_shape_ok(r.threads, r.items_per_thread)) return LB_ERR_INVALID_ARG;
    // Host bases over the non-empty matrices.
    std::vector<int> ro_pos, row_base(1, 0), nz_base(1, 0), col_base;
    long long rows = 0, cols = 0, nnz = 0, pos = 0;
    for (int i = 0; i < count; ++i) {
        if (!sizes_ok(h_m[i], h_n[i], h_nnz[i])) return LB_ERR_INVALID_ARG;
        if (h_m[i] > 0) {
            ro_pos.push_back(static_cast<int>(pos));
            rows += h_m[i];
            nnz += h_nnz[i];
            if (rows >= INT_MAX || nnz >= INT_MAX || pos >= INT_MAX) return LB_ERR_INVALID_ARG;
            row_base.push_back(static_cast<int>(rows));
            nz_base.push_back(static_cast<int>(nnz));
            col_base.push_back(static_cast<int>(cols));
        }
        pos += static_cast<long long>(h_m[i]) + 1;
        cols += h_n[i];
        if (cols >= INT_MAX) return LB_ERR_INVALID_ARG;
    }
    if (rows > 0 && !row_offsets_concat) return LB_ERR_INVALID_ARG;
    lb_batched_plan *p = new (std::nothrow) lb_batched_plan();
    if (!p) return LB_ERR_NO_MEMORY;
    cudaGetDevice(&p->device);
    p->count = count;
    p->kc = static_cast<int>(ro_pos.size());
    p->total_rows = rows;
    p->total_cols = cols;
    p->total_nnz = nnz;
    p->sched = s == LB_SCHED_THREAD_MAPPED ? LB_SCHED_THREAD_MAPPED : LB_SCHED_MERGE_PATH;
    p->tune = r;
    p->tile_items = merge_tile_items(r.items_per_thread);
    p->G = num_tiles_of(rows, nnz, p->tile_items);
    const int kc = p->kc;
    int *d_ro_pos = nullptr;
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err) {
        if (d_ro_pos) dev_free(d_ro_pos);
        lb_batched_plan_destroy(p);
        return from_cuda(err);
    };
    if ((e = dmalloc(&p->ro_g, static_cast<size_t>(rows) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->mat_nz_base, static_cast<size_t>(kc) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->mat_col_base, static_cast<size_t>(kc) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->tile_row, static_cast<size_t>(p->G) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->tile_nz, static_cast<size_t>(p->G) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->tile_mat, static_cast<size_t>(p->G) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->carry_row, static_cast<size_t>(p->G))) != cudaSuccess ||
        (e = dmalloc(&p->carry_val, static_cast<size_t>(p->G))) != cudaSuccess ||
        (e = dmalloc(&d_ro_pos, static_cast<size_t>(kc) + 1)) != cudaSuccess ||
        (e = dmalloc(&p->mat_row_base, static_cast<size_t>(kc) + 1)) != cudaSuccess)
        return fail(e);
    if (kc == 0) {
        const int zero = 0;
        e = cudaMemcpy(p->ro_g, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->tile_row, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->tile_nz, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->tile_mat, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(e);
        dev_free(d_ro_pos);
        *out = p;
        return LB_OK;
    }
    // Synchronous copies: the host vectors die at return.
    if ((e = cudaMemcpy(d_ro_pos, ro_pos.data(), kc * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->mat_row_base, row_base.data(), (kc + 1) * sizeof(int), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(p->mat_nz_base, nz_base.data(), (kc + 1) * sizeof(int), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(p->mat_col_base, col_base.data(), kc * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e);
    e = launch_block_diag_offsets(kc, d_ro_pos, p->mat_row_base, p->mat_nz_base, row_offsets_concat,
                                  static_cast<int>(rows), p->ro_g, stream);
    if (e == cudaSuccess)
        e = launch_partition(static_cast<int>(rows), nnz, p->ro_g, p->tile_items, p->tile_row, p->tile_nz, stream);
    if (e == cudaSuccess) e = launch_tile_matrix(p->G, p->tile_nz, kc, p->mat_nz_base, p->tile_mat, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // the index scratch is freed below
    if (e != cudaSuccess) return fail(e);
    dev_free(d_ro_pos);
    *out = p;
    return LB_OK;
}

lb_status lb_batched_plan_schedule(const lb_batched_plan *p, lb_schedule *s) {
    if (!p || !s) return LB_ERR_INVALID_ARG;
    *s = p->sched;
    return LB_OK;
}

lb_status lb_batched_plan_info(const lb_batched_plan *p, lb_tuning *t, int *num_tiles, int *tile_items) {
    if (!p) return LB_ERR_INVALID_ARG;
    if (t) *t = p->tune;
    if (num_tiles) *num_tiles = p->G;
    if (tile_items) *tile_items = p->tile_items;
    return LB_OK;
}

lb_status lb_batched_plan_partition(const lb_batched_plan *p, int *tile_row, int *tile_nz, int *num_tiles) {
    if (!p || !num_tiles) return LB_ERR_INVALID_ARG;
    *num_tiles = p->G;
    if (!tile_row) return LB_OK;
    if (!tile_nz || !on_device(p->device)) return LB_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    const size_t bytes = (static_cast<size_t>(p->G) + 1) * sizeof(int);
    if (e == cudaSuccess) e = cudaMemcpy(tile_row, p->tile_row, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(tile_nz, p->tile_nz, bytes, cudaMemcpyDeviceToHost);
    return from_cuda(e);
}

lb_status lb_spmv_batched(const lb_batched_plan *p, const int *col_idx_concat, const void *values_concat,
                          lb_dtype vdt, const float *x_concat, float *y_concat, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!p || !dtype_ok(vdt)) return LB_ERR_INVALID_ARG;
    if (p->total_rows == 0) return LB_OK;
    if (!y_concat || (p->total_nnz > 0 && (!col_idx_concat || !values_concat || !x_concat)))
        return LB_ERR_INVALID_ARG;
    if (!on_device(p->device)) return LB_ERR_INVALID_ARG;
    if (p->total_nnz == 0)
        return from_cuda(cudaMemsetAsync(y_concat, 0, static_cast<size_t>(p->total_rows) * sizeof(float), stream));
    if (!aligned(col_idx_concat, 4) || !aligned(values_concat, value_bytes(vdt)) || !aligned(x_concat, 4) ||
        !aligned(y_concat, 4))
        return LB_ERR_INVALID_ARG;
    if (p->sched == LB_SCHED_THREAD_MAPPED) {
        if (g_ev_before) cudaEventRecord(g_ev_before, stream);
        const cudaError_t e = launch_batched_rows(vdt, p->total_rows, p->ro_g, col_idx_concat, values_concat, x_concat,
                                                  p->total_cols, y_concat, p->kc, p->mat_row_base, p->mat_col_base,
                                                  p->G, p->tile_row, stream);
        if (g_ev_after) cudaEventRecord(g_ev_after, stream);
        return from_cuda(e);
    }
    int *err = device_error_word();
    if (!err) return LB_ERR_CUDA;
    MergeArgs a{};
    a.num_tiles = p->G;
    a.num_rows = static_cast<int>(p->total_rows);
    a.num_atoms = static_cast<int>(p->total_nnz);
    a.tile_row = p->tile_row;
    a.tile_nz = p->tile_nz;
    a.row_end = p->ro_g + 1;
    a.idx = col_idx_concat;
    a.val = values_concat;
    a.x = x_concat;
    a.x_len = p->total_cols;
    a.y = y_concat;
    a.carry_row = p->carry_row;
    a.carry_val = p->carry_val;
    a.mat_nz_base = p->mat_nz_base;
    a.mat_col_base = p->mat_col_base;
    a.tile_mat = p->tile_mat;
    a.err = err;
    set_merge_alignment(a, value_bytes(vdt));
    return from_cuda(launch_merge_spmv(vdt, kBatched, p->tune.threads, p->tune.items_per_thread, a, stream,
                                       g_ev_before, g_ev_after));
}

void lb_batched_plan_destroy(lb_batched_plan *p) {
    if (!p) return;
    int *ints[] = {p->ro_g,    p->mat_nz_base, p->mat_col_base, p->mat_row_base,
                   p->tile_row, p->tile_nz,     p->tile_mat,     p->carry_row};
    for (int *q : ints)
        if (q) dev_free(q);
    if (p->carry_val) dev_free(p->carry_val);
    delete p;
}

lb_status lb_sssp(int n, int nnz, const int *row_offsets, const int *col_idx, const float *weights, int source,
                  float *dist, int *iterations, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (n <= 0 || nnz < 0 || source < 0 || source >= n || !row_offsets || !dist || !iterations) return LB_ERR_INVALID_ARG;
    if (nnz > 0 && !col_idx) return LB_ERR_INVALID_ARG;
    return from_cuda(run_sssp(n, nnz, row_offsets, col_idx, weights, source, dist, iterations, stream));
}

lb_status lb_coo_row_offsets(int m, int nnz, const int *row_idx, int *row_offsets, int *d_status,
                             cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (m < 0 || nnz < 0 || (m == 0 && nnz != 0) || !row_offsets || !d_status || (nnz > 0 && !row_idx))
        return LB_ERR_INVALID_ARG;
    return from_cuda(launch_coo_offsets(m, nnz, row_idx, row_offsets, d_status, stream));
}

lb_status lb_validate_csr(int m, int n, int nnz, const int *row_offsets, const int *col_idx, int check_sorted,
                          int *d_status, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!sizes_ok(m, n, nnz) || !d_status || !row_offsets || (nnz > 0 && !col_idx)) return LB_ERR_INVALID_ARG;
    return from_cuda(launch_validate(m, n, nnz, row_offsets, col_idx, check_sorted, d_status, stream));
}

lb_status lb_device_error(int *status, int clear) {
    if (!status) return LB_ERR_INVALID_ARG;
    int *w = device_error_word();
    if (!w) return LB_ERR_CUDA;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status, w, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && clear) e = cudaMemset(w, 0, sizeof(int));
    return from_cuda(e);
}

}  // extern "C"

namespace lb {

void set_merge_alignment(MergeArgs &a, size_t value_bytes) {
    // The kernel's lanes start 32-byte aligned in the index array; the values (and the saved
    // gathers) take the same vector loads and stores when their own phase matches.
    const uintptr_t ip = reinterpret_cast<uintptr_t>(a.idx);
    const uintptr_t iph = (ip >> 2) & 7u;
    const uintptr_t vp = reinterpret_cast<uintptr_t>(a.val);
    const uintptr_t xp = reinterpret_cast<uintptr_t>(a.xg);
    a.vec_vals = 0;
    if (a.val && value_bytes == 4) a.vec_vals = (vp & 3u) == 0 && ((vp >> 2) & 7u) == iph;
    if (a.val && value_bytes == 2) a.vec_vals = (vp & 1u) == 0 && ((vp >> 1) & 7u) == iph;
    a.vec_xg = a.xg != nullptr && (xp & 3u) == 0 && ((xp >> 2) & 7u) == iph;
}

cudaError_t launch_merge_spmv(lb_dtype vdt, int mode, int threads, int ipt, const MergeArgs &a, cudaStream_t stream,
                              cudaEvent_t ev_before, cudaEvent_t ev_after) {
    if (mode == kGatherSum) return launch_merge_f32(mode, threads, ipt, a, stream, ev_before, ev_after);
    switch (vdt) {
        case LB_F32:
            return launch_merge_f32(mode, threads, ipt, a, stream, ev_before, ev_after);
        case LB_BF16:
            return launch_merge_bf16(mode, threads, ipt, a, stream, ev_before, ev_after);
        case LB_F16:
            return launch_merge_f16(mode, threads, ipt, a, stream, ev_before, ev_after);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lb
