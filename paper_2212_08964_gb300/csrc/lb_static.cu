// lb_static.cu -- lb_spmv_static: the one-shot merge-path SpMV with a fixed, statically
// allocated device workspace, for callers that must not allocate device memory.
//
// Who cannot allocate, and why.  lb_spmv takes its per-call workspace (partition and carry
// arrays, about 16 bytes per tile) from cudaMallocAsync on the caller's stream.  Some callers
// cannot let a library do that:
//   - a process whose device memory is already reserved by another allocator (a framework's
//     caching allocator, or an arena sized to the card), where an extra allocation from the
//     CUDA default pool can fail with out-of-memory even though the call needs only a little;
//   - latency-bound loops where an allocation may block on the memory pool or the driver;
//   - code that has promised its host framework that every device allocation goes through
//     that framework's own allocator.
// For them this file keeps the workspace in a file-scope __device__ array, sized once at
// compile time, and the entry point makes no allocating call of any kind.
//
// The dissertation has no counterpart: it describes the kernels, not how their workspace is
// provided.
#include <mutex>

#include "lb_internal.cuh"

using namespace lb;

namespace {

constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;  // merge-path launch shape used by this entry point
constexpr int kIpt = 8;
constexpr int kTileItems = LB_SPMV_STATIC_TILE_ITEMS;
constexpr int kMaxTiles = LB_SPMV_STATIC_MAX_TILES;
static_assert(kTileItems == merge_tile_items(kIpt), "tile size must match the (256, 8) merge-path shape");

// Workspace layout, in 4-byte words:
//   tile_row[kMaxTiles + 1] | tile_nz[kMaxTiles + 1] | carry_row[kMaxTiles] | carry_val[kMaxTiles]
constexpr size_t kCarryRowWord = 2 * (static_cast<size_t>(kMaxTiles) + 1);
constexpr size_t kCarryValWord = kCarryRowWord + kMaxTiles;
constexpr size_t kWords = kCarryValWord + kMaxTiles;

}  // namespace

// One copy per device, loaded with this library's module (8 MiB).
static __device__ __align__(256) int g_lb_static_ws[kWords];

namespace {

// Device address of g_lb_static_ws on the current device, looked up once per device (with that
// device current) and cached; nullptr if the lookup fails.  The same first call also does the
// merge-path kernel's host-side set-up for all three value types, so no later call on the
// device does any.
int *static_workspace() {
    static int *ptrs[kMaxDevices] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    if (ptrs[dev]) return ptrs[dev];
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lb_static_ws) != cudaSuccess || !p) return nullptr;
        if (prepare_merge_f32(kThreads, kIpt) != cudaSuccess || prepare_merge_bf16(kThreads, kIpt) != cudaSuccess ||
            prepare_merge_f16(kThreads, kIpt) != cudaSuccess)
            return nullptr;
        ptrs[dev] = static_cast<int *>(p);
    }
    return ptrs[dev];
}

lb_status status_of(cudaError_t e) { return e == cudaSuccess ? LB_OK : LB_ERR_CUDA; }

}  // namespace

extern "C" lb_status lb_spmv_static(int m, int n, int nnz, const int *row_offsets, const int *col_idx,
                                    const void *values, lb_dtype vdt, const float *x, float *y,
                                    cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (m < 0 || n < 0 || nnz < 0 || ((m == 0 || n == 0) && nnz != 0)) return LB_ERR_INVALID_ARG;
    if (vdt != LB_F32 && vdt != LB_BF16 && vdt != LB_F16) return LB_ERR_INVALID_ARG;
    if (m == 0) return LB_OK;
    if (!row_offsets || !y) return LB_ERR_INVALID_ARG;
    if (nnz > 0 && (!col_idx || !values || !x)) return LB_ERR_INVALID_ARG;
    const uintptr_t vmask = vdt == LB_F32 ? 3u : 1u;
    if ((reinterpret_cast<uintptr_t>(col_idx) & 3u) || (reinterpret_cast<uintptr_t>(values) & vmask) ||
        (reinterpret_cast<uintptr_t>(x) & 3u) || (reinterpret_cast<uintptr_t>(y) & 3u))
        return LB_ERR_INVALID_ARG;
    const long long work = static_cast<long long>(m) + nnz;
    if (work > static_cast<long long>(kMaxTiles) * kTileItems) return LB_ERR_TOO_LARGE;
    if (nnz == 0) return status_of(cudaMemsetAsync(y, 0, static_cast<size_t>(m) * sizeof(float), stream));

    int *ws = static_workspace();
    int *err = device_error_ptr();
    if (!ws || !err) return LB_ERR_CUDA;
    const int G = static_cast<int>((work + kTileItems - 1) / kTileItems);
    int *tile_row = ws;
    int *tile_nz = ws + kMaxTiles + 1;
    int *carry_row = ws + kCarryRowWord;
    float *carry_val = reinterpret_cast<float *>(ws + kCarryValWord);

    // The partition writes every tile boundary and each tile writes its own carry, so nothing
    // is needed from an earlier call.  The carry rows are still filled with -1 first, a row
    // the fixup skips, so that no carry of an earlier call can ever be added again.
    cudaError_t e = cudaMemsetAsync(carry_row, 0xff, static_cast<size_t>(G) * sizeof(int), stream);
    if (e == cudaSuccess) e = launch_partition(m, nnz, row_offsets, kTileItems, tile_row, tile_nz, stream);
    if (e != cudaSuccess) return status_of(e);
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
    set_merge_alignment(a, vdt == LB_F32 ? 4 : 2);
    return status_of(launch_merge_spmv(vdt, kPlain, kThreads, kIpt, a, stream, nullptr, nullptr));
}
