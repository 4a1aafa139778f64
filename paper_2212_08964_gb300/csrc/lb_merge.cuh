// lb_merge.cuh -- persistent merge-path SpMV (work-oriented schedule) for sm_103a.
//
// The schedule is the dissertation's work-oriented merge path (Ch.3 Sec. "Work-Oriented",
// Alg. alg:work-oriented; Ch.4 Sec. "Merge-path load balancing"): rows and nonzeros count
// as one work item each, the (rows + nnz) items are cut into tiles of equal size, and a
// split of the merge of row ends with nonzero indices gives every tile its starting row and
// nonzero.  Rows completed inside a tile are written directly; the row left open at the end
// of a tile goes out as a carry and is added by the fixup pass ("Fix-up" procedure of the
// same algorithm).  The split is hierarchical as the paper describes: tiles over the whole
// matrix (computed once by the partition kernel), then threads inside a tile by a second
// merge-path search over shared memory.
//
// GB300 realisation (not in the paper, which targets V100):
//   * persistent CTAs (one wave of resident CTAs) stride over fixed-size tiles, so the
//     partition and the summation order do not depend on the SM count;
//   * each tile's row ends, column indices and values are staged in shared memory by 1-D
//     bulk TMA copies (cp.async.bulk + mbarrier), double-buffered so the next tile streams in
//     while the current one computes; the ragged (< 16 B) ends of each array slice are
//     fetched with plain loads, so any pointer alignment works;
//   * the streamed arrays carry an L2 evict-first hint, leaving L2 to the gathered x;
//   * products are formed with all of a thread's gathers in flight, then the per-thread
//     carries are combined by a block-wide segmented scan (warp shuffles + one shared-memory
//     step) instead of atomics, so results are deterministic;
//   * completed rows are staged in shared memory and written to y with coalesced stores.
#pragma once

#include <mutex>

#include "lb_internal.cuh"

namespace lb {

template <int THREADS, int IPT, int SV>
struct MergeShape {
    static constexpr int T = THREADS * IPT;  // work items per tile
    static constexpr int WARPS = THREADS / 32;
    // One stage: row ends (4 B per row), indices (4 B per atom), values or perm (SV B per
    // atom), each padded to 16 B at both ends.  rows + atoms <= T.
    static constexpr int STAGE = ((4 + SV) * T + 128 + 127) / 128 * 128;
    static constexpr size_t SMEM = 128 + 2 * (size_t)STAGE + (size_t)T * 4 + 2 * 32 * 4;
};

// Where one array slice [e_lo, e_hi) lands in a stage.  Shared memory mirrors the global
// byte address modulo 16, so the 16-byte-aligned middle of the slice moves with one bulk copy
// and at most 15 bytes at each end move with plain loads.
struct Seg {
    uint32_t first;       // stage offset of element e_lo
    uint32_t next;        // 16-byte-aligned stage offset after this slice
    uint32_t head;        // elements before the bulk part
    uint32_t tail;        // first element after the bulk part
    uint32_t count;       // elements in the slice
    uint32_t bulk_bytes;  // bytes in the bulk part (multiple of 16, may be 0)
    uintptr_t bulk_src;   // global address of the bulk part
};

__device__ __forceinline__ Seg make_seg(const void *base, long long e_lo, long long e_hi, uint32_t sz, uint32_t off) {
    const uintptr_t lo = reinterpret_cast<uintptr_t>(base) + static_cast<uintptr_t>(e_lo) * sz;
    const uintptr_t hi = reinterpret_cast<uintptr_t>(base) + static_cast<uintptr_t>(e_hi) * sz;
    const uintptr_t a0 = lo & ~static_cast<uintptr_t>(15);
    uintptr_t A = (lo + 15) & ~static_cast<uintptr_t>(15);
    if (A > hi) A = hi;
    uintptr_t B = hi & ~static_cast<uintptr_t>(15);
    if (B < A) B = A;
    Seg s;
    s.first = off + static_cast<uint32_t>(lo - a0);
    s.next = off + static_cast<uint32_t>(((hi + 15) & ~static_cast<uintptr_t>(15)) - a0);
    s.head = static_cast<uint32_t>((A - lo) / sz);
    s.tail = static_cast<uint32_t>((B - lo) / sz);
    s.count = static_cast<uint32_t>(e_hi - e_lo);
    s.bulk_bytes = static_cast<uint32_t>(B - A);
    s.bulk_src = A;
    return s;
}

template <typename V, int MODE>
struct MergeTraits {
    static constexpr uint32_t SV = (MODE == kTransposed) ? 4u : static_cast<uint32_t>(sizeof(V));
    __device__ static const void *third(const MergeArgs &a) {
        return (MODE == kTransposed) ? static_cast<const void *>(a.perm) : a.val;
    }
};

struct TileSegs {
    Seg re, idx, val;
};

template <typename V, int MODE>
__device__ __forceinline__ TileSegs tile_segs(const MergeArgs &a, int r0, int r1, int k0, int k1) {
    TileSegs t;
    t.re = make_seg(a.row_end, r0, r1, 4, 0);
    t.idx = make_seg(a.idx, k0, k1, 4, t.re.next);
    t.val = make_seg(MergeTraits<V, MODE>::third(a), k0, k1, MergeTraits<V, MODE>::SV, t.idx.next);
    return t;
}

__device__ __forceinline__ void copy_ragged(unsigned char *stage, uint32_t first, const void *gfirst, uint32_t sz,
                                            uint32_t rel) {
    const char *src = static_cast<const char *>(gfirst) + static_cast<size_t>(rel) * sz;
    unsigned char *dst = stage + first + rel * sz;
    if (sz == 4)
        *reinterpret_cast<int *>(dst) = __ldg(reinterpret_cast<const int *>(src));
    else
        *reinterpret_cast<unsigned short *>(dst) = __ldg(reinterpret_cast<const unsigned short *>(src));
}

// A tile from a valid partition has rows + atoms <= T; anything else means the offsets were
// not a valid CSR prefix sum, and the tile is skipped rather than overflow shared memory.
template <int T_ITEMS>
__device__ __forceinline__ bool tile_ok(int r0, int r1, int k0, int k1) {
    const int nr = r1 - r0, nk = k1 - k0;
    return nr >= 0 && nk >= 0 && nr + nk <= T_ITEMS;
}

// Start moving tile [r0, r1) x [k0, k1) into `stage`: thread 0 issues the bulk copies, threads
// 0..47 copy the ragged ends (at most 7 elements per end and array).
template <typename V, int MODE, int T_ITEMS>
__device__ __forceinline__ void stage_tile(const MergeArgs &a, unsigned char *stage, uint64_t *bar, int r0, int r1,
                                           int k0, int k1, uint64_t pol) {
    const int tid = threadIdx.x;
    if (!tile_ok<T_ITEMS>(r0, r1, k0, k1)) {  // malformed offsets: stage nothing
        if (tid == 0) mbar_arrive_expect_tx(bar, 0);
        return;
    }
    const TileSegs t = tile_segs<V, MODE>(a, r0, r1, k0, k1);
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, t.re.bulk_bytes + t.idx.bulk_bytes + t.val.bulk_bytes);
        if (t.re.bulk_bytes)
            bulk_g2s(stage + t.re.first + t.re.head * 4u, reinterpret_cast<const void *>(t.re.bulk_src),
                     t.re.bulk_bytes, bar, pol);
        if (t.idx.bulk_bytes)
            bulk_g2s(stage + t.idx.first + t.idx.head * 4u, reinterpret_cast<const void *>(t.idx.bulk_src),
                     t.idx.bulk_bytes, bar, pol);
        if (t.val.bulk_bytes)
            bulk_g2s(stage + t.val.first + t.val.head * MergeTraits<V, MODE>::SV,
                     reinterpret_cast<const void *>(t.val.bulk_src), t.val.bulk_bytes, bar, pol);
    }
    if (tid < 48) {
        const int which = tid >> 4;
        const bool tail = ((tid >> 3) & 1) != 0;
        const uint32_t e = tid & 7;
        const uint32_t first = which == 0 ? t.re.first : (which == 1 ? t.idx.first : t.val.first);
        const uint32_t head = which == 0 ? t.re.head : (which == 1 ? t.idx.head : t.val.head);
        const uint32_t tl = which == 0 ? t.re.tail : (which == 1 ? t.idx.tail : t.val.tail);
        const uint32_t count = which == 0 ? t.re.count : (which == 1 ? t.idx.count : t.val.count);
        const uint32_t sz = which == 2 ? MergeTraits<V, MODE>::SV : 4u;
        const void *gfirst =
            which == 0 ? static_cast<const void *>(a.row_end + r0)
                       : (which == 1 ? static_cast<const void *>(a.idx + k0)
                                     : static_cast<const void *>(static_cast<const char *>(MergeTraits<V, MODE>::third(a)) +
                                                                 static_cast<size_t>(k0) * sz));
        const uint32_t rel = tail ? tl + e : e;
        const bool ok = tail ? (rel < count) : (e < head);
        if (ok) copy_ragged(stage, first, gfirst, sz, rel);
    }
}

struct TileBounds {
    int r0, r1, k0, k1, m0, m1;
};

template <int MODE>
__device__ __forceinline__ TileBounds load_bounds(const MergeArgs &a, int tile) {
    TileBounds b;
    b.r0 = __ldg(a.tile_row + tile);
    b.r1 = __ldg(a.tile_row + tile + 1);
    b.k0 = __ldg(a.tile_nz + tile);
    b.k1 = __ldg(a.tile_nz + tile + 1);
    if (MODE == kBatched) {
        b.m0 = __ldg(a.tile_mat + tile);
        b.m1 = __ldg(a.tile_mat + tile + 1);
    } else {
        b.m0 = b.m1 = 0;
    }
    return b;
}

// Column base of nonzero k inside a tile whose nonzeros lie in matrices [m0, m1].
__device__ __forceinline__ int batched_col_base(const MergeArgs &a, int m0, int m1, int k) {
    int lo = m0, hi = m1;
    while (lo < hi) {  // largest i in [m0, m1] with mat_nz_base[i] <= k
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(a.mat_nz_base + mid) <= k)
            lo = mid;
        else
            hi = mid - 1;
    }
    return __ldg(a.mat_col_base + lo);
}

template <typename V, int THREADS, int IPT, int MODE>
__global__ void __launch_bounds__(THREADS) merge_spmv_kernel(const MergeArgs a) {
    using Sh = MergeShape<THREADS, IPT, static_cast<int>(MergeTraits<V, MODE>::SV)>;
    constexpr int T = Sh::T;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    unsigned char *stages = smem + 128;
    float *s_out = reinterpret_cast<float *>(smem + 128 + 2 * Sh::STAGE);
    int *s_wf = reinterpret_cast<int *>(s_out + T);
    float *s_wv = reinterpret_cast<float *>(s_wf + 32);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int G = a.num_tiles;
    int tile = blockIdx.x;
    if (tile >= G) return;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint64_t pol = policy_evict_first();

    TileBounds cur = load_bounds<MODE>(a, tile);
    stage_tile<V, MODE, T>(a, stages, &bar[0], cur.r0, cur.r1, cur.k0, cur.k1, pol);
    int next_tile = tile + gridDim.x;
    TileBounds nxt = {0, 0, 0, 0, 0, 0};
    if (next_tile < G) nxt = load_bounds<MODE>(a, next_tile);
    uint32_t phases = 0;

    for (int it = 0; tile < G; ++it) {
        const int s = it & 1;
        unsigned char *stage = stages + s * Sh::STAGE;

        // Stream the next tile into the other stage; fetch the bounds of the one after.
        const int after_tile = next_tile + gridDim.x;
        TileBounds aft = {0, 0, 0, 0, 0, 0};
        if (next_tile < G) {
            stage_tile<V, MODE, T>(a, stages + (s ^ 1) * Sh::STAGE, &bar[s ^ 1], nxt.r0, nxt.r1, nxt.k0, nxt.k1, pol);
            if (after_tile < G) aft = load_bounds<MODE>(a, after_tile);
        }

        const bool ok = mbar_wait_bounded(&bar[s], (phases >> s) & 1u, kWaitLimitNs);
        phases ^= 1u << s;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(a.err, static_cast<int>(LB_ERR_TIMEOUT));
            if (next_tile < G) mbar_wait_bounded(&bar[s ^ 1], (phases >> (s ^ 1)) & 1u, kWaitLimitNs);
            return;
        }

        if (!tile_ok<T>(cur.r0, cur.r1, cur.k0, cur.k1)) {
            if (tid == 0) {
                atomicExch(a.err, static_cast<int>(LB_ERR_BAD_MATRIX));
                a.carry_row[tile] = a.num_rows;  // the fixup skips it
                a.carry_val[tile] = 0.f;
            }
        } else {
        const int nr = cur.r1 - cur.r0;
        const int nk = cur.k1 - cur.k0;
        const int k0 = cur.k0;
        const TileSegs segs = tile_segs<V, MODE>(a, cur.r0, cur.r1, cur.k0, cur.k1);
        const int *s_re = reinterpret_cast<const int *>(stage + segs.re.first);
        const int *s_idx = reinterpret_cast<const int *>(stage + segs.idx.first);
        float *s_y = s_out;
        float *s_p = s_out + nr;

        // 1. Products of the tile's atoms, all of a thread's gathers in flight at once.
        {
            int col[IPT];
            float vv[IPT];
#pragma unroll
            for (int u = 0; u < IPT; ++u) {
                const int j = tid + u * THREADS;
                col[u] = 0;
                vv[u] = 0.f;
                if (j < nk) {
                    col[u] = s_idx[j];
                    if (MODE == kTransposed) {
                        const int p = reinterpret_cast<const int *>(stage + segs.val.first)[j];
                        vv[u] = to_f32(__ldg(static_cast<const V *>(a.val) + p));
                    } else {
                        vv[u] = to_f32(reinterpret_cast<const V *>(stage + segs.val.first)[j]);
                    }
                    if (MODE == kBatched) col[u] += batched_col_base(a, cur.m0, cur.m1, k0 + j);
                }
            }
            float xv[IPT];
#pragma unroll
            for (int u = 0; u < IPT; ++u) {
                const int j = tid + u * THREADS;
                xv[u] = (j < nk) ? __ldg(a.x + col[u]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < IPT; ++u) {
                const int j = tid + u * THREADS;
                if (j < nk) s_p[j] = vv[u] * xv[u];
            }
        }
        __syncthreads();

        // 2. Thread-level merge path inside the tile: find this thread's start on diagonal
        //    d0, then consume its items (row ends close a row, nonzeros accumulate).
        const int items = nr + nk;
        const int d0 = min(tid * IPT, items);
        const int d1 = min(d0 + IPT, items);
        int lo = max(0, d0 - nk), hi = min(d0, nr);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (mid + (s_re[mid] - k0) < d0)
                lo = mid + 1;
            else
                hi = mid;
        }
        int i = lo, j = d0 - lo;
        float acc = 0.f, head = 0.f;
        int head_row = -1;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (d0 + q < d1) {
                if (i < nr && s_re[i] - k0 <= j) {
                    if (head_row < 0) {
                        head = acc;
                        head_row = i;
                    } else {
                        s_y[i] = acc;
                    }
                    acc = 0.f;
                    ++i;
                } else {
                    acc += s_p[j];
                    ++j;
                }
            }
        }

        // 3. Block-wide segmented scan of (ends a row?, partial after the last row end): a
        //    thread's first completed row receives the partials of the threads before it back
        //    to the last one that ended a row.
        int fi = head_row >= 0;
        float vi = acc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float vu = __shfl_up_sync(0xffffffffu, vi, off);
            const int fu = __shfl_up_sync(0xffffffffu, fi, off);
            if (lane >= off) {
                if (!fi) vi = vu + vi;
                fi |= fu;
            }
        }
        if (lane == 31) {
            s_wf[warp] = fi;
            s_wv[warp] = vi;
        }
        __syncthreads();
        float pv = 0.f;
        for (int w = 0; w < warp; ++w) {
            const int fw = s_wf[w];
            const float vw = s_wv[w];
            pv = fw ? vw : pv + vw;
        }
        float ve = __shfl_up_sync(0xffffffffu, vi, 1);
        int fe = __shfl_up_sync(0xffffffffu, fi, 1);
        if (lane == 0) {
            ve = 0.f;
            fe = 0;
        }
        if (head_row >= 0) s_y[head_row] = head + (fe ? ve : pv + ve);
        if (tid == THREADS - 1) {
            a.carry_row[tile] = cur.r1;
            a.carry_val[tile] = fi ? vi : pv + vi;
        }
        __syncthreads();

        // 4. Completed rows of the tile, coalesced.
        for (int r = tid; r < nr; r += THREADS) a.y[cur.r0 + r] = s_y[r];
        }

        tile = next_tile;
        cur = nxt;
        next_tile = after_tile;
        nxt = aft;
        fence_proxy_async_smem();
        __syncthreads();
    }
}

// Resident CTAs per SM of one kernel instance on the current device (computed once per
// device; also raises the kernel's dynamic shared-memory limit).
template <typename V, int THREADS, int IPT, int MODE>
int merge_blocks_per_sm() {
    using Sh = MergeShape<THREADS, IPT, static_cast<int>(MergeTraits<V, MODE>::SV)>;
    constexpr int kMaxDev = 64;
    static int cache[kMaxDev] = {0};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 0;
    if (cache[dev] > 0) return cache[dev];
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        auto kern = merge_spmv_kernel<V, THREADS, IPT, MODE>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(Sh::SMEM)) !=
            cudaSuccess)
            return 0;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, THREADS, Sh::SMEM) != cudaSuccess) return 0;
        cache[dev] = nb > 0 ? nb : 1;
    }
    return cache[dev];
}

template <typename V, int THREADS, int IPT, int MODE>
cudaError_t launch_merge_cfg(const MergeArgs &a, cudaStream_t st, cudaEvent_t eb, cudaEvent_t ea) {
    using Sh = MergeShape<THREADS, IPT, static_cast<int>(MergeTraits<V, MODE>::SV)>;
    const int per_sm = merge_blocks_per_sm<V, THREADS, IPT, MODE>();
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const long long wave = static_cast<long long>(per_sm) * current_sm_count();
    const int grid = static_cast<int>(a.num_tiles < wave ? a.num_tiles : wave);
    if (eb) cudaEventRecord(eb, st);
    merge_spmv_kernel<V, THREADS, IPT, MODE><<<grid, THREADS, Sh::SMEM, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (ea) cudaEventRecord(ea, st);
    if (e != cudaSuccess) return e;
    return launch_fixup(a.num_tiles, a.num_rows, a.carry_row, a.carry_val, a.y, st);
}

// The (threads, items per thread) shapes compiled into the library.
#define LB_MERGE_SHAPES(X) X(128, 8) X(256, 4) X(256, 8) X(256, 12) X(256, 16) X(512, 8)

template <typename V, int MODE>
cudaError_t dispatch_merge_shape(int threads, int ipt, const MergeArgs &a, cudaStream_t st, cudaEvent_t eb,
                                 cudaEvent_t ea) {
#define LB_TRY_SHAPE(TH, IP) \
    if (threads == TH && ipt == IP) return launch_merge_cfg<V, TH, IP, MODE>(a, st, eb, ea);
    LB_MERGE_SHAPES(LB_TRY_SHAPE)
#undef LB_TRY_SHAPE
    return cudaErrorInvalidValue;
}

template <typename V>
cudaError_t dispatch_merge(int mode, int threads, int ipt, const MergeArgs &a, cudaStream_t st, cudaEvent_t eb,
                           cudaEvent_t ea) {
    if (a.num_tiles <= 0) return cudaSuccess;
    switch (mode) {
        case kPlain:
            return dispatch_merge_shape<V, kPlain>(threads, ipt, a, st, eb, ea);
        case kBatched:
            return dispatch_merge_shape<V, kBatched>(threads, ipt, a, st, eb, ea);
        case kTransposed:
            return dispatch_merge_shape<V, kTransposed>(threads, ipt, a, st, eb, ea);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace lb
