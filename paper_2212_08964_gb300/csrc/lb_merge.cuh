// lb_merge.cuh -- persistent, warp-specialized merge-path SpMV (work-oriented schedule) for sm_103a.
//
// The schedule is the dissertation's work-oriented merge path (Ch.3 Sec. "Work-Oriented",
// Alg. alg:work-oriented; Ch.4 Sec. "Merge-path load balancing"): rows and nonzeros count
// as one work item each, the (rows + nnz) items are cut into tiles of equal size, and a
// split of the merge of row ends with nonzero indices gives every tile its starting row and
// nonzero.  Rows completed inside a tile are written directly; the row left open at the end
// of a tile goes out as a carry and is added by the fixup pass ("Fix-up" procedure of the
// same algorithm).  The tile-level split is computed once by the partition kernel.
//
// Inside a tile the paper splits the work again, by a second merge-path search per thread,
// and walks row ends and nonzeros one by one.  This kernel keeps the tile split and computes
// the same row sums with a segmented scan over the tile's nonzeros: products, one bit per
// position where a row starts, a scan that restarts at those bits, and each row's sum read at
// its last nonzero.  No atomics touch y and the summation order is fixed, so results are
// deterministic.
//
// GB300 realisation.  Random 4-byte gathers of x are the limiting resource (the L1 handles
// one scattered sector per cycle), so the kernel is organised to keep them issuing without
// pause, with three warp roles per CTA connected by shared-memory mbarriers:
//   * a producer warp moves each tile's row ends, indices and values into a shared-memory
//     stage with 1-D bulk TMA copies (three stages in flight);
//   * gather warps (GW) read their IPT consecutive slots of a staged tile with vector loads,
//     issue the x gathers, build their slots' row-start bits from the staged row ends while
//     the gathers are in flight, then scan their own products (restarting at row starts)
//     into one of two product buffers, with one aggregate per thread.  When the forward saves
//     its gathers for the values gradient, a warp writes them over its own staged indices and
//     stores them 32 consecutive per instruction before it releases the stage;
//   * scan warps (SW): the first scans the gather threads' aggregates into the carry into
//     each thread's first row; then all of them read each finished row's sum at its last
//     nonzero, write y with coalesced stores, and write the open row's partial sum as the
//     tile's carry.
// Stages and product buffers are recycled through "done" barriers, so no role waits for
// another except when a buffer is genuinely empty or full.  Every wait is bounded: a kernel
// that gives up records LB_ERR_TIMEOUT and returns.
//
// Persistent CTAs (one wave) take tiles blockIdx.x + i * gridDim.x, so the partition and the
// summation order do not depend on the SM count.  Shared memory mirrors global addresses
// modulo 16: a slice whose 16-byte aligned superset lies inside its array moves with one bulk
// copy; slices touching an array's first or last 8 elements also move their ragged ends with
// plain loads.  The streamed arrays carry an L2 evict-first hint, leaving L2 to x.
#pragma once

#include <mutex>
#include <type_traits>

#include "lb_internal.cuh"

namespace lb {

// Shape of one CTA: GW gather warps with IPT slots per thread; a tile holds T slots.  SV is
// the size of a staged value (0 for the gather-sum, which stages only row ends and positions);
// NS is the number of shared-memory stages, NB the number of product buffers, RB the register
// budget per thread that sets the resident CTAs per SM.
template <int GW, int IPT, int SV, int NS, int NB, int RB>
struct MergeShape {
    static_assert(IPT == 8 || IPT == 16, "items per thread: 8 or 16 (one byte or halfword of flags)");
    static constexpr int GT = GW * 32;   // gather threads
    static constexpr int T = GT * IPT;   // slots per tile
    // Work items per tile: a tile's first nonzero sits up to 7 slots past a 16-byte boundary,
    // so 8 slots are kept free for that lead.
    static constexpr int TILE_ITEMS = T - 8;
    static constexpr int SW = 4;                  // scan warps
    static constexpr int ST = SW * 32;            // scan threads
    static constexpr int GPS = GT / ST;           // gather threads per scan thread
    static constexpr int THREADS = GT + ST + 32;  // + one producer warp
    static constexpr int NSTAGE = NS;
    // One stage: row ends (4 B per row), indices (4 B per atom), values (SV B per atom, none
    // for the gather-sum product), each padded to 16 B at both ends.  rows + atoms <= T.
    static constexpr int STAGE = ((4 + SV) * T + 128 + 127) / 128 * 128;
    static constexpr int P_FLOATS = T + (T / 32) * 4;  // slot values with 4 floats of padding per 32
    static constexpr int HDR = 512;                    // mbarriers + stage headers
    // Row-start bits of each gather warp's slots (IPT words per warp, private to the warp).
    static constexpr size_t BITS = (static_cast<size_t>(GW) * IPT * 4 + 127) / 128 * 128;
    // Per product buffer: slot values, and per gather thread its aggregate, first-segment-start
    // position and carry-in.  Buffers start 128-byte aligned (accessed as float4).
    static constexpr size_t BUF = (static_cast<size_t>(P_FLOATS) * 4 + 3 * GT * 4 + 127) / 128 * 128;
    static_assert((P_FLOATS * 4) % 16 == 0, "slot values must keep 16-byte alignment");
    static constexpr int NBUF = NB;
    static constexpr size_t SMEM = HDR + NSTAGE * static_cast<size_t>(STAGE) + BITS + NBUF * BUF;
    // Resident CTAs per SM from shared memory (228 KB per SM, 1 KB reserved per CTA), capped
    // by the register budget.
    static constexpr int BY_SMEM = static_cast<int>((228 * 1024) / (SMEM + 1024));
    static constexpr int BY_REGS = 65536 / (THREADS * RB);
    static constexpr int MIN_BLOCKS_RAW = BY_SMEM < BY_REGS ? BY_SMEM : BY_REGS;
    static constexpr int MIN_BLOCKS = MIN_BLOCKS_RAW < 1 ? 1 : MIN_BLOCKS_RAW;
};

// One product buffer in shared memory.
template <int GT>
struct ProdBuf {
    float *val;  // inclusive segmented scan of each gather thread's own slots (padded)
    float *agg;  // per gather thread: sum after its last segment start (or of all its slots)
    int *ff;     // per gather thread: first slot (0..IPT-1) starting a segment, IPT if none
    float *cin;  // per gather thread: carry into its first segment
};

// Index of slot j in a padded product buffer: 4 floats of padding after every 32 keep the
// blocked 128-bit accesses free of bank conflicts.
__device__ __forceinline__ int ppad(int j) { return j + ((j >> 5) << 2); }

// Per-stage header written by the producer before it arms the stage's mbarrier.
struct StageHdr {
    int r0, r1, k0, k1, m0, m1;
    uint32_t re_first, idx_first, val_first;
    int ok;
};

// Shared-memory mbarriers of one CTA.
struct Bars {
    uint64_t full[4];    // stage s holds tile data (producer arm + TMA bytes)
    uint64_t gdone[4];   // gather warps finished reading stage s (one arrival per gather warp)
    uint64_t sdone[4];   // scan warps finished with stage s (one arrival)
    uint64_t pready[2];  // product buffer b filled (one arrival per gather warp)
    uint64_t pfree[2];   // product buffer b consumed (one arrival)
};

// Where one array slice [e_lo, e_hi) of an array holding n_elems elements lands in a stage.
struct Seg {
    uint32_t first;       // stage offset of element e_lo
    uint32_t next;        // 16-byte-aligned stage offset after this slice
    uint32_t bulk_off;    // stage offset of the bulk copy
    uint32_t bulk_bytes;  // bytes moved by TMA (multiple of 16, may be 0)
    uint32_t head;        // elements [0, head) of the slice move by plain loads
    uint32_t tail;        // elements [tail, count) of the slice move by plain loads
    uint32_t count;       // elements in the slice
    uintptr_t bulk_src;   // global address of the bulk copy
};

__device__ __forceinline__ Seg make_seg(const void *base, long long e_lo, long long e_hi, long long n_elems,
                                        uint32_t sz, uint32_t off) {
    const uintptr_t b = reinterpret_cast<uintptr_t>(base);
    const uintptr_t lo = b + static_cast<uintptr_t>(e_lo) * sz;
    const uintptr_t hi = b + static_cast<uintptr_t>(e_hi) * sz;
    const uintptr_t a0 = lo & ~static_cast<uintptr_t>(15);
    const uintptr_t a1 = (hi + 15) & ~static_cast<uintptr_t>(15);
    Seg s;
    s.first = off + static_cast<uint32_t>(lo - a0);
    s.next = off + static_cast<uint32_t>(a1 - a0);
    s.count = static_cast<uint32_t>(e_hi - e_lo);
    if (e_hi <= e_lo) {
        s.bulk_off = off;
        s.bulk_bytes = 0;
        s.head = 0;
        s.tail = 0;
        s.bulk_src = a0;
    } else if (a0 >= b && a1 <= b + static_cast<uintptr_t>(n_elems) * sz) {
        // The aligned superset stays inside the array: one bulk copy, no plain loads.
        s.bulk_off = off;
        s.bulk_bytes = static_cast<uint32_t>(a1 - a0);
        s.head = 0;
        s.tail = s.count;
        s.bulk_src = a0;
    } else {
        uintptr_t A = (lo + 15) & ~static_cast<uintptr_t>(15);
        if (A > hi) A = hi;
        uintptr_t B = hi & ~static_cast<uintptr_t>(15);
        if (B < A) B = A;
        s.head = static_cast<uint32_t>((A - lo) / sz);
        s.tail = static_cast<uint32_t>((B - lo) / sz);
        s.bulk_bytes = static_cast<uint32_t>(B - A);
        s.bulk_off = s.first + s.head * sz;
        s.bulk_src = A;
    }
    return s;
}

template <typename V, int MODE>
struct MergeTraits {
    // Bytes per atom of the staged values; the gather-sum product stages none (its atoms are
    // the gathered values themselves).
    static constexpr uint32_t SV = (MODE == kGatherSum) ? 0u : static_cast<uint32_t>(sizeof(V));
    static constexpr int NSLICE = SV > 0 ? 3 : 2;  // staged arrays: row ends, indices[, values]
    static constexpr int NS = 3;                   // stages
    static constexpr int NB = 2;                   // product buffers
    static constexpr int RB = 56;                  // registers per thread
};

// A tile from a valid partition has rows + atoms <= TILE_ITEMS; anything else means the
// offsets were not a valid CSR prefix sum, and the tile is skipped rather than overflow
// shared memory.
template <int T_ITEMS>
__device__ __forceinline__ bool tile_ok(int r0, int r1, int k0, int k1) {
    const int nr = r1 - r0, nk = k1 - k0;
    return nr >= 0 && nk >= 0 && nr + nk <= T_ITEMS;
}

// A slice whose aligned superset stays inside its array moves entirely by TMA; only tiles
// touching the first or last 8 elements of an array can need plain loads.
__device__ __forceinline__ bool edge_tile(const MergeArgs &a, int r0, int r1, int k0, int k1) {
    return r0 < 8 || r1 > a.num_rows - 8 || k0 < 8 || k1 > a.num_atoms - 8;
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

// Producer: move tile b into `stage` and arm its mbarrier (all 32 lanes of the producer warp
// call this; lane 0 writes the header and arms the barrier).
template <typename V, int MODE, int T_ITEMS>
__device__ __forceinline__ void produce_tile(const MergeArgs &a, uint64_t *bar, StageHdr *hdr, unsigned char *stage,
                                             const TileBounds &b, uint64_t pol) {
    const int lane = threadIdx.x & 31;
    // Earlier plain writes into this stage must be ordered before the new bulk writes.
    fence_proxy_async_smem();
    if (!tile_ok<T_ITEMS>(b.r0, b.r1, b.k0, b.k1)) {  // malformed offsets: stage nothing
        if (lane == 0) {
            hdr->r0 = b.r0;
            hdr->r1 = b.r1;
            hdr->k0 = b.k0;
            hdr->k1 = b.k1;
            hdr->ok = 0;
            mbar_arrive_expect_tx(bar, 0);
        }
        return;
    }
    constexpr uint32_t SV = MergeTraits<V, MODE>::SV;
    constexpr int NSL = MergeTraits<V, MODE>::NSLICE;
    constexpr unsigned kSliceMask = (1u << NSL) - 1u;
    if (!edge_tile(a, b.r0, b.r1, b.k0, b.k1)) {
        // Interior tile: every slice's aligned superset lies inside its array.  Lanes 0, 1 (and
        // 2) each place one slice (row ends, indices, values).
        if (lane < NSL) {
            const uintptr_t base = lane == 0 ? reinterpret_cast<uintptr_t>(a.row_end)
                                             : (lane == 1 ? reinterpret_cast<uintptr_t>(a.idx)
                                                          : reinterpret_cast<uintptr_t>(a.val));
            const uint32_t sz = lane == 2 ? SV : 4u;
            const uint32_t e_lo = static_cast<uint32_t>(lane == 0 ? b.r0 : b.k0);
            const uint32_t e_hi = static_cast<uint32_t>(lane == 0 ? b.r1 : b.k1);
            const uintptr_t lo = base + static_cast<uintptr_t>(e_lo) * sz;
            const uintptr_t hi = base + static_cast<uintptr_t>(e_hi) * sz;
            const uintptr_t a0 = lo & ~static_cast<uintptr_t>(15);
            const uint32_t bytes = static_cast<uint32_t>(((hi + 15) & ~static_cast<uintptr_t>(15)) - a0);
            const uint32_t b1 = __shfl_up_sync(kSliceMask, bytes, 1);
            const uint32_t b2 = NSL > 2 ? __shfl_up_sync(kSliceMask, bytes, 2) : 0u;
            const uint32_t off = (lane >= 1 ? b1 : 0u) + (lane >= 2 ? b2 : 0u);
            const uint32_t first = off + static_cast<uint32_t>(lo & 15);
            const uint32_t total = __shfl_sync(kSliceMask, off + bytes, NSL - 1);
            const uint32_t f1 = __shfl_sync(kSliceMask, first, 1);
            const uint32_t f2 = NSL > 2 ? __shfl_sync(kSliceMask, first, 2) : 0u;
            if (lane == 0) {
                hdr->r0 = b.r0;
                hdr->r1 = b.r1;
                hdr->k0 = b.k0;
                hdr->k1 = b.k1;
                hdr->m0 = b.m0;
                hdr->m1 = b.m1;
                hdr->re_first = first;
                hdr->idx_first = f1;
                hdr->val_first = f2;
                hdr->ok = 1;
                mbar_arrive_expect_tx(bar, total);
            }
            __syncwarp(kSliceMask);  // the transaction count is armed before any copy lands
            if (bytes) bulk_g2s(stage + off, reinterpret_cast<const void *>(a0), bytes, bar, pol);
        }
        return;
    }
    // Edge tile: general placement; the ragged ends (at most 7 elements per end and slice)
    // move with plain loads by the producer lanes before the barrier is armed.
    Seg t[3];
    t[0] = make_seg(a.row_end, b.r0, b.r1, a.num_rows, 4, 0);
    t[1] = make_seg(a.idx, b.k0, b.k1, a.num_atoms, 4, t[0].next);
    if (NSL > 2) {
        t[2] = make_seg(a.val, b.k0, b.k1, a.num_atoms, SV, t[1].next);
    } else {
        t[2] = t[1];  // no value slice: nothing moves for it
        t[2].first = 0;
        t[2].bulk_bytes = 0;
        t[2].head = 0;
        t[2].tail = 0;
        t[2].count = 0;
    }
    for (int q = lane; q < 16 * NSL; q += 32) {
        const int which = q >> 4;
        const bool tail = ((q >> 3) & 1) != 0;
        const uint32_t e = q & 7;
        // Fields picked by value (a dynamic index into t[] would put it in local memory).
        const uint32_t g_first = which == 0 ? t[0].first : (which == 1 ? t[1].first : t[2].first);
        const uint32_t g_head = which == 0 ? t[0].head : (which == 1 ? t[1].head : t[2].head);
        const uint32_t g_tail = which == 0 ? t[0].tail : (which == 1 ? t[1].tail : t[2].tail);
        const uint32_t g_count = which == 0 ? t[0].count : (which == 1 ? t[1].count : t[2].count);
        const uint32_t sz = which == 2 ? SV : 4u;
        const uint32_t rel = tail ? g_tail + e : e;
        const bool ok = tail ? (rel < g_count) : (e < g_head);
        if (!ok) continue;
        const char *src = which == 0 ? reinterpret_cast<const char *>(a.row_end + b.r0)
                                     : (which == 1 ? reinterpret_cast<const char *>(a.idx + b.k0)
                                                   : static_cast<const char *>(a.val) + static_cast<size_t>(b.k0) * sz);
        src += static_cast<size_t>(rel) * sz;
        unsigned char *dst = stage + g_first + rel * sz;
        if (sz == 4)
            *reinterpret_cast<int *>(dst) = __ldg(reinterpret_cast<const int *>(src));
        else
            *reinterpret_cast<unsigned short *>(dst) = __ldg(reinterpret_cast<const unsigned short *>(src));
    }
    __syncwarp();
    if (lane == 0) {
        hdr->r0 = b.r0;
        hdr->r1 = b.r1;
        hdr->k0 = b.k0;
        hdr->k1 = b.k1;
        hdr->m0 = b.m0;
        hdr->m1 = b.m1;
        hdr->re_first = t[0].first;
        hdr->idx_first = t[1].first;
        hdr->val_first = t[2].first;
        hdr->ok = 1;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, t[0].bulk_bytes + t[1].bulk_bytes + t[2].bulk_bytes);
#pragma unroll
        for (int w = 0; w < NSL; ++w)
            if (t[w].bulk_bytes)
                bulk_g2s(stage + t[w].bulk_off, reinterpret_cast<const void *>(t[w].bulk_src), t[w].bulk_bytes, bar,
                         pol);
    }
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

// A 16-bit value's bits widened to FP32 (BF16: shift into the high half; FP16: convert).
template <typename V>
__device__ __forceinline__ float half_bits_to_f32(unsigned short bits) {
    if constexpr (std::is_same<V, __nv_bfloat16>::value)
        return __uint_as_float(static_cast<uint32_t>(bits) << 16);
    else
        return __half2float(__ushort_as_half(bits));
}

// Blocked tile layout.  Slot s of a tile is element (16-byte-aligned start) + s of its index
// slice in shared memory; the tile's first nonzero sits at slot `lead` (0..7).  Gather thread
// g owns slots [g*IPT, (g+1)*IPT).  Slots outside [lead, lead + nk) are padding with product 0.
__device__ __forceinline__ int tile_lead(const StageHdr &h) { return static_cast<int>(h.idx_first & 15u) >> 2; }

// Gather thread g's slots of one tile: values in vv, gathers x[col] issued into xv (indices and
// values by vector shared loads; the products are formed after other work by the caller).
template <typename V, int IPT, int MODE>
__device__ __forceinline__ void gather_issue(const MergeArgs &a, const unsigned char *stage, const StageHdr &h, int g,
                                             float (&vv)[IPT], float (&xv)[IPT]) {
    const int nk = h.k1 - h.k0;
    const int lead = tile_lead(h);
    const int slot0 = g * IPT;
    const int item0 = slot0 - lead;  // tile item of this thread's first slot
    int col[IPT];
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        col[q] = 0;
        vv[q] = 0.f;
        xv[q] = 0.f;
    }
    if (item0 + IPT <= 0 || item0 >= nk) return;  // nothing of the tile in this thread's slots
    const unsigned char *idx0 = stage + h.idx_first - lead * 4;  // slot 0, 16-byte aligned
#pragma unroll
    for (int q = 0; q < IPT; q += 4) {
        const int4 c = *reinterpret_cast<const int4 *>(idx0 + (slot0 + q) * 4);
        col[q] = c.x;
        col[q + 1] = c.y;
        col[q + 2] = c.z;
        col[q + 3] = c.w;
    }
    constexpr uint32_t SV = MergeTraits<V, MODE>::SV;
    const unsigned char *val_item0 = stage + h.val_first;  // tile item 0
    const uintptr_t vslot0 = reinterpret_cast<uintptr_t>(val_item0) - static_cast<uintptr_t>(lead) * SV;
    if (SV == 0) {  // gather-sum: the gathered value is the product
#pragma unroll
        for (int q = 0; q < IPT; ++q)
            if (item0 + q >= 0 && item0 + q < nk) vv[q] = 1.f;
    } else if (SV == 4) {
        int raw[IPT];
        if ((vslot0 & 15u) == 0) {
#pragma unroll
            for (int q = 0; q < IPT; q += 4) {
                const int4 t = *reinterpret_cast<const int4 *>(vslot0 + static_cast<uintptr_t>(slot0 + q) * 4);
                raw[q] = t.x;
                raw[q + 1] = t.y;
                raw[q + 2] = t.z;
                raw[q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const int it = item0 + q;
                raw[q] = (it >= 0 && it < nk) ? reinterpret_cast<const int *>(val_item0)[it] : 0;
            }
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int it = item0 + q;
            if (it >= 0 && it < nk) vv[q] = __int_as_float(raw[q]);
        }
    } else {
        unsigned short raw[IPT];
        if ((vslot0 & 15u) == 0 && IPT % 8 == 0) {
#pragma unroll
            for (int q = 0; q < IPT; q += 8) {
                const uint4 t = *reinterpret_cast<const uint4 *>(vslot0 + static_cast<uintptr_t>(slot0 + q) * 2);
                const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    raw[q + 2 * e] = static_cast<unsigned short>(w[e] & 0xffffu);
                    raw[q + 2 * e + 1] = static_cast<unsigned short>(w[e] >> 16);
                }
            }
        } else if ((vslot0 & 7u) == 0) {
#pragma unroll
            for (int q = 0; q < IPT; q += 4) {
                const uint2 t = *reinterpret_cast<const uint2 *>(vslot0 + static_cast<uintptr_t>(slot0 + q) * 2);
                raw[q] = static_cast<unsigned short>(t.x & 0xffffu);
                raw[q + 1] = static_cast<unsigned short>(t.x >> 16);
                raw[q + 2] = static_cast<unsigned short>(t.y & 0xffffu);
                raw[q + 3] = static_cast<unsigned short>(t.y >> 16);
            }
        } else {
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const int it = item0 + q;
                raw[q] = (it >= 0 && it < nk) ? reinterpret_cast<const unsigned short *>(val_item0)[it] : 0;
            }
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int it = item0 + q;
            if (it >= 0 && it < nk) vv[q] = half_bits_to_f32<V>(raw[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int it = item0 + q;
        if (it >= 0 && it < nk) {
            int c = col[q];
            if (MODE == kBatched) c += batched_col_base(a, h.m0, h.m1, h.k0 + it);
            xv[q] = __ldg(a.x + c);
        }
    }
}

// The forward product's saved gathers, xg[k] = x[col_idx[k]], written coalesced.  A warp's
// gathered values first replace its own staged column indices: its slots holding the tile's
// nonzeros ([lead, lead + nk), the staged indices themselves), which nothing reads any more.
// The warp then reads them back lane by lane, so each store instruction writes 32 consecutive
// nonzeros (streaming stores).  Runs before the warp releases the stage.
template <int IPT>
__device__ __forceinline__ void save_gathered(float *xg, unsigned char *stage, const StageHdr &h, int g, int gwarp,
                                              const float (&xv)[IPT]) {
    const int lane = threadIdx.x & 31;
    const int nk = h.k1 - h.k0, lead = tile_lead(h);
    float *slots = reinterpret_cast<float *>(stage + h.idx_first - lead * 4);  // slot 0, 16-byte aligned
    const int slot0 = g * IPT;
    if (slot0 >= lead && slot0 + IPT <= lead + nk) {
#pragma unroll
        for (int q = 0; q < IPT; q += 4)
            *reinterpret_cast<float4 *>(slots + slot0 + q) = make_float4(xv[q], xv[q + 1], xv[q + 2], xv[q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < IPT; ++q)
            if (slot0 + q >= lead && slot0 + q < lead + nk) slots[slot0 + q] = xv[q];
    }
    __syncwarp();
    const int S0 = gwarp * 32 * IPT;
    float *dst = xg + h.k0 - lead;  // slot s holds nonzero k0 - lead + s
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int sl = S0 + q * 32 + lane;
        if (sl >= lead && sl < lead + nk) __stcs(dst + sl, slots[sl]);
    }
}

// Row-start bits of one gather warp's 32 * IPT slots of a tile, built by the warp alone from
// the staged row ends (row r0 + r + 1 starts at slot s_re[r] - k0 + lead; slots are
// non-decreasing in r): a 32-way lower-bound search for the first row start in the warp's
// slots, then the row starts in range OR-ed into the warp's private bit words.  Returns this
// lane's IPT bits and leaves the words cleared.
template <int IPT>
__device__ __forceinline__ uint32_t warp_row_start_flags(const unsigned char *stage, const StageHdr &h, int gwarp,
                                                         uint32_t *wbits) {
    const int lane = threadIdx.x & 31;
    const int S0 = gwarp * 32 * IPT;
    const int nr = h.r1 - h.r0, nk = h.k1 - h.k0, lead = tile_lead(h);
    const int *s_re = reinterpret_cast<const int *>(stage + h.re_first);
    const int lo_slot = S0 > lead + 1 ? S0 : lead + 1;        // item 0 starts no segment
    const int hi_slot = (S0 + 32 * IPT) < (nk + lead) ? (S0 + 32 * IPT) : (nk + lead);  // exclusive
    auto slot_of = [&](int r) { return s_re[r] - h.k0 + lead; };
    int lo = 0, hi = nr;  // first r with slot_of(r) >= lo_slot lies in [lo, hi]
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) >> 5;
        const int q = lo + lane * step;
        const int cnt = __popc(__ballot_sync(0xffffffffu, q < hi && slot_of(q) < lo_slot));
        const int nlo = cnt > 0 ? lo + (cnt - 1) * step + 1 : lo;
        const int nhi = lo + cnt * step < hi ? lo + cnt * step : hi;
        lo = nlo;
        hi = nhi;
    }
    {
        const int q = lo + lane;
        lo += __popc(__ballot_sync(0xffffffffu, q < hi && slot_of(q) < lo_slot));
    }
    if (lo_slot < hi_slot) {
        for (int rb = lo;; rb += 32) {
            const int r = rb + lane;
            const int sl = r < nr ? slot_of(r) : 0x40000000;
            const bool in = sl < hi_slot;
            if (in) atomicOr(&wbits[(sl - S0) >> 5], 1u << ((sl - S0) & 31));
            if (!__shfl_sync(0xffffffffu, static_cast<int>(in), 31)) break;
        }
    }
    __syncwarp();
    const uint32_t mine = (IPT == 8) ? static_cast<uint32_t>(reinterpret_cast<const unsigned char *>(wbits)[lane])
                                     : static_cast<uint32_t>(reinterpret_cast<const unsigned short *>(wbits)[lane]);
    __syncwarp();
    if (lane < IPT) wbits[lane] = 0u;
    __syncwarp();
    return mine;
}

// Named barriers: id 1 over the scan warps, id 2 over the gather warps.
template <int ID, int NTHREADS>
__device__ __forceinline__ void group_bar() {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NTHREADS) : "memory");
}

// The same barrier with an OR vote, so a group takes the same branch.
template <int ID, int NTHREADS>
__device__ __forceinline__ bool group_bar_any(bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(pred)), "n"(ID), "n"(NTHREADS)
        : "memory");
    return r != 0;
}

template <typename V, int GW, int IPT, int MODE>
__global__ void __launch_bounds__(MergeShape<GW, IPT, static_cast<int>(MergeTraits<V, MODE>::SV), MergeTraits<V, MODE>::NS, MergeTraits<V, MODE>::NB, MergeTraits<V, MODE>::RB>::THREADS,
                                  MergeShape<GW, IPT, static_cast<int>(MergeTraits<V, MODE>::SV), MergeTraits<V, MODE>::NS, MergeTraits<V, MODE>::NB, MergeTraits<V, MODE>::RB>::MIN_BLOCKS)
    merge_spmv_kernel(const MergeArgs a) {
    using Sh = MergeShape<GW, IPT, static_cast<int>(MergeTraits<V, MODE>::SV), MergeTraits<V, MODE>::NS, MergeTraits<V, MODE>::NB, MergeTraits<V, MODE>::RB>;
    constexpr int NS = Sh::NSTAGE;
    constexpr int NB = Sh::NBUF;
    static_assert(NB >= 1 && NB <= 2, "one or two product buffers");
    static_assert(NS <= static_cast<int>(sizeof(Bars::full) / sizeof(uint64_t)), "one barrier set per stage");
    constexpr int GT = Sh::GT;
    extern __shared__ __align__(128) unsigned char smem[];
    Bars *bars = reinterpret_cast<Bars *>(smem);
    StageHdr *hdrs = reinterpret_cast<StageHdr *>(smem + 256);
    unsigned char *stages = smem + Sh::HDR;
    uint32_t *wbits_all = reinterpret_cast<uint32_t *>(stages + NS * Sh::STAGE);  // per gather warp
    unsigned char *bufmem = stages + NS * Sh::STAGE + Sh::BITS;
    auto buf = [&](int b) {
        unsigned char *p = bufmem + b * Sh::BUF;
        ProdBuf<GT> pb;
        pb.val = reinterpret_cast<float *>(p);
        pb.agg = pb.val + Sh::P_FLOATS;
        pb.ff = reinterpret_cast<int *>(pb.agg + GT);
        pb.cin = reinterpret_cast<float *>(pb.ff + GT);
        return pb;
    };

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int G = a.num_tiles;
    if (static_cast<int>(blockIdx.x) >= G) return;
    const int n_my = (G - static_cast<int>(blockIdx.x) + static_cast<int>(gridDim.x) - 1) / static_cast<int>(gridDim.x);
    auto tile_of = [&](int i) { return static_cast<int>(blockIdx.x) + i * static_cast<int>(gridDim.x); };

    if (tid == 0) {
        for (int q = 0; q < NS; ++q) {
            mbar_init(&bars->full[q], 1);
            mbar_init(&bars->gdone[q], GW);
            mbar_init(&bars->sdone[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&bars->pready[q], GW);
            mbar_init(&bars->pfree[q], 1);
        }
        mbar_fence_init();
    }
    for (int w = tid; w < static_cast<int>(Sh::BITS / 4); w += Sh::THREADS) wbits_all[w] = 0u;
    __syncthreads();

    if (warp < GW) {
        // ---------------------------------------------------------------- gather warps
        // Per tile: products of this thread's IPT slots, the scan of those slots restarting at
        // row starts, and the thread's aggregate for the scan warps.  No barrier: each warp
        // runs at its own pace.
        const int g = tid;
        for (int i = 0; i < n_my; ++i) {
            const int s = i % NS, b = i % NB;
            bool ok = mbar_wait_bounded(&bars->full[s], (i / NS) & 1, kWaitLimitNs);
            if (ok && i >= NB) ok = mbar_wait_bounded(&bars->pfree[b], ((i - NB) / NB) & 1, kWaitLimitNs);
            if (!__all_sync(0xffffffffu, ok)) {  // the whole warp leaves together
                if (lane == 0) atomicExch(a.err, static_cast<int>(LB_ERR_TIMEOUT));
                return;
            }
            const StageHdr h = hdrs[s];
            const ProdBuf<GT> pb = buf(b);
            float vv[IPT], xv[IPT];
            uint32_t flags = 0;
            if (h.ok) {
                // Gathers first; the row-start bits are found while they are in flight.
                gather_issue<V, IPT, MODE>(a, stages + s * Sh::STAGE, h, g, vv, xv);
                flags = warp_row_start_flags<IPT>(stages + s * Sh::STAGE, h, warp, wbits_all + warp * IPT);
            } else {
#pragma unroll
                for (int q = 0; q < IPT; ++q) vv[q] = xv[q] = 0.f;
            }
            __syncwarp();
            // The stage is no longer read here, unless the gathers are saved through it.
            const bool save = MODE == kPlain && a.xg != nullptr && h.ok;
            if (!save && lane == 0) mbar_arrive(&bars->gdone[s]);
            float v[IPT];
#pragma unroll
            for (int q = 0; q < IPT; ++q) v[q] = vv[q] * xv[q];
            if (save) {
                save_gathered<IPT>(a.xg, stages + s * Sh::STAGE, h, g, warp, xv);
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars->gdone[s]);
            }
#pragma unroll
            for (int q = 1; q < IPT; ++q)
                if (!((flags >> q) & 1u)) v[q] += v[q - 1];
#pragma unroll
            for (int q = 0; q < IPT; q += 4)
                *reinterpret_cast<float4 *>(pb.val + ppad(g * IPT + q)) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            pb.agg[g] = v[IPT - 1];
            pb.ff[g] = flags ? __ffs(flags) - 1 : IPT;
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars->pready[b]);
        }
    } else if (warp < GW + Sh::SW) {
        // ---------------------------------------------------------------- scan warps
        // Per tile: the first scan warp scans the gather threads' aggregates (the carry into
        // each thread's first segment); then every scan warp reads rows' sums at their last
        // nonzero, and the last thread writes the tile's carry.
        constexpr int ST = Sh::ST;
        constexpr int PER = GT / 32;  // aggregates per lane of the first scan warp
        static_assert(PER % 4 == 0, "aggregates are read four at a time");
        const int st = tid - GT;
        for (int i = 0; i < n_my; ++i) {
            const int s = i % NS, b = i % NB;
            bool ok = mbar_wait_bounded(&bars->pready[b], (i / NB) & 1, kWaitLimitNs);
            if (ok) ok = mbar_wait_bounded(&bars->full[s], (i / NS) & 1, kWaitLimitNs);
            const ProdBuf<GT> pb = buf(b);
            if (ok && st < 32) {
                int fl[PER];
                float ag[PER];
#pragma unroll
                for (int q = 0; q < PER; q += 4) {
                    const int4 f4 = *reinterpret_cast<const int4 *>(pb.ff + st * PER + q);
                    const float4 a4 = *reinterpret_cast<const float4 *>(pb.agg + st * PER + q);
                    fl[q] = f4.x < IPT;
                    fl[q + 1] = f4.y < IPT;
                    fl[q + 2] = f4.z < IPT;
                    fl[q + 3] = f4.w < IPT;
                    ag[q] = a4.x;
                    ag[q + 1] = a4.y;
                    ag[q + 2] = a4.z;
                    ag[q + 3] = a4.w;
                }
                int fi = fl[0];
                float vi = ag[0];
#pragma unroll
                for (int q = 1; q < PER; ++q) {
                    vi = fl[q] ? ag[q] : vi + ag[q];
                    fi |= fl[q];
                }
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float vu = __shfl_up_sync(0xffffffffu, vi, off);
                    const int fu = __shfl_up_sync(0xffffffffu, fi, off);
                    if (lane >= off) {
                        if (!fi) vi = vu + vi;
                        fi |= fu;
                    }
                }
                float ve = __shfl_up_sync(0xffffffffu, vi, 1);
                int fe = __shfl_up_sync(0xffffffffu, fi, 1);
                if (lane == 0) {
                    ve = 0.f;
                    fe = 0;
                }
                float c = ve;  // carry into gather thread st*PER (a single warp: no earlier warps)
                float cin[PER];
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    cin[q] = c;
                    c = fl[q] ? ag[q] : c + ag[q];
                }
#pragma unroll
                for (int q = 0; q < PER; q += 4)
                    *reinterpret_cast<float4 *>(pb.cin + st * PER + q) = make_float4(cin[q], cin[q + 1], cin[q + 2], cin[q + 3]);
            }
            if (group_bar_any<1, ST>(!ok)) {  // the scan warps leave together
                if (st == 0) atomicExch(a.err, static_cast<int>(LB_ERR_TIMEOUT));
                return;
            }
            const StageHdr h = hdrs[s];
            const int tile = tile_of(i);
            if (!h.ok) {
                if (st == 0) {
                    atomicExch(a.err, static_cast<int>(LB_ERR_BAD_MATRIX));
                    a.carry_row[tile] = a.num_rows;  // the fixup skips it
                    a.carry_val[tile] = 0.f;
                }
            } else {
                const int nr = h.r1 - h.r0;
                const int nk = h.k1 - h.k0;
                const int k0 = h.k0;
                const int lead = tile_lead(h);
                const int *s_re = reinterpret_cast<const int *>(stages + s * Sh::STAGE + h.re_first);
                // Scan value at slot e: the owner's own inclusive value, plus the carry into the
                // owner when e lies before the owner's first segment start.
                auto value_at = [&](int e) {
                    const int owner = e / IPT;
                    const float v = pb.val[ppad(e)];
                    return (e - owner * IPT) < pb.ff[owner] ? pb.cin[owner] + v : v;
                };
                for (int r = st; r < nr; r += ST) {
                    const int end = s_re[r] - k0;
                    const int start = r > 0 ? s_re[r - 1] - k0 : 0;
                    a.y[h.r0 + r] = end > start ? value_at(end - 1 + lead) : 0.f;
                }
                if (st == ST - 1) {
                    const int open_start = nr > 0 ? s_re[nr - 1] - k0 : 0;
                    a.carry_row[tile] = h.r1;
                    a.carry_val[tile] = nk > open_start ? value_at(nk - 1 + lead) : 0.f;
                }
            }
            group_bar<1, ST>();  // buffer and stage are free
            if (st == 0) {
                mbar_arrive(&bars->pfree[b]);
                mbar_arrive(&bars->sdone[s]);
            }
        }
    } else {
        // ---------------------------------------------------------------- producer warp
        const uint64_t pol = policy_evict_first();
        TileBounds nb = load_bounds<MODE>(a, tile_of(0));
        for (int j = 0; j < n_my; ++j) {
            const int s = j % NS;
            const TileBounds cur = nb;
            if (j + 1 < n_my) nb = load_bounds<MODE>(a, tile_of(j + 1));
            if (j >= NS) {
                const uint32_t par = ((j - NS) / NS) & 1;
                bool ok = mbar_wait_bounded(&bars->gdone[s], par, kWaitLimitNs);
                if (ok) ok = mbar_wait_bounded(&bars->sdone[s], par, kWaitLimitNs);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) atomicExch(a.err, static_cast<int>(LB_ERR_TIMEOUT));
                    return;
                }
            }
            produce_tile<V, MODE, Sh::TILE_ITEMS>(a, &bars->full[s], &hdrs[s], stages + s * Sh::STAGE, cur, pol);
        }
    }
}

// Resident CTAs per SM of one kernel instance on the current device (computed once per
// device; also raises the kernel's dynamic shared-memory limit).
template <typename V, int GW, int IPT, int MODE>
int merge_blocks_per_sm() {
    using Sh = MergeShape<GW, IPT, static_cast<int>(MergeTraits<V, MODE>::SV), MergeTraits<V, MODE>::NS, MergeTraits<V, MODE>::NB, MergeTraits<V, MODE>::RB>;
    constexpr int kMaxDev = 64;
    static int cache[kMaxDev] = {0};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 0;
    if (cache[dev] > 0) return cache[dev];
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        auto kern = merge_spmv_kernel<V, GW, IPT, MODE>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(Sh::SMEM)) !=
            cudaSuccess)
            return 0;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, Sh::THREADS, Sh::SMEM) != cudaSuccess) return 0;
        nb = nb > 0 ? nb : 1;
        // Ask for no more shared memory than the resident CTAs use: the rest of the SM's
        // unified L1/shared memory stays L1, which holds the random gathers in flight (their
        // rate falls steeply as the L1 share shrinks).
        int max_smem = 0;
        if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            max_smem <= 0)
            return 0;
        const long long need = static_cast<long long>(nb) * (Sh::SMEM + 1024);
        int pct = static_cast<int>((need * 100 + max_smem - 1) / max_smem);
        if (pct > 100) pct = 100;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess) return 0;
        cache[dev] = nb;
    }
    return cache[dev];
}

template <typename V, int GW, int IPT, int MODE>
cudaError_t launch_merge_cfg(const MergeArgs &a, cudaStream_t st, cudaEvent_t eb, cudaEvent_t ea) {
    using Sh = MergeShape<GW, IPT, static_cast<int>(MergeTraits<V, MODE>::SV), MergeTraits<V, MODE>::NS, MergeTraits<V, MODE>::NB, MergeTraits<V, MODE>::RB>;
    const int per_sm = merge_blocks_per_sm<V, GW, IPT, MODE>();
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const long long wave = static_cast<long long>(per_sm) * current_sm_count();
    const int grid = static_cast<int>(a.num_tiles < wave ? a.num_tiles : wave);
    if (eb) cudaEventRecord(eb, st);
    merge_spmv_kernel<V, GW, IPT, MODE><<<grid, Sh::THREADS, Sh::SMEM, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (ea) cudaEventRecord(ea, st);
    if (e != cudaSuccess) return e;
    return launch_fixup(a.num_tiles, a.num_rows, a.carry_row, a.carry_val, a.y, st);
}

// The (gather threads, items per thread) shapes compiled into the library.
#define LB_MERGE_SHAPES(X) X(128, 16) X(256, 8) X(256, 16) X(384, 8) X(512, 8)

template <typename V, int MODE>
cudaError_t dispatch_merge_shape(int threads, int ipt, const MergeArgs &a, cudaStream_t st, cudaEvent_t eb,
                                 cudaEvent_t ea) {
#define LB_TRY_SHAPE(TH, IP) \
    if (threads == TH && ipt == IP) return launch_merge_cfg<V, TH / 32, IP, MODE>(a, st, eb, ea);
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
        case kGatherSum:
            // The gathered values are FP32 whatever the matrix's value type: one instance.
            if constexpr (std::is_same<V, float>::value)
                return dispatch_merge_shape<V, kGatherSum>(threads, ipt, a, st, eb, ea);
            else
                return cudaErrorInvalidValue;
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace lb
