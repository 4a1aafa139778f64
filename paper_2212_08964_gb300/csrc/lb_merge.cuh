// lb_merge.cuh -- warp-tiled merge-path SpMV (work-oriented schedule) for sm_103a.
//
// The schedule is the dissertation's work-oriented merge path (Ch.3 Sec. "Work-Oriented",
// Alg. alg:work-oriented; Ch.4 Sec. "Merge-path load balancing"): rows and nonzeros count
// as one work item each, the (rows + nnz) items are cut into tiles of equal size, and a
// split of the merge of row ends with nonzero indices gives every tile its starting row and
// nonzero.  Rows completed inside a tile are written directly; the row left open at the end
// of a tile goes out as a carry and is added by the fixup pass ("Fix-up" procedure of the
// same algorithm).  The tile-level split is computed once by the partition kernel.
//
// Tiles are sized for one warp: 32 lanes x IPT slots, at most 32 * IPT - 8 work items.  The
// paper splits a tile again by a merge-path search per thread and walks row ends and
// nonzeros one by one; here a warp computes the same row sums with a segmented scan over the
// tile's nonzeros: lane l owns IPT consecutive nonzero slots, a row start sets a flag at its
// first slot, each lane scans its own products restarting at flags, a shuffle scan of the 32
// lane totals gives every lane the carry into its first row, and each row's sum is read at
// its last nonzero.  No atomics touch y and the summation order is fixed, so results are
// deterministic.
//
// GB300 realisation.  Random 4-byte gathers of x are the limiting resource: every gather is
// its own 32-byte sector request from L1 to L2, and the L1 holds the requests in flight, so
// the gather rate falls with every kilobyte that shared memory takes from the SM's unified
// 256 KB array.  The kernel therefore uses no staging buffers and no block-wide barriers:
//   * every warp is independent and persistent (tiles w, w + W, w + 2W, ... of the W warps
//     of one wave), and keeps only its tile's scanned slot values and row-start flags in
//     shared memory (1.4 KB per warp at IPT = 8), so L1 keeps about 200 KB of the array;
//   * indices and values stream with 256-bit loads (one full 32-byte sector per lane and
//     instruction, L1 bypassed, L2 evict-first so that x stays resident);
//   * the next tile's indices are loaded while this tile's gathers are in flight, so the
//     gathers of consecutive tiles follow each other without waiting for the index stream;
//   * y is written with consecutive rows on consecutive lanes (coalesced).
// There is no wait on any flag or barrier, so no kernel here can hang on a lost signal.
// Persistent warps take tiles in a fixed order, so the partition and the summation order do
// not depend on the SM count.
#pragma once

#include <mutex>
#include <type_traits>

#include "lb_warp.cuh"

namespace lb {

// A tile's bounds: rows [r0, r1) end inside it, nonzeros [k0, k1) lie in it; batched tiles
// also carry the matrices m0 <= m1 of their first nonzero and of the next tile's first one.
struct WBounds {
    int r0, r1, k0, k1, m0, m1;
};

// Lanes 0..3 (5 when batched) each load one word of tile t's bounds; the others load nothing.
template <int MODE>
__device__ __forceinline__ int bounds_word(const MergeArgs &a, int t, int lane) {
    int v = 0;
    if (lane < 2)
        v = __ldg(a.tile_row + t + lane);
    else if (lane < 4)
        v = __ldg(a.tile_nz + t + lane - 2);
    else if (MODE == kBatched && lane < 6)
        v = __ldg(a.tile_mat + t + lane - 4);
    return v;
}

template <int MODE>
__device__ __forceinline__ WBounds bounds_bcast(int w) {
    WBounds b;
    b.r0 = __shfl_sync(0xffffffffu, w, 0);
    b.r1 = __shfl_sync(0xffffffffu, w, 1);
    b.k0 = __shfl_sync(0xffffffffu, w, 2);
    b.k1 = __shfl_sync(0xffffffffu, w, 3);
    if (MODE == kBatched) {
        b.m0 = __shfl_sync(0xffffffffu, w, 4);
        b.m1 = __shfl_sync(0xffffffffu, w, 5);
    } else {
        b.m0 = b.m1 = 0;
    }
    return b;
}

// A tile from a valid partition of valid offsets always passes; anything else (offsets that
// are not a CSR prefix sum) is skipped with LB_ERR_BAD_MATRIX instead of reading out of bounds.
template <int IPT>
__device__ __forceinline__ bool wtile_ok(const MergeArgs &a, const WBounds &b) {
    return b.r0 >= 0 && b.r0 <= b.r1 && b.r1 <= a.num_rows && b.k0 >= 0 && b.k0 <= b.k1 && b.k1 <= a.num_atoms &&
           (b.r1 - b.r0) + (b.k1 - b.k0) <= WarpTile<IPT>::ITEMS;
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

// This lane's gather indices for one tile.  Batched: a tile inside one matrix returns that
// matrix's column base in cb, added only when the gathers are issued (adding it here would
// wait for the index load at once, instead of while the current tile is worked on); a tile
// spanning matrices adds each slot's base to its index and returns cb = 0.  Lanes whose slots
// all lie outside the tile load nothing; slots outside the tile may hold neighbouring indices,
// which are never gathered.
template <int IPT, int MODE>
__device__ __forceinline__ void load_idx(const MergeArgs &a, const WBounds &b, bool ok, int iph, int lane,
                                         uint64_t pol, int (&col)[IPT], int &cb) {
#pragma unroll
    for (int q = 0; q < IPT; ++q) col[q] = 0;
    cb = 0;
    if (!ok) return;
    const int lead = (iph + b.k0) & 7;
    const int e0 = b.k0 - lead + IPT * lane;
    if (e0 >= b.k1 || e0 + IPT <= b.k0) return;
    if (e0 >= 0 && e0 + IPT <= a.num_atoms) {
#pragma unroll
        for (int h = 0; h < IPT; h += 8) {
            uint32_t r[8];
            ld_stream8(a.idx + e0 + h, pol, r);
#pragma unroll
            for (int q = 0; q < 8; ++q) col[h + q] = static_cast<int>(r[q]);
        }
    } else {  // the array's first or last 32 bytes: element by element
#pragma unroll
        for (int q = 0; q < IPT; ++q)
            if (e0 + q >= b.k0 && e0 + q < b.k1) col[q] = __ldg(a.idx + e0 + q);
    }
    if (MODE == kBatched) {
        if (b.m0 == b.m1) {
            cb = __ldg(a.mat_col_base + b.m0);
        } else {
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                if (e0 + q >= b.k0 && e0 + q < b.k1) col[q] += batched_col_base(a, b.m0, b.m1, e0 + q);
        }
    }
}

// This lane's values (1 for the gather-sum product, whose gathered entries are the terms).
template <typename V, int IPT, int MODE>
__device__ __forceinline__ void load_vals(const MergeArgs &a, int e0, uint32_t vm, uint64_t pol, float (&vv)[IPT]) {
#pragma unroll
    for (int q = 0; q < IPT; ++q) vv[q] = 0.f;
    if (MODE == kGatherSum) {
#pragma unroll
        for (int q = 0; q < IPT; ++q) vv[q] = 1.f;
        return;
    }
    if (vm == 0) return;
    const bool vec = a.vec_vals && e0 >= 0 && e0 + IPT <= a.num_atoms;
    if (sizeof(V) == 4) {
        const float *v = static_cast<const float *>(a.val);
        if (vec) {
#pragma unroll
            for (int h = 0; h < IPT; h += 8) {
                uint32_t r[8];
                ld_stream8(v + e0 + h, pol, r);
#pragma unroll
                for (int q = 0; q < 8; ++q) vv[h + q] = __uint_as_float(r[q]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                if ((vm >> q) & 1u) vv[q] = __ldg(v + e0 + q);
        }
    } else {
        const unsigned short *v = static_cast<const unsigned short *>(a.val);
        if (vec) {
#pragma unroll
            for (int h = 0; h < IPT; h += 8) {
                uint32_t r[4];
                ld_stream4(v + e0 + h, pol, r);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    vv[h + 2 * q] = half_bits_to_f32<V>(r[q] & 0xffffu);
                    vv[h + 2 * q + 1] = half_bits_to_f32<V>(r[q] >> 16);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                if ((vm >> q) & 1u) vv[q] = half_bits_to_f32<V>(__ldg(v + e0 + q));
        }
    }
}

// Row-start flags of one tile, packed into this lane's IPT bits (bit q: a row starts at the
// lane's slot q), and the row end of the tile's last complete row (k0 if none).  Row r + 1
// starts at nonzero row_end[r]; the flag is set only strictly inside the tile, where a
// segment of the scan restarts.  e_first returns this lane's row end of the first 32 rows.
// The lane's flag bytes are cleared again after reading.
template <int IPT>
__device__ __forceinline__ uint32_t row_start_flags(const MergeArgs &a, const WBounds &b, int kb, int lane,
                                                    unsigned char *flg, int &e_first, int &e_last) {
    const int nr = b.r1 - b.r0;
    e_first = 0;
    e_last = b.k0;
    // One chunk of 32 row ends; row-heavy tiles (up to 248 rows) take four chunks per step,
    // their loads issued together: one latency instead of one per chunk.
    auto chunk = [&](int j, int e) {
        if (j == 0) e_first = e;
        if (j + lane < nr && e > b.k0 && e < b.k1) flg[e - kb] = 1;
        const int src = nr - 1 - j < 31 ? nr - 1 - j : 31;
        const int el = __shfl_sync(0xffffffffu, e, src);
        if (j + 32 >= nr) e_last = el;
    };
    if (nr <= 32) {
        if (nr > 0) chunk(0, lane < nr ? __ldg(a.row_end + b.r0 + lane) : 0);
    } else {
        for (int j0 = 0; j0 < nr; j0 += 128) {
            int ec[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + 32 * u;
                ec[u] = j + lane < nr ? __ldg(a.row_end + b.r0 + j + lane) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + 32 * u < nr) chunk(j0 + 32 * u, ec[u]);  // warp-uniform
        }
    }
    __syncwarp();
    uint32_t f;
    if (IPT == 8) {
        uint2 *p = reinterpret_cast<uint2 *>(flg + 8 * lane);
        const uint2 w = *p;
        *p = make_uint2(0u, 0u);
        // Flag bytes are 0 or 1: multiplying by 0x00204081 lines byte i up at bit 21 + i with
        // no two partial products sharing a bit.
        f = ((w.x * 0x00204081u) >> 21 & 0xfu) | (((w.y * 0x00204081u) >> 21 & 0xfu) << 4);
    } else {
        uint4 *p = reinterpret_cast<uint4 *>(flg + 16 * lane);
        const uint4 w = *p;
        *p = make_uint4(0u, 0u, 0u, 0u);
        f = ((w.x * 0x00204081u) >> 21 & 0xfu) | (((w.y * 0x00204081u) >> 21 & 0xfu) << 4) |
            (((w.z * 0x00204081u) >> 21 & 0xfu) << 8) | (((w.w * 0x00204081u) >> 21 & 0xfu) << 12);
    }
    return f;
}

// Launch bounds: at IPT = 8, 64 registers per thread keep 32 warps per SM resident.
template <int IPT>
struct MergeLaunch {
    static constexpr int MAX_THREADS = 512;
    static constexpr int MIN_BLOCKS = IPT == 8 ? 2 : 1;
};

// Each warp works through its tiles t, t + W, t + 2W, ...; the next tile's indices (and the
// bounds of the one after) are loaded while this tile's gathers are in flight.
template <typename V, int IPT, int MODE>
__global__ void __launch_bounds__(MergeLaunch<IPT>::MAX_THREADS, MergeLaunch<IPT>::MIN_BLOCKS)
    merge_spmv_kernel(const MergeArgs a) {
    using WT = WarpTile<IPT>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    float *vbuf = reinterpret_cast<float *>(smem + wib * WT::BYTES);
    unsigned char *flg = smem + wib * WT::BYTES + WT::VALS * 4;
    const int G = a.num_tiles;
    const int nw = static_cast<int>(gridDim.x) * wpc;
    int t = static_cast<int>(blockIdx.x) * wpc + wib;
    if (t >= G) return;  // the whole warp leaves; there are no block-wide barriers
#pragma unroll
    for (int q = 0; q < IPT; q += 4) *reinterpret_cast<uint32_t *>(flg + IPT * lane + q) = 0u;
    __syncwarp();

    const uint64_t pol = policy_evict_first();
    const int iph = static_cast<int>((reinterpret_cast<uintptr_t>(a.idx) >> 2) & 7);
    const bool save = MODE == kPlain && a.xg != nullptr;

    WBounds cur = bounds_bcast<MODE>(bounds_word<MODE>(a, t, lane));
    int col[IPT], cb;
    load_idx<IPT, MODE>(a, cur, wtile_ok<IPT>(a, cur), iph, lane, pol, col, cb);
    int bw_next = t + nw < G ? bounds_word<MODE>(a, t + nw, lane) : 0;

    for (; t < G; t += nw) {
        const bool ok = wtile_ok<IPT>(a, cur);
        const int nk = cur.k1 - cur.k0;
        const int lead = (iph + cur.k0) & 7;
        const int kb = cur.k0 - lead;
        const int e0 = kb + IPT * lane;
        const uint32_t vm = ok ? slot_mask<IPT>(e0, cur.k0, cur.k1) : 0u;

        const bool has_next = t + nw < G;
        const WBounds nxt = bounds_bcast<MODE>(bw_next);
        float p[IPT], xv[IPT];
        int e_first, e_last;
        uint32_t f;
        if constexpr (MODE == kGatherSum) {
            // The transposed product (no values) finds its row starts before issuing its
            // gathers; the products issue their gathers first and find row starts while they
            // are in flight (each measured the faster order for its mode).
            if (!ok) {
                if (lane == 0) {
                    atomicExch(a.err, static_cast<int>(LB_ERR_BAD_MATRIX));
                    a.carry_row[t] = -1;  // the fixup skips it
                    a.carry_val[t] = 0.f;
                }
                if (has_next) {
                    load_idx<IPT, MODE>(a, nxt, wtile_ok<IPT>(a, nxt), iph, lane, pol, col, cb);
                    bw_next = t + 2 * nw < G ? bounds_word<MODE>(a, t + 2 * nw, lane) : 0;
                }
                cur = nxt;
                continue;
            }
            load_vals<V, IPT, MODE>(a, e0, vm, pol, p);
            f = row_start_flags<IPT>(a, cur, kb, lane, flg, e_first, e_last);
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                xv[q] = (((vm >> q) & 1u) && LB_IN_RANGE(col[q] + cb, a.x_len)) ? __ldg(a.x + (col[q] + cb)) : 0.f;
            if (has_next) {
                load_idx<IPT, MODE>(a, nxt, wtile_ok<IPT>(a, nxt), iph, lane, pol, col, cb);
                bw_next = t + 2 * nw < G ? bounds_word<MODE>(a, t + 2 * nw, lane) : 0;
            }
        } else {
            // 1. This tile's gathers.
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                xv[q] = (((vm >> q) & 1u) && LB_IN_RANGE(col[q] + cb, a.x_len)) ? __ldg(a.x + (col[q] + cb)) : 0.f;

            // 2. The next tile's indices (and the bounds of the one after) while they are in flight.
            if (has_next) {
                load_idx<IPT, MODE>(a, nxt, wtile_ok<IPT>(a, nxt), iph, lane, pol, col, cb);
                bw_next = t + 2 * nw < G ? bounds_word<MODE>(a, t + 2 * nw, lane) : 0;
            }

            if (!ok) {
                if (lane == 0) {
                    atomicExch(a.err, static_cast<int>(LB_ERR_BAD_MATRIX));
                    a.carry_row[t] = -1;  // the fixup skips it
                    a.carry_val[t] = 0.f;
                }
                cur = nxt;
                continue;
            }

            // 3. Values, and the row starts found from the row ends, while the gathers are in flight.
            load_vals<V, IPT, MODE>(a, e0, vm, pol, p);
            e_first = 0, e_last = cur.k0;
            f = cur.r1 > cur.r0 ? row_start_flags<IPT>(a, cur, kb, lane, flg, e_first, e_last) : 0u;
        }

        // 4. Saved gathers for the values gradient, one 32-byte store per lane when aligned.
        if (save && vm != 0u) {
            if (vm == (1u << IPT) - 1u && a.vec_xg) {
#pragma unroll
                for (int h = 0; h < IPT; h += 8) st_stream8(a.xg + e0 + h, pol, xv + h);
            } else {
#pragma unroll
                for (int q = 0; q < IPT; ++q)
                    if ((vm >> q) & 1u) __stcs(a.xg + e0 + q, xv[q]);
            }
        }

        // 5. Products, scanned inside the lane (restarting at row starts), then across lanes.
#pragma unroll
        for (int q = 0; q < IPT; ++q) p[q] = ((vm >> q) & 1u) ? p[q] * xv[q] : 0.f;
        if (cur.r1 == cur.r0) {
            // No row ends in the tile: it lies inside one row, and only its sum (the carry) is
            // needed: the lane's products in order, then a fixed shuffle tree.
            float sum = p[0];
#pragma unroll
            for (int q = 1; q < IPT; ++q) sum += p[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
            if (lane == 0) {
                a.carry_row[t] = cur.r1;
                a.carry_val[t] = sum;
            }
            cur = nxt;
            continue;
        }
#pragma unroll
        for (int q = 1; q < IPT; ++q)
            if (!((f >> q) & 1u)) p[q] += p[q - 1];
        // Across lanes: lane L's last segment began in lane seg, the last lane at or before L
        // holding a row start (lane 0 if none), and a step adds lane L - off's partial sum
        // only while that lane lies in the same segment.
        float v = p[IPT - 1];
        const uint32_t starts = __ballot_sync(0xffffffffu, f != 0u) & (0xffffffffu >> (31 - lane));
        const int seg = starts ? 31 - __clz(starts) : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float vu = __shfl_up_sync(0xffffffffu, v, off);
            if (lane - off >= seg) v += vu;
        }
        float cin = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) cin = 0.f;
        const int ff = f ? __ffs(f) - 1 : IPT;  // slots before the lane's first row start continue its row
#pragma unroll
        for (int q = 0; q < IPT; ++q)
            if (q < ff) p[q] += cin;
#pragma unroll
        for (int q = 0; q < IPT; q += 4)
            *reinterpret_cast<float4 *>(vbuf + ppad(IPT * lane + q)) = make_float4(p[q], p[q + 1], p[q + 2], p[q + 3]);
        __syncwarp();

        // 6. Rows ending in the tile read their sums at their last nonzero (consecutive rows on
        // consecutive lanes); the open row leaves as the tile's carry.
        const int nr = cur.r1 - cur.r0;
        int e_prev = cur.k0;
        auto write_rows = [&](int j, int e) {
            int ep = __shfl_up_sync(0xffffffffu, e, 1);
            if (lane == 0) ep = e_prev;
            e_prev = __shfl_sync(0xffffffffu, e, 31);
            if (j + lane < nr) {
                float yv = 0.f;
                if (e > ep && e > cur.k0 && e <= cur.k1) yv = vbuf[ppad(e - 1 - kb)];
                a.y[cur.r0 + j + lane] = yv;
            }
        };
        if (nr <= 32) {
            write_rows(0, e_first);
        } else {
            for (int j0 = 0; j0 < nr; j0 += 128) {
                int ec[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + 32 * u;
                    ec[u] = j == 0 ? e_first : (j + lane < nr ? __ldg(a.row_end + cur.r0 + j + lane) : 0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (j0 + 32 * u < nr) write_rows(j0 + 32 * u, ec[u]);  // warp-uniform
            }
        }
        if (lane == 0) {
            a.carry_row[t] = cur.r1;
            a.carry_val[t] = (nk > 0 && cur.k1 > e_last) ? vbuf[ppad(cur.k1 - 1 - kb)] : 0.f;
        }
        __syncwarp();  // the value buffer and flags are free for the next tile
        cur = nxt;
    }
}

// Resident CTAs per SM of one kernel instance at `threads` threads per CTA, cached per device
// and CTA size.  The first query of an instance on a device also sets its shared-memory
// carveout to what a full SM of its warps uses (the rest of the unified array stays L1, which
// holds the random gathers in flight).
template <typename V, int IPT, int MODE>
int merge_blocks_per_sm(int threads) {
    constexpr int kMaxDev = 64;
    static int cache[kMaxDev][5] = {};
    static bool carved[kMaxDev] = {};
    static std::mutex mu;
    const int slot = threads / 128 - 1;  // 128, 256, 384, 512 threads
    int dev = 0;
    if (slot < 0 || slot > 3 || threads % 128 != 0) return 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 0;
    if (cache[dev][slot] > 0) return cache[dev][slot];
    std::lock_guard<std::mutex> lock(mu);
    auto kern = merge_spmv_kernel<V, IPT, MODE>;
    if (!carved[dev]) {
        int max_smem = 0, max_warps = 0;
        if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            max_smem <= 0)
            return 0;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return 0;
        // Warps per SM that the registers allow; each holds WarpTile::BYTES, and every resident
        // CTA (at least 128 threads) costs 1 KB of reserved shared memory.
        const int regs = fa.numRegs > 0 ? fa.numRegs : 64;
        max_warps = 65536 / (regs * 32);
        if (max_warps > 64) max_warps = 64;
        const long long need = static_cast<long long>(max_warps) * WarpTile<IPT>::BYTES + (max_warps / 4) * 1024;
        int pct = static_cast<int>((need * 100 + max_smem - 1) / max_smem);
        if (pct > 100) pct = 100;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess) return 0;
        carved[dev] = true;
    }
    int nb = 0;
    const size_t smem = static_cast<size_t>(threads / 32) * WarpTile<IPT>::BYTES;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess) return 0;
    cache[dev][slot] = nb > 0 ? nb : 1;
    return cache[dev][slot];
}

template <typename V, int IPT, int MODE>
cudaError_t launch_merge_cfg(int threads, const MergeArgs &a, cudaStream_t st, cudaEvent_t eb, cudaEvent_t ea) {
    const int per_sm = merge_blocks_per_sm<V, IPT, MODE>(threads);
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const int wpc = threads / 32;
    const long long wave = static_cast<long long>(per_sm) * current_sm_count();
    const long long need = (static_cast<long long>(a.num_tiles) + wpc - 1) / wpc;
    const int grid = static_cast<int>(need < wave ? need : wave);
    const size_t smem = static_cast<size_t>(wpc) * WarpTile<IPT>::BYTES;
    if (eb) cudaEventRecord(eb, st);
    merge_spmv_kernel<V, IPT, MODE><<<grid, threads, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (ea) cudaEventRecord(ea, st);
    if (e != cudaSuccess) return e;
    return launch_fixup(a.num_tiles, a.num_rows, a.carry_row, a.carry_val, a.y, st);
}

// The (threads per CTA, items per lane) shapes compiled into the library.  A tile holds
// 32 * items - 8 work items whatever the CTA size.
#define LB_MERGE_SHAPES(X) X(128, 16) X(256, 8) X(256, 16) X(384, 8) X(512, 8)

template <typename V, int MODE>
cudaError_t dispatch_merge_shape(int threads, int ipt, const MergeArgs &a, cudaStream_t st, cudaEvent_t eb,
                                 cudaEvent_t ea) {
#define LB_TRY_SHAPE(TH, IP) \
    if (threads == TH && ipt == IP) return launch_merge_cfg<V, IP, MODE>(TH, a, st, eb, ea);
    LB_MERGE_SHAPES(LB_TRY_SHAPE)
#undef LB_TRY_SHAPE
    return cudaErrorInvalidValue;
}

// The host-side set-up of one plain-product shape (carveout and occupancy query) without a
// launch, so that a caller can do it before any stream capture.
template <typename V>
cudaError_t prepare_merge_plain(int threads, int ipt) {
#define LB_PREP_SHAPE(TH, IP)                                                                  \
    if (threads == TH && ipt == IP)                                                           \
        return merge_blocks_per_sm<V, IP, kPlain>(TH) > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
    LB_MERGE_SHAPES(LB_PREP_SHAPE)
#undef LB_PREP_SHAPE
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
