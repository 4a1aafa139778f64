// lb_spmm.cu -- load-balanced SpMM, C = A B with B dense (n x kc, row-major), over the
// merge-path partition of A.
//
// The dissertation's SpMM is its SpMV with one more loop, over the columns of B (Ch.4 Sec.
// "Application Space", the SpMM listing); the schedules and their work split carry over
// unchanged.  The tiles are merge-path tiles (rows + nonzeros in equal shares), the row left
// open at the end of a tile goes out as a carry of kc values, and a fixup adds the carries of
// each row in tile order, exactly as for SpMV.  Two kernels, by the width of B:
//
// kc <= 4: the warp-tiled SpMV kernel with a quad of columns in place of each scalar
// (spmm_warp_kernel, warp tiles of 248 items).  Where SpMV gathers one 4-byte x per nonzero,
// this gathers B's whole row (up to 16 bytes, one request).  Per tile, each warp loads the
// tile's indices and values (256-bit per lane, 8 slots per lane; the next tile's indices load
// while this tile works), counts the row ends per slot in shared memory (every slot's row, the
// scan's row starts and the slots holding a row's last nonzero follow), gathers, multiplies,
// scans the products in the lane and across lanes (segmented at row starts), and the lane
// holding a row's last nonzero writes the row; the open row's quad goes to the tile's carry.
// The kernel also runs 2 or 4 lane groups on one tile, each with its own quad (NG); measured
// on wider B that costs more than the block kernel, so only NG = 1 is launched.
//
// kc > 4: a block-tile kernel (spmm_block_kernel, the plan's tiles of up to 2040 items) with
// threads arranged as (column quad, nonzero range): each thread walks its range of nonzeros in
// order, accumulating B[col][4q .. 4q+3] * value per row with FMAs and writing rows that start
// and end inside its range; the first and last partial row of every range meet in shared
// memory.  Per nonzero and quad that is a load and four FMAs, against a load, a multiply and
// scan additions in the warp kernel, which wins beyond one quad.
//
// Summation order is fixed in both (slot or range order in a tile, tile order in the fixup),
// so results are deterministic.
#include "lb_merge.cuh"

namespace lb {

namespace {

template <bool VEC>
__device__ __forceinline__ float4 load_b4(const float *__restrict__ B, long long row, int kc, int q) {
    const int c0 = 4 * q;
    if (VEC) return __ldg(reinterpret_cast<const float4 *>(B + row * kc) + q);
    const float *p = B + row * kc + c0;
    float4 r;
    r.x = c0 < kc ? __ldg(p) : 0.f;
    r.y = c0 + 1 < kc ? __ldg(p + 1) : 0.f;
    r.z = c0 + 2 < kc ? __ldg(p + 2) : 0.f;
    r.w = c0 + 3 < kc ? __ldg(p + 3) : 0.f;
    return r;
}

template <bool VEC>
__device__ __forceinline__ void store_c4(float *__restrict__ C, long long row, int kc, int q, float4 v) {
    const int c0 = 4 * q;
    if (VEC) {
        reinterpret_cast<float4 *>(C + row * kc)[q] = v;
        return;
    }
    float *p = C + row * kc + c0;
    if (c0 < kc) p[0] = v.x;
    if (c0 + 1 < kc) p[1] = v.y;
    if (c0 + 2 < kc) p[2] = v.z;
    if (c0 + 3 < kc) p[3] = v.w;
}

__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

__device__ __forceinline__ void fma4(float4 &acc, float v, float4 b) {
    acc.x = fmaf(v, b.x, acc.x);
    acc.y = fmaf(v, b.y, acc.y);
    acc.z = fmaf(v, b.z, acc.z);
    acc.w = fmaf(v, b.w, acc.w);
}

template <int W>
__device__ __forceinline__ float4 shfl_up4(float4 v, int off) {
    return make_float4(__shfl_up_sync(0xffffffffu, v.x, off, W), __shfl_up_sync(0xffffffffu, v.y, off, W),
                       __shfl_up_sync(0xffffffffu, v.z, off, W), __shfl_up_sync(0xffffffffu, v.w, off, W));
}

constexpr int kIpt = 8;  // slots per lane

struct SpmmArgs {
    MergeArgs t;  // the tiles, rows, column indices, values and the error word (x, y unused)
    const float *B;
    float *C;
    int kc;
    float *carry_val;  // [G * kc]; t.carry_row[G] holds the rows
};

}  // namespace

// Work items per tile of the warp-tiled kernel: 32 lanes x 8 slots, less 8.
int spmm_warp_tile_items() { return 32 * kIpt - 8; }

template <typename V, int NG, bool VEC>
__global__ void __launch_bounds__(256, 2) spmm_warp_kernel(const SpmmArgs s) {
    constexpr int LG = 32 / NG;       // lanes per group
    constexpr int SLOTS = LG * kIpt;  // slots per tile
    const MergeArgs &a = s.t;
    extern __shared__ __align__(16) int smem_cnt[];
    const int lane = threadIdx.x & 31;
    const int grp = lane / LG, li = lane % LG;
    const int wib = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    int *cnt = smem_cnt + wib * SLOTS;  // row ends per slot of the current tile
    const int G = a.num_tiles;
    const int nw = static_cast<int>(gridDim.x) * wpc;
    int t = static_cast<int>(blockIdx.x) * wpc + wib;
    if (t >= G) return;
    if (grp == 0) {
        *reinterpret_cast<int4 *>(cnt + kIpt * li) = make_int4(0, 0, 0, 0);
        *reinterpret_cast<int4 *>(cnt + kIpt * li + 4) = make_int4(0, 0, 0, 0);
    }
    __syncwarp();
    const uint64_t pol = policy_evict_first();
    const int iph = static_cast<int>((reinterpret_cast<uintptr_t>(a.idx) >> 2) & 7);
    const int kc = s.kc;
    const int nq = (kc + 3) >> 2;
    const unsigned gmask = (NG == 1) ? 0xffffffffu : (((1u << LG) - 1u) << (grp * LG));

    // Tile bounds; the lane's slots start at element kb + 8 li (group-relative lanes).
    auto tile_ok = [&](const WBounds &b) {
        return b.r0 >= 0 && b.r0 <= b.r1 && b.r1 <= a.num_rows && b.k0 >= 0 && b.k0 <= b.k1 &&
               b.k1 <= a.num_atoms && (b.r1 - b.r0) + (b.k1 - b.k0) <= SLOTS - 8;
    };
    auto load_cols = [&](const WBounds &b, bool ok, int (&col)[kIpt]) {
#pragma unroll
        for (int q = 0; q < kIpt; ++q) col[q] = 0;
        if (!ok) return;
        const int e0 = b.k0 - ((iph + b.k0) & 7) + kIpt * li;
        if (e0 >= b.k1 || e0 + kIpt <= b.k0) return;
        if (e0 >= 0 && e0 + kIpt <= a.num_atoms) {
            uint32_t r[8];
            ld_stream8(a.idx + e0, pol, r);
#pragma unroll
            for (int q = 0; q < 8; ++q) col[q] = static_cast<int>(r[q]);
        } else {
#pragma unroll
            for (int q = 0; q < kIpt; ++q)
                if (e0 + q >= b.k0 && e0 + q < b.k1) col[q] = __ldg(a.idx + e0 + q);
        }
    };

    WBounds cur = bounds_bcast<kPlain>(bounds_word<kPlain>(a, t, lane));
    int col[kIpt];
    load_cols(cur, tile_ok(cur), col);
    int bw_next = t + nw < G ? bounds_word<kPlain>(a, t + nw, lane) : 0;

    for (; t < G; t += nw) {
        const bool ok = tile_ok(cur);
        const WBounds nxt = bounds_bcast<kPlain>(bw_next);
        const bool has_next = t + nw < G;
        int col_next[kIpt];
        if (has_next) {
            load_cols(nxt, tile_ok(nxt), col_next);
            bw_next = t + 2 * nw < G ? bounds_word<kPlain>(a, t + 2 * nw, lane) : 0;
        }
        if (!ok) {
            if (lane == 0) {
                atomicExch(a.err, static_cast<int>(LB_ERR_BAD_MATRIX));
                a.carry_row[t] = -1;  // the fixup skips it
            }
        } else {
            const int lead = (iph + cur.k0) & 7;
            const int kb = cur.k0 - lead;
            const int e0 = kb + kIpt * li;
            const uint32_t vm = slot_mask<kIpt>(e0, cur.k0, cur.k1);
            float vv[kIpt];
            load_vals<V, kIpt, kPlain>(a, e0, vm, pol, vv);

            // Row ends inside the tile, counted per slot: a row ending at nonzero e (its last
            // nonzero is e - 1) counts at slot e - kb, the next row's first nonzero.
            const int nr = cur.r1 - cur.r0;
            int e_last = cur.k0;  // end of the tile's last complete row (k0 if none)
            for (int j = 0; j < nr; j += 32) {
                const bool in = j + lane < nr;
                const int e = in ? __ldg(a.row_end + cur.r0 + j + lane) : 0;
                if (in && e >= cur.k0 && e < cur.k1) atomicAdd(cnt + (e - kb), 1);
                if (j + 32 >= nr) e_last = __shfl_sync(0xffffffffu, e, (nr - 1) & 31);
            }
            __syncwarp();
            int c[kIpt];
            {
                const int4 c0 = *reinterpret_cast<const int4 *>(cnt + kIpt * li);
                const int4 c1 = *reinterpret_cast<const int4 *>(cnt + kIpt * li + 4);
                c[0] = c0.x, c[1] = c0.y, c[2] = c0.z, c[3] = c0.w, c[4] = c1.x, c[5] = c1.y, c[6] = c1.z, c[7] = c1.w;
            }
            __syncwarp();
            if (grp == 0) {
                *reinterpret_cast<int4 *>(cnt + kIpt * li) = make_int4(0, 0, 0, 0);
                *reinterpret_cast<int4 *>(cnt + kIpt * li + 4) = make_int4(0, 0, 0, 0);
            }
            // Row starts (scan segments), rows' last nonzeros, and the row of each slot.
            uint32_t f = 0u, last = 0u;
            const int c_next = __shfl_down_sync(0xffffffffu, c[0], 1, LG);  // the group's next lane
            int tot = 0;
#pragma unroll
            for (int q = 0; q < kIpt; ++q) {
                tot += c[q];
                if (c[q] > 0) f |= 1u << q;
                const int cn = q + 1 < kIpt ? c[q + 1] : (li < LG - 1 ? c_next : 0);
                const int k = e0 + q;
                // Slot q holds a row's last nonzero: a row ends right after it inside the tile,
                // or it is the tile's last nonzero and the tile's last complete row ends there.
                if (((vm >> q) & 1u) && ((k + 1 < cur.k1 && cn > 0) || (k + 1 == cur.k1 && e_last == cur.k1)))
                    last |= 1u << q;
            }
            int incl = tot;
#pragma unroll
            for (int off = 1; off < LG; off <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, off, LG);
                if (li >= off) incl += u;
            }
            const int row_base = cur.r0 + incl - tot;  // rows ended before this lane's first slot
            const uint32_t starts =
                ((__ballot_sync(0xffffffffu, f != 0u) & gmask) >> (grp * LG)) & (0xffffffffu >> (31 - li));
            const int seg = starts ? 31 - __clz(starts) : 0;
            const int ff = f ? __ffs(f) - 1 : kIpt;
            // The slot holding the tile's last nonzero, when the open row has nonzeros here.
            const bool open_here = cur.k1 > e_last && cur.k1 - 1 >= e0 && cur.k1 - 1 < e0 + kIpt;
            const int q_open = cur.k1 - 1 - e0;

            const int npass = (nq + NG - 1) / NG;  // the same trip count in every group
            for (int pass = 0; pass < npass; ++pass) {
                const int qd = pass * NG + grp;
                const bool act = qd < nq;
                float4 p[kIpt];
#pragma unroll
                for (int q = 0; q < kIpt; ++q)
                    p[q] = act && ((vm >> q) & 1u) && LB_IN_RANGE(col[q], a.x_len) ? load_b4<VEC>(s.B, col[q], kc, qd)
                                                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < kIpt; ++q)
                    p[q] = make_float4(p[q].x * vv[q], p[q].y * vv[q], p[q].z * vv[q], p[q].w * vv[q]);
#pragma unroll
                for (int q = 1; q < kIpt; ++q)
                    if (!((f >> q) & 1u)) p[q] = add4(p[q], p[q - 1]);
                float4 v = p[kIpt - 1];
#pragma unroll
                for (int off = 1; off < LG; off <<= 1) {
                    const float4 vu = shfl_up4<LG>(v, off);
                    if (li - off >= seg) v = add4(v, vu);
                }
                float4 cin = shfl_up4<LG>(v, 1);
                if (li == 0) cin = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < kIpt; ++q)
                    if (q < ff) p[q] = add4(p[q], cin);
                if (act) {
                    int row = row_base;
#pragma unroll
                    for (int q = 0; q < kIpt; ++q) {
                        row += c[q];
                        if ((last >> q) & 1u) store_c4<VEC>(s.C, row, kc, qd, p[q]);
                        if (open_here && q == q_open) store_c4<VEC>(s.carry_val, t, kc, qd, p[q]);
                    }
                }
            }
            // Rows whose part inside the tile is empty, and an open row without nonzeros here.
            int e_prev = cur.k0;
            for (int j = 0; j < nr; j += 32) {
                const bool in = j + lane < nr;
                const int e = in ? __ldg(a.row_end + cur.r0 + j + lane) : 0;
                int sp = __shfl_up_sync(0xffffffffu, e, 1);
                if (lane == 0) sp = e_prev;
                e_prev = __shfl_sync(0xffffffffu, e, 31);
                if (in && e <= sp)
                    for (int qd = 0; qd < nq; ++qd)
                        store_c4<VEC>(s.C, cur.r0 + j + lane, kc, qd, make_float4(0.f, 0.f, 0.f, 0.f));
            }
            if (cur.k1 <= e_last)
                for (int qd = lane; qd < nq; qd += 32) store_c4<VEC>(s.carry_val, t, kc, qd, make_float4(0.f, 0.f, 0.f, 0.f));
            if (lane == 0) a.carry_row[t] = cur.r1;
        }
        if (has_next) {
#pragma unroll
            for (int q = 0; q < kIpt; ++q) col[q] = col_next[q];
        }
        __syncwarp();  // the counts are cleared for the next tile
        cur = nxt;
    }
}

// kc = 8 or 16 with B, C and the carries 32-byte aligned: the warp-tiled kernel with B's row
// gathered 8 columns at a time, one 256-bit load per slot (one request per nonzero and chunk,
// as in SpMV).  Per chunk, each lane walks its 8 slots once with a running sum per column: a
// row start (a slot where row ends were counted) closes the lane's first segment (its head)
// or a finished row, which the lane writes at once; the running sum left at the end (the
// lane's tail, or its whole sum when no row starts in it) goes into a segmented shuffle scan
// across lanes, whose carry-in completes the head row and the tile's open row.  The row
// structure (counts per slot, row starts, the slots holding rows' last nonzeros) is worked
// out once per tile and reused by every chunk.  Wider B stays on the block kernel, whose
// threads gather a whole 128-byte row of B in one instruction: chunks gathered apart fetch
// the same DRAM line again once B no longer fits in L2.
constexpr int kWideCols = 8;

__device__ __forceinline__ void gather_b8(const float *p, float (&r)[kWideCols]) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
        : "l"(p));
}

__device__ __forceinline__ void store_c8(float *p, const float (&v)[kWideCols]) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}

// 128 threads per CTA.  A lane's 8 slots gather in two groups of 4 (32 registers in flight):
// the second group's gathers go out when the first group's products are summed.  That fits
// 128 registers, 4 CTAs (16 warps) per SM; all 8 slots in flight at once take 167 registers
// and 12 warps, measured 10% slower when B fits in L2 (and the same when it does not), and 4
// groups of 2 slower at every size.
constexpr int kWideThreads = 128;
constexpr int kWideMinBlocks = 4;
constexpr int kWideGroups = 2;

template <typename V>
__global__ void __launch_bounds__(kWideThreads, kWideMinBlocks) spmm_wide_kernel(const SpmmArgs s) {
    constexpr int W = kWideCols;
    const MergeArgs &a = s.t;
    extern __shared__ __align__(16) int smem_cnt[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    int *cnt = smem_cnt + wib * 32 * kIpt;  // row ends per slot of the current tile
    const int G = a.num_tiles;
    const int nw = static_cast<int>(gridDim.x) * wpc;
    int t = static_cast<int>(blockIdx.x) * wpc + wib;
    if (t >= G) return;
    *reinterpret_cast<int4 *>(cnt + kIpt * lane) = make_int4(0, 0, 0, 0);
    *reinterpret_cast<int4 *>(cnt + kIpt * lane + 4) = make_int4(0, 0, 0, 0);
    __syncwarp();
    const uint64_t pol = policy_evict_first();
    const int iph = static_cast<int>((reinterpret_cast<uintptr_t>(a.idx) >> 2) & 7);
    const int kc = s.kc;
    const int nch = kc / W;

    auto tile_ok = [&](const WBounds &b) {
        return b.r0 >= 0 && b.r0 <= b.r1 && b.r1 <= a.num_rows && b.k0 >= 0 && b.k0 <= b.k1 &&
               b.k1 <= a.num_atoms && (b.r1 - b.r0) + (b.k1 - b.k0) <= 32 * kIpt - 8;
    };
    auto load_cols = [&](const WBounds &b, bool ok, int (&col)[kIpt]) {
#pragma unroll
        for (int q = 0; q < kIpt; ++q) col[q] = 0;
        if (!ok) return;
        const int e0 = b.k0 - ((iph + b.k0) & 7) + kIpt * lane;
        if (e0 >= b.k1 || e0 + kIpt <= b.k0) return;
        if (e0 >= 0 && e0 + kIpt <= a.num_atoms) {
            uint32_t r[8];
            ld_stream8(a.idx + e0, pol, r);
#pragma unroll
            for (int q = 0; q < 8; ++q) col[q] = static_cast<int>(r[q]);
        } else {
#pragma unroll
            for (int q = 0; q < kIpt; ++q)
                if (e0 + q >= b.k0 && e0 + q < b.k1) col[q] = __ldg(a.idx + e0 + q);
        }
    };

    WBounds cur = bounds_bcast<kPlain>(bounds_word<kPlain>(a, t, lane));
    int col[kIpt];
    load_cols(cur, tile_ok(cur), col);
    int bw_next = t + nw < G ? bounds_word<kPlain>(a, t + nw, lane) : 0;

    for (; t < G; t += nw) {
        const bool ok = tile_ok(cur);
        const WBounds nxt = bounds_bcast<kPlain>(bw_next);
        const bool has_next = t + nw < G;
        if (!ok) {
            if (lane == 0) {
                atomicExch(a.err, static_cast<int>(LB_ERR_BAD_MATRIX));
                a.carry_row[t] = -1;  // the fixup skips it
            }
            if (has_next) {
                load_cols(nxt, tile_ok(nxt), col);
                bw_next = t + 2 * nw < G ? bounds_word<kPlain>(a, t + 2 * nw, lane) : 0;
            }
            cur = nxt;
            continue;
        }
        const int kb = cur.k0 - ((iph + cur.k0) & 7);
        const int e0 = kb + kIpt * lane;
        const uint32_t vm = slot_mask<kIpt>(e0, cur.k0, cur.k1);
        uint32_t gm = 0u;  // slots whose gather is in range
#pragma unroll
        for (int q = 0; q < kIpt; ++q)
            if (((vm >> q) & 1u) && LB_IN_RANGE(col[q], a.x_len)) gm |= 1u << q;

        // 1. The first chunk's gathers (of its first slot group).
        constexpr int GS = kIpt / kWideGroups;
        float b[GS][W];
        auto gather_group = [&](int g, int ch) {
#pragma unroll
            for (int i = 0; i < GS; ++i) {
                const int q = g * GS + i;
                if ((gm >> q) & 1u) {
                    gather_b8(s.B + static_cast<long long>(col[q]) * kc + ch * W, b[i]);
                } else {
#pragma unroll
                    for (int j = 0; j < W; ++j) b[i][j] = 0.f;
                }
            }
        };
        gather_group(0, 0);

        // 2. While they are in flight: the next tile's indices (kept apart while this tile
        // still gathers further chunks), the values and the row structure.
        int col_next[kIpt];
        if (has_next) {
            load_cols(nxt, tile_ok(nxt), col_next);
            bw_next = t + 2 * nw < G ? bounds_word<kPlain>(a, t + 2 * nw, lane) : 0;
        }
        float vv[kIpt];
        load_vals<V, kIpt, kPlain>(a, e0, vm, pol, vv);
#pragma unroll
        for (int q = 0; q < kIpt; ++q)
            if (!((vm >> q) & 1u)) vv[q] = 0.f;  // slots outside the tile add nothing
        const int nr = cur.r1 - cur.r0;
        int e_last = cur.k0;  // end of the tile's last complete row (k0 if none)
        for (int j = 0; j < nr; j += 32) {
            const bool in = j + lane < nr;
            const int e = in ? __ldg(a.row_end + cur.r0 + j + lane) : 0;
            if (in && e >= cur.k0 && e < cur.k1) atomicAdd(cnt + (e - kb), 1);
            if (j + 32 >= nr) e_last = __shfl_sync(0xffffffffu, e, (nr - 1) & 31);
        }
        __syncwarp();
        int c[kIpt];
        {
            const int4 c0 = *reinterpret_cast<const int4 *>(cnt + kIpt * lane);
            const int4 c1 = *reinterpret_cast<const int4 *>(cnt + kIpt * lane + 4);
            c[0] = c0.x, c[1] = c0.y, c[2] = c0.z, c[3] = c0.w, c[4] = c1.x, c[5] = c1.y, c[6] = c1.z, c[7] = c1.w;
        }
        __syncwarp();
        *reinterpret_cast<int4 *>(cnt + kIpt * lane) = make_int4(0, 0, 0, 0);
        *reinterpret_cast<int4 *>(cnt + kIpt * lane + 4) = make_int4(0, 0, 0, 0);
        uint32_t f = 0u, last = 0u, cpk0 = 0u, cpk1 = 0u;  // counts packed a byte per slot (<= 248)
        const int c_next = __shfl_down_sync(0xffffffffu, c[0], 1);
        int tot = 0;
#pragma unroll
        for (int q = 0; q < kIpt; ++q) {
            tot += c[q];
            if (c[q] > 0) f |= 1u << q;
            if (q < 4)
                cpk0 |= static_cast<uint32_t>(c[q]) << (8 * q);
            else
                cpk1 |= static_cast<uint32_t>(c[q]) << (8 * (q - 4));
            const int cn = q + 1 < kIpt ? c[q + 1] : (lane < 31 ? c_next : 0);
            const int k = e0 + q;
            // Slot q holds a row's last nonzero: a row ends right after it inside the tile, or
            // it is the tile's last nonzero and the tile's last complete row ends there.
            if (((vm >> q) & 1u) && ((k + 1 < cur.k1 && cn > 0) || (k + 1 == cur.k1 && e_last == cur.k1)))
                last |= 1u << q;
        }
        int incl = tot;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += u;
        }
        const int row_base = cur.r0 + incl - tot;  // rows ended before this lane's first slot
        const uint32_t starts = __ballot_sync(0xffffffffu, f != 0u) & (0xffffffffu >> (31 - lane));
        const int seg = starts ? 31 - __clz(starts) : 0;
        const bool open_here = cur.k1 > e_last && cur.k1 - 1 >= e0 && cur.k1 - 1 < e0 + kIpt;
        const int m = a.num_rows;

#pragma unroll 1
        for (int ch = 0; ch < nch; ++ch) {
            // 3. The lane's slots in order, with a running sum per column.
            float acc[W], head[W];
#pragma unroll
            for (int j = 0; j < W; ++j) acc[j] = 0.f, head[j] = 0.f;
            bool started = false;
            int row = row_base, row_h = -1;
#pragma unroll
            for (int q = 0; q < kIpt; ++q) {
                if (q % GS == 0 && (ch > 0 || q > 0)) gather_group(q / GS, ch);
                const float *bq = b[q % GS];
                if ((f >> q) & 1u) {
                    if (!started) {
#pragma unroll
                        for (int j = 0; j < W; ++j) head[j] = acc[j];
                    }
                    started = true;
#pragma unroll
                    for (int j = 0; j < W; ++j) acc[j] = 0.f;
                }
#pragma unroll
                for (int j = 0; j < W; ++j) acc[j] = fmaf(vv[q], bq[j], acc[j]);
                row += static_cast<int>(((q < 4 ? cpk0 : cpk1) >> (8 * (q & 3))) & 0xffu);
                if ((last >> q) & 1u) {
                    if (started) {
                        if (static_cast<unsigned>(row) < static_cast<unsigned>(m))
                            store_c8(s.C + static_cast<long long>(row) * kc + ch * W, acc);
                    } else {
                        row_h = row;
                    }
                }
            }
            if (!started) {
#pragma unroll
                for (int j = 0; j < W; ++j) head[j] = acc[j];
            }
            // 4. Across lanes: lane L's running sums join those of the lanes back to the last
            // one holding a row start (seg), whose tail begins the segment.
            float v[W], cin[W];
#pragma unroll
            for (int j = 0; j < W; ++j) v[j] = acc[j];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    const float vu = __shfl_up_sync(0xffffffffu, v[j], off);
                    if (lane - off >= seg) v[j] += vu;
                }
            }
#pragma unroll
            for (int j = 0; j < W; ++j) {
                cin[j] = __shfl_up_sync(0xffffffffu, v[j], 1);
                if (lane == 0) cin[j] = 0.f;
            }
            if (row_h >= 0 && row_h < m) {
                float o[W];
#pragma unroll
                for (int j = 0; j < W; ++j) o[j] = cin[j] + head[j];
                store_c8(s.C + static_cast<long long>(row_h) * kc + ch * W, o);
            }
            if (open_here) {  // the open row's sum in this tile: its tail here, or all of it with the carry-in
                float o[W];
#pragma unroll
                for (int j = 0; j < W; ++j) o[j] = started ? acc[j] : cin[j] + acc[j];
                store_c8(s.carry_val + static_cast<long long>(t) * kc + ch * W, o);
            }
        }

        // 5. Rows whose part inside the tile is empty, and an open row without nonzeros here.
        int e_prev = cur.k0;
        for (int j = 0; j < nr; j += 32) {
            const bool in = j + lane < nr;
            const int e = in ? __ldg(a.row_end + cur.r0 + j + lane) : 0;
            int sp = __shfl_up_sync(0xffffffffu, e, 1);
            if (lane == 0) sp = e_prev;
            e_prev = __shfl_sync(0xffffffffu, e, 31);
            if (in && e <= sp) {
                float z[W];
#pragma unroll
                for (int j2 = 0; j2 < W; ++j2) z[j2] = 0.f;
                for (int cc = 0; cc < kc; cc += W) store_c8(s.C + static_cast<long long>(cur.r0 + j + lane) * kc + cc, z);
            }
        }
        if (cur.k1 <= e_last)
            for (int cc = lane; cc < kc; cc += 32) s.carry_val[static_cast<long long>(t) * kc + cc] = 0.f;
        if (lane == 0) a.carry_row[t] = cur.r1;
        if (has_next) {
#pragma unroll
            for (int q = 0; q < kIpt; ++q) col[q] = col_next[q];
        }
        __syncwarp();  // the counts are cleared for the next tile
        cur = nxt;
    }
}

// NQ column quads per pass (a power of two, <= THREADS); NG = THREADS / NQ nonzero ranges.
template <typename V, int THREADS, int TMAX, bool VEC>
__global__ void __launch_bounds__(THREADS) spmm_block_kernel(int G, int m, int n, int kc, int nq, const int *__restrict__ tile_row,
                                                       const int *__restrict__ tile_nz,
                                                       const int *__restrict__ row_end, const int *__restrict__ ci,
                                                       const V *__restrict__ values, const float *__restrict__ B,
                                                       float *__restrict__ C, int *__restrict__ carry_row,
                                                       float *__restrict__ carry_val) {
    constexpr int IPT = TMAX / THREADS;
    constexpr int WARPS = THREADS / 32;
    static_assert(IPT % 4 == 0, "slots are scanned four at a time");
    __shared__ int s_re[TMAX];
    __shared__ __align__(16) int s_row[TMAX];
    __shared__ int s_col[TMAX];
    __shared__ float s_val[TMAX];
    __shared__ int wsum[WARPS];
    __shared__ int p_row[2][THREADS];       // per thread: first and last partial row (-1: none)
    __shared__ float4 p_acc[2][THREADS];    // their partial sums
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kq = (kc + 3) >> 2;           // column quads of C
    const int ng = THREADS / nq;            // nonzero ranges per pass
    const int q_loc = tid % nq, g = tid / nq;
    for (int i = tid; i < TMAX; i += THREADS) s_row[i] = 0;
    __syncthreads();
    for (int tile = blockIdx.x; tile < G; tile += gridDim.x) {
        const int r0 = __ldg(tile_row + tile), r1 = __ldg(tile_row + tile + 1);
        const int k0 = __ldg(tile_nz + tile), k1 = __ldg(tile_nz + tile + 1);
        const int nr = r1 - r0, nk = k1 - k0;
        if (nr < 0 || nk < 0 || nr > TMAX || nk > TMAX) continue;  // malformed offsets (block-uniform)
        for (int j = tid; j < nk; j += THREADS) {
            const int c = __ldg(ci + k0 + j);
            const bool in = LB_IN_RANGE(c, n);  // always true outside the range-checked build
            s_col[j] = in ? c : 0;
            s_val[j] = in ? to_f32(values[k0 + j]) : 0.f;
        }
        for (int r = tid; r < nr; r += THREADS) {
            const int e = __ldg(row_end + r0 + r) - k0;  // first nonzero of the next row, tile-local
            s_re[r] = e;
            if (e >= 0 && e < nk) atomicAdd(&s_row[e], 1);
        }
        __syncthreads();
        // Rows: inclusive prefix sum of the per-slot row-end counts.
        {
            const int s0 = tid * IPT;
            int c[IPT];
#pragma unroll
            for (int q = 0; q < IPT; q += 4) {
                const int4 t = *reinterpret_cast<const int4 *>(s_row + s0 + q);
                c[q] = t.x;
                c[q + 1] = t.y;
                c[q + 2] = t.z;
                c[q + 3] = t.w;
            }
#pragma unroll
            for (int q = 1; q < IPT; ++q) c[q] += c[q - 1];
            const int tot = c[IPT - 1];
            int incl = tot;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            int base = incl - tot;
            for (int w = 0; w < warp; ++w) base += wsum[w];
#pragma unroll
            for (int q = 0; q < IPT; q += 4)
                *reinterpret_cast<int4 *>(s_row + s0 + q) =
                    make_int4(base + c[q], base + c[q + 1], base + c[q + 2], base + c[q + 3]);
        }
        __syncthreads();
        // Rows ending in this tile without nonzeros in it start as zeros (carries from earlier
        // tiles, if any, are added by the fixup).
        for (int r = tid; r < nr; r += THREADS) {
            const int start = r > 0 ? s_re[r - 1] : 0;
            if (s_re[r] <= start && start >= 0)
                for (int c = 0; c < kc; ++c) C[static_cast<long long>(r0 + r) * kc + c] = 0.f;
        }
        const int len = (nk + ng - 1) / ng;  // nonzeros per range
        const int jb = g * len, je = min(nk, jb + len);
        for (int qb = 0; qb < kq; qb += nq) {
            const int q = qb + q_loc;
            const bool active = q < kq;
            if (active && g == 0) {  // the tile's carry is 0 unless the open row has nonzeros here
                float *cv = carry_val + static_cast<long long>(tile) * kc + 4 * q;
                if (4 * q < kc) cv[0] = 0.f;
                if (4 * q + 1 < kc) cv[1] = 0.f;
                if (4 * q + 2 < kc) cv[2] = 0.f;
                if (4 * q + 3 < kc) cv[3] = 0.f;
            }
            if (nr == 0) {
                // No row ends in the tile: all its nonzeros belong to the open row.  Each range
                // sums its products, a tree over the ranges (fixed order) adds them up, and the
                // total is the tile's carry.
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                if (active) {
                    constexpr int U = 8;
                    for (int j0 = jb; j0 < je; j0 += U) {
                        float4 b[U];
                        float vl[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int j = j0 + u;
                            const bool in = j < je;
                            vl[u] = in ? s_val[j] : 0.f;
                            b[u] = in ? load_b4<VEC>(B, s_col[j], kc, q) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) fma4(acc, vl[u], b[u]);
                    }
                }
                p_acc[0][tid] = acc;
                __syncthreads();
                for (int half = ng >> 1; half > 0; half >>= 1) {  // ng is a power of two
                    if (g < half) p_acc[0][tid] = add4(p_acc[0][tid], p_acc[0][tid + half * nq]);
                    __syncthreads();
                }
                if (active && g == 0) {
                    const float4 sum = p_acc[0][tid];
                    float *cv = carry_val + static_cast<long long>(tile) * kc + 4 * q;
                    if (4 * q < kc) cv[0] = sum.x;
                    if (4 * q + 1 < kc) cv[1] = sum.y;
                    if (4 * q + 2 < kc) cv[2] = sum.z;
                    if (4 * q + 3 < kc) cv[3] = sum.w;
                }
                __syncthreads();
                continue;
            }
            // Walk this range's nonzeros in order.
            int cur = -1, first_row = -1;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f), first_acc = acc;
            if (active) {
                // Eight nonzeros at a time: their B rows are requested together before any is
                // used, so each thread keeps eight gathers in flight.
                constexpr int U = 8;
                for (int j0 = jb; j0 < je; j0 += U) {
                    float4 b[U];
                    int rw[U];
                    float vl[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int j = j0 + u;
                        const bool in = j < je;
                        rw[u] = in ? s_row[j] : -1;
                        vl[u] = in ? s_val[j] : 0.f;
                        b[u] = in ? load_b4<VEC>(B, s_col[j], kc, q) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (rw[u] < 0) break;
                        if (rw[u] != cur) {
                            if (cur >= 0) {
                                if (first_row < 0) {
                                    first_row = cur;
                                    first_acc = acc;
                                } else {
                                    store_c4<VEC>(C, r0 + cur, kc, q, acc);  // started and ended in this range
                                }
                            }
                            cur = rw[u];
                            acc = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        fma4(acc, vl[u], b[u]);
                    }
                }
            }
            if (first_row < 0) {  // the range holds at most one row
                p_row[0][tid] = cur;
                p_acc[0][tid] = acc;
                p_row[1][tid] = -1;
            } else {
                p_row[0][tid] = first_row;
                p_acc[0][tid] = first_acc;
                p_row[1][tid] = cur;
                p_acc[1][tid] = acc;
            }
            __syncthreads();
            // Join the ranges' partial rows: the range where a row first appears in this tile
            // (its head) sums that row's partials forward through the ranges it spans, then
            // writes the row to C (it ends in the tile) or to the tile's carry (the open row).
            if (active) {
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    const int R = p_row[w][tid];
                    if (R < 0) continue;
                    if (w == 0 && g > 0) {  // the first partial is a head unless range g-1 ends in R
                        const int tp = (g - 1) * nq + q_loc;
                        const int prev_last = p_row[1][tp] >= 0 ? p_row[1][tp] : p_row[0][tp];
                        if (prev_last == R) continue;
                    }
                    float4 sum = p_acc[w][tid];
                    if (w == 1 || p_row[1][tid] < 0) {  // R is this range's last row: it may go on
                        for (int g2 = g + 1; g2 < ng; ++g2) {
                            const int t2 = g2 * nq + q_loc;
                            if (p_row[0][t2] != R) break;
                            sum = add4(sum, p_acc[0][t2]);
                            if (p_row[1][t2] >= 0) break;  // a new row starts inside range g2
                        }
                    }
                    if (R < nr) {
                        store_c4<VEC>(C, r0 + R, kc, q, sum);
                    } else {
                        float *cv = carry_val + static_cast<long long>(tile) * kc + 4 * q;
                        if (4 * q < kc) cv[0] = sum.x;
                        if (4 * q + 1 < kc) cv[1] = sum.y;
                        if (4 * q + 2 < kc) cv[2] = sum.z;
                        if (4 * q + 3 < kc) cv[3] = sum.w;
                    }
                }
            }
            __syncthreads();
        }
        if (tid == 0) carry_row[tile] = r1;
        // Ready for the next tile: counts back to zero.
        for (int i = tid; i < TMAX; i += THREADS) s_row[i] = 0;
        __syncthreads();
    }
}

// Fixup: C[r][:] += the carries of row r, in tile order.  A warp per run of equal carry
// rows: it finds the run's end 32 tiles per probe; a run of one tile is added column by
// column; a longer run is summed by the lanes over the run's carries as one contiguous array
// (coalesced, eight loads in flight per lane), each lane keeping one column with compensated
// addition when 32 % kc == 0, joined by a fixed shuffle tree; otherwise lanes take columns
// and walk the run.
__global__ void spmm_fixup_kernel(int G, int m, int kc, const int *__restrict__ carry_row,
                                  const float *__restrict__ carry_val, float *__restrict__ C) {
    const int lane = threadIdx.x & 31;
    const long long warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
    for (long long c = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; c < G; c += warps) {
        const int r = __ldg(carry_row + c);
        if (static_cast<unsigned>(r) >= static_cast<unsigned>(m)) continue;
        if (c > 0 && __ldg(carry_row + c - 1) == r) continue;
        long long end = c + 1;
        for (;;) {  // 32 tiles per probe
            const long long p = end + lane;
            const bool same = p < G && __ldg(carry_row + p) == r;
            const unsigned b = __ballot_sync(0xffffffffu, same);
            const int run = b == 0xffffffffu ? 32 : __ffs(~b) - 1;  // leading tiles of the probe in the run
            end += run;
            if (run < 32) break;
        }
        const long long len = end - c;
        float *crow = C + static_cast<long long>(r) * kc;
        if (len == 1) {
            for (int col = lane; col < kc; col += 32) crow[col] += __ldg(carry_val + c * kc + col);
        } else if (kc <= 32 && 32 % kc == 0) {
            const float *base = carry_val + c * kc;
            const long long total = len * kc;
            float s = 0.f, comp = 0.f;
            long long i = lane;
            for (; i + 7 * 32 < total; i += 8 * 32) {
                float u[8];
#pragma unroll
                for (int h = 0; h < 8; ++h) u[h] = __ldg(base + i + 32 * h);
#pragma unroll
                for (int h = 0; h < 8; ++h) kbn_add(s, comp, u[h]);
            }
            for (; i < total; i += 32) kbn_add(s, comp, __ldg(base + i));
            s += comp;
            for (int off = 16; off >= kc; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (lane < kc) crow[lane] += s;
        } else {
            for (int col = lane; col < kc; col += 32) {
                float s = 0.f, comp = 0.f;
                for (long long u = c; u < end; ++u) kbn_add(s, comp, __ldg(carry_val + u * kc + col));
                crow[col] += s + comp;
            }
        }
    }
}

template <typename V, bool VEC>
static cudaError_t launch_spmm_warp_t(const SpmmArgs &s, cudaStream_t st) {
    auto kern = spmm_warp_kernel<V, 1, VEC>;
    constexpr int threads = 256;
    const size_t smem = static_cast<size_t>(threads / 32) * 32 * kIpt * sizeof(int);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    long long grid = static_cast<long long>(per_sm > 0 ? per_sm : 1) * current_sm_count();
    const long long need = (static_cast<long long>(s.t.num_tiles) + threads / 32 - 1) / (threads / 32);
    if (grid > need) grid = need;
    kern<<<static_cast<int>(grid), threads, smem, st>>>(s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    long long fb = (static_cast<long long>(s.t.num_tiles) + 7) / 8;
    const long long cap = static_cast<long long>(current_sm_count()) * 8;
    if (fb > cap) fb = cap;
    spmm_fixup_kernel<<<static_cast<int>(fb), 256, 0, st>>>(s.t.num_tiles, s.t.num_rows, s.kc, s.t.carry_row,
                                                           s.carry_val, s.C);
    return cudaGetLastError();
}

cudaError_t launch_spmm_warp(lb_dtype vdt, int G, int m, int n, int nnz, int kc, const int *tile_row,
                             const int *tile_nz, const int *row_end, const int *ci, const void *values, const float *B,
                             float *C, int *carry_row, float *carry_val, int *err, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    if (kc > 4) return cudaErrorInvalidValue;
    SpmmArgs s{};
    s.t.num_tiles = G;
    s.t.num_rows = m;
    s.t.num_atoms = nnz;
    s.t.tile_row = tile_row;
    s.t.tile_nz = tile_nz;
    s.t.row_end = row_end;
    s.t.idx = ci;
    s.t.val = values;
    s.t.x_len = n;
    s.t.carry_row = carry_row;
    s.t.err = err;
    set_merge_alignment(s.t, vdt == LB_F32 ? 4 : 2);
    s.B = B;
    s.C = C;
    s.kc = kc;
    s.carry_val = carry_val;
    const bool vec = kc == 4 && (reinterpret_cast<uintptr_t>(B) & 15u) == 0 && (reinterpret_cast<uintptr_t>(C) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(carry_val) & 15u) == 0;
    switch (vdt) {
        case LB_F32:
            return vec ? launch_spmm_warp_t<float, true>(s, st) : launch_spmm_warp_t<float, false>(s, st);
        case LB_BF16:
            return vec ? launch_spmm_warp_t<__nv_bfloat16, true>(s, st) : launch_spmm_warp_t<__nv_bfloat16, false>(s, st);
        case LB_F16:
            return vec ? launch_spmm_warp_t<__half, true>(s, st) : launch_spmm_warp_t<__half, false>(s, st);
    }
    return cudaErrorInvalidValue;
}

template <typename V>
static cudaError_t launch_spmm_wide_t(const SpmmArgs &s, cudaStream_t st) {
    auto kern = spmm_wide_kernel<V>;
    constexpr int threads = kWideThreads;
    const size_t smem = static_cast<size_t>(threads / 32) * 32 * kIpt * sizeof(int);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    long long grid = static_cast<long long>(per_sm > 0 ? per_sm : 1) * current_sm_count();
    const long long need = (static_cast<long long>(s.t.num_tiles) + threads / 32 - 1) / (threads / 32);
    if (grid > need) grid = need;
    kern<<<static_cast<int>(grid), threads, smem, st>>>(s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    long long fb = (static_cast<long long>(s.t.num_tiles) + 7) / 8;
    const long long cap = static_cast<long long>(current_sm_count()) * 8;
    if (fb > cap) fb = cap;
    spmm_fixup_kernel<<<static_cast<int>(fb), 256, 0, st>>>(s.t.num_tiles, s.t.num_rows, s.kc, s.t.carry_row,
                                                           s.carry_val, s.C);
    return cudaGetLastError();
}

bool spmm_wide_ok(int kc, const float *B, const float *C) {
    return (kc == 8 || kc == 16) && (reinterpret_cast<uintptr_t>(B) & 31u) == 0 &&
           (reinterpret_cast<uintptr_t>(C) & 31u) == 0;
}

cudaError_t launch_spmm_wide(lb_dtype vdt, int G, int m, int n, int nnz, int kc, const int *tile_row,
                             const int *tile_nz, const int *row_end, const int *ci, const void *values, const float *B,
                             float *C, int *carry_row, float *carry_val, int *err, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    if (!spmm_wide_ok(kc, B, C) || (reinterpret_cast<uintptr_t>(carry_val) & 31u) != 0) return cudaErrorInvalidValue;
    SpmmArgs s{};
    s.t.num_tiles = G;
    s.t.num_rows = m;
    s.t.num_atoms = nnz;
    s.t.tile_row = tile_row;
    s.t.tile_nz = tile_nz;
    s.t.row_end = row_end;
    s.t.idx = ci;
    s.t.val = values;
    s.t.x_len = n;
    s.t.carry_row = carry_row;
    s.t.err = err;
    set_merge_alignment(s.t, vdt == LB_F32 ? 4 : 2);
    s.B = B;
    s.C = C;
    s.kc = kc;
    s.carry_val = carry_val;
    switch (vdt) {
        case LB_F32:
            return launch_spmm_wide_t<float>(s, st);
        case LB_BF16:
            return launch_spmm_wide_t<__nv_bfloat16>(s, st);
        case LB_F16:
            return launch_spmm_wide_t<__half>(s, st);
    }
    return cudaErrorInvalidValue;
}

template <typename V, int TMAX, bool VEC>
static cudaError_t launch_spmm_block_t(int G, int m, int n, int kc, const int *tile_row, const int *tile_nz, const int *row_end,
                                 const int *ci, const V *values, const float *B, float *C, int *carry_row,
                                 float *carry_val, cudaStream_t st) {
    constexpr int THREADS = 256;
    const int kq = (kc + 3) / 4;
    int nq = 1;
    while (nq < kq && nq < 32) nq <<= 1;  // up to 32 quads (128 columns) per pass
    auto kern = spmm_block_kernel<V, THREADS, TMAX, VEC>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0);
    if (e != cudaSuccess) return e;
    long long grid = static_cast<long long>(per_sm > 0 ? per_sm : 1) * current_sm_count();
    if (grid > G) grid = G;
    kern<<<static_cast<int>(grid), THREADS, 0, st>>>(G, m, n, kc, nq, tile_row, tile_nz, row_end, ci, values, B, C,
                                                     carry_row, carry_val);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    long long fb = (static_cast<long long>(G) + 7) / 8;
    const long long cap = static_cast<long long>(current_sm_count()) * 8;
    if (fb > cap) fb = cap;
    spmm_fixup_kernel<<<static_cast<int>(fb), 256, 0, st>>>(G, m, kc, carry_row, carry_val, C);
    return cudaGetLastError();
}

template <typename V>
static cudaError_t launch_spmm_block_v(int G, int m, int n, int kc, int tile_items, const int *tile_row, const int *tile_nz,
                                 const int *row_end, const int *ci, const void *values, const float *B, float *C,
                                 int *carry_row, float *carry_val, cudaStream_t st) {
    const V *v = static_cast<const V *>(values);
    const bool vec = kc % 4 == 0 && (reinterpret_cast<uintptr_t>(B) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(C) & 15u) == 0;
    if (tile_items > 2048) return cudaErrorInvalidValue;  // shared-memory staging holds 2048 items
    return vec ? launch_spmm_block_t<V, 2048, true>(G, m, n, kc, tile_row, tile_nz, row_end, ci, v, B, C, carry_row, carry_val,
                                              st)
               : launch_spmm_block_t<V, 2048, false>(G, m, n, kc, tile_row, tile_nz, row_end, ci, v, B, C, carry_row,
                                               carry_val, st);
}

cudaError_t launch_spmm_block(lb_dtype vdt, int G, int m, int n, int kc, int tile_items, const int *tile_row,
                              const int *tile_nz, const int *row_end, const int *ci, const void *values,
                              const float *B, float *C, int *carry_row, float *carry_val, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    switch (vdt) {
        case LB_F32:
            return launch_spmm_block_v<float>(G, m, n, kc, tile_items, tile_row, tile_nz, row_end, ci, values, B, C,
                                              carry_row, carry_val, st);
        case LB_BF16:
            return launch_spmm_block_v<__nv_bfloat16>(G, m, n, kc, tile_items, tile_row, tile_nz, row_end, ci, values,
                                                      B, C, carry_row, carry_val, st);
        case LB_F16:
            return launch_spmm_block_v<__half>(G, m, n, kc, tile_items, tile_row, tile_nz, row_end, ci, values, B, C,
                                               carry_row, carry_val, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lb
