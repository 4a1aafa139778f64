// lb_backward.cu -- the per-nonzero passes over the forward merge-path partition: row ids of
// the nonzeros (for the transpose), dvalues gathering x, and the CSR-order backward pass
// (dvalues from saved gathers, the scaled values for dx in CSC buckets, or their float
// reductions into dx).
#include <cstdint>

#include "lb_internal.cuh"

namespace lb {

// ------------------------------------------------------------------------------------------
// Per-nonzero maps over the forward merge-path partition.  Each tile stages its row ends;
// each thread finds the row of its first nonzero by one binary search and walks forward over
// its IPT consecutive nonzeros (row ends are sorted), recording row ids in shared memory;
// a second, coalesced pass reads the column indices and writes the outputs.

template <int THREADS, int IPT, bool ROWID>
__global__ void __launch_bounds__(THREADS) tile_rows_kernel(int G, const int *__restrict__ tile_row,
                                                            const int *__restrict__ tile_nz,
                                                            const int *__restrict__ row_end,
                                                            const int *__restrict__ ci, const float *__restrict__ g,
                                                            const float *__restrict__ x, float *__restrict__ dv,
                                                            int *__restrict__ rowid) {
    constexpr int T = THREADS * IPT;
    __shared__ int s_re[T];
    __shared__ int s_row[T];
    for (int tile = blockIdx.x; tile < G; tile += gridDim.x) {
        const int r0 = __ldg(tile_row + tile), r1 = __ldg(tile_row + tile + 1);
        const int k0 = __ldg(tile_nz + tile), k1 = __ldg(tile_nz + tile + 1);
        const int nr = r1 - r0, nk = k1 - k0;
        if (nr < 0 || nk < 0 || nr > T || nk > T) continue;  // malformed offsets (block-uniform)
        for (int r = threadIdx.x; r < nr; r += THREADS) s_re[r] = __ldg(row_end + r0 + r) - k0;
        __syncthreads();
        const int base = threadIdx.x * IPT;
        if (base < nk) {
            int lo = 0, hi = nr;  // rows of the tile ending at or before `base`
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_re[mid] <= base)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            int i = lo;
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const int j = base + q;
                if (j < nk) {
                    while (i < nr && s_re[i] <= j) ++i;
                    s_row[j] = i;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < IPT; ++u) {
            const int j = threadIdx.x + u * THREADS;
            if (j < nk) {
                const int k = k0 + j;
                const int row = r0 + s_row[j];
                if (ROWID)
                    rowid[k] = row;
                else
                    dv[k] = __ldg(g + row) * __ldg(x + __ldg(ci + k));
            }
        }
        __syncthreads();
    }
}

template <bool ROWID>
static cudaError_t launch_tile_rows(int G, int tile_items, const int *tile_row, const int *tile_nz,
                                    const int *row_end, const int *ci, const float *g, const float *x, float *dv,
                                    int *rowid, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    int grid = G;
    const int cap = current_sm_count() * 6;
    if (grid > cap) grid = cap;
    // The staged row ends must fit: a tile holds at most tile_items rows.
    if (tile_items <= 1024)
        tile_rows_kernel<256, 4, ROWID><<<grid, 256, 0, st>>>(G, tile_row, tile_nz, row_end, ci, g, x, dv, rowid);
    else if (tile_items <= 2048)
        tile_rows_kernel<256, 8, ROWID><<<grid, 256, 0, st>>>(G, tile_row, tile_nz, row_end, ci, g, x, dv, rowid);
    else if (tile_items <= 4096)
        tile_rows_kernel<256, 16, ROWID><<<grid, 256, 0, st>>>(G, tile_row, tile_nz, row_end, ci, g, x, dv, rowid);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// One streaming pass over the nonzeros in CSR order, tile by tile over the forward partition:
//   pv[pos(k)] = values[k] * g[row(k)]   (pos = bucket_pos, or the identity), when pv is given;
//   dv[k]      = g[row(k)] * xg[k]        (the values gradient from saved gathers), when dv is.
// The rows come without any search: every row end inside the tile adds 1 to a per-slot count
// in shared memory, and a slot's row is the inclusive prefix sum of the counts (each thread
// sums its IPT slots, the block scans the thread totals).  Slot 0 of a tile sits 16 bytes
// aligned in the nonzero arrays (the tile's first nonzero at slot `lead`), so each thread
// moves its IPT consecutive entries with vector loads and stores where the arrays allow.  The
// scaled values go to shared memory and out in a second, lane-consecutive pass, so that the
// scattered bucket positions of neighbouring nonzeros coalesce as well as they can.
template <typename V, int IPT>
__device__ __forceinline__ void load_values(const V *src, bool vec, bool full, int j0, int nk, float (&o)[IPT]) {
    if (full && vec) {
        if constexpr (sizeof(V) == 4) {
#pragma unroll
            for (int q = 0; q < IPT; q += 4) {
                const float4 t = __ldcs(reinterpret_cast<const float4 *>(src + q));
                o[q] = t.x;
                o[q + 1] = t.y;
                o[q + 2] = t.z;
                o[q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < IPT; q += 4) {
                const uint2 t = __ldcs(reinterpret_cast<const uint2 *>(src + q));
                const uint32_t w[2] = {t.x, t.y};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    V lo, hi;
                    const unsigned short bl = static_cast<unsigned short>(w[e] & 0xffffu);
                    const unsigned short bh = static_cast<unsigned short>(w[e] >> 16);
                    memcpy(&lo, &bl, 2);
                    memcpy(&hi, &bh, 2);
                    o[q + 2 * e] = to_f32(lo);
                    o[q + 2 * e + 1] = to_f32(hi);
                }
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < IPT; ++q) o[q] = (j0 + q >= 0 && j0 + q < nk) ? to_f32(src[q]) : 0.f;
    }
}

template <int IPT>
__device__ __forceinline__ void load_ints(const int *src, bool vec, bool full, int j0, int nk, int (&o)[IPT]) {
    if (full && vec) {
#pragma unroll
        for (int q = 0; q < IPT; q += 4) {
            const int4 t = __ldcs(reinterpret_cast<const int4 *>(src + q));
            o[q] = t.x;
            o[q + 1] = t.y;
            o[q + 2] = t.z;
            o[q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < IPT; ++q) o[q] = (j0 + q >= 0 && j0 + q < nk) ? __ldcs(src + q) : 0;
    }
}

// SCATTER: instead of the bucketed scaled values, add each v[k] * g[row(k)] into dx[col(k)]
// with a float reduction in L2 (dx must start at zero).  No CSC view is needed; the sums of a
// column then arrive in no fixed order, so dx is not bit-reproducible (it stays within the
// FP32 tolerance of the transposed product).
template <typename V, int THREADS, int IPT, bool SCATTER>
__global__ void __launch_bounds__(THREADS) csr_backward_kernel(int G, int m, const int *__restrict__ tile_row,
                                                               const int *__restrict__ tile_nz,
                                                               const int *__restrict__ row_end,
                                                               const float *__restrict__ g,
                                                               const V *__restrict__ values,
                                                               const int *__restrict__ bucket_pos,
                                                               float *__restrict__ pv, const float *__restrict__ xg,
                                                               float *__restrict__ dv, const int *__restrict__ ci,
                                                               float *__restrict__ dx_acc) {
    constexpr int T = THREADS * IPT;
    constexpr int WARPS = THREADS / 32;
    static_assert(IPT % 4 == 0, "slots move four at a time");
    __shared__ __align__(16) int cnt[T];
    __shared__ __align__(16) float s_pv[T];
    __shared__ int wsum[WARPS];
    for (int i = threadIdx.x; i < T; i += THREADS) cnt[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool want_pv = !SCATTER && pv != nullptr, want_dv = dv != nullptr;
    const bool vec_ci = (reinterpret_cast<uintptr_t>(ci) & 15u) == 0;
    // Slot 0 of every tile is 16-byte aligned in an array whose base is (4-byte elements) or
    // 8-byte aligned (2-byte values, moved four at a time).
    const bool vec_xg = (reinterpret_cast<uintptr_t>(xg) & 15u) == 0;
    const bool vec_dv = (reinterpret_cast<uintptr_t>(dv) & 15u) == 0;
    const bool vec_v = (reinterpret_cast<uintptr_t>(values) & (sizeof(V) == 4 ? 15u : 7u)) == 0;
    for (int tile = blockIdx.x; tile < G; tile += gridDim.x) {
        const int r0 = __ldg(tile_row + tile), r1 = __ldg(tile_row + tile + 1);
        const int k0 = __ldg(tile_nz + tile), k1 = __ldg(tile_nz + tile + 1);
        const int nr = r1 - r0, nk = k1 - k0;
        const int lead = k0 & 3;  // nonzero k0 - lead is a multiple of 4
        if (nr < 0 || nk < 0 || nk + lead > T) continue;  // malformed offsets (block-uniform)
        const int s0 = threadIdx.x * IPT;
        const int j0 = s0 - lead;  // tile item of this thread's first slot
        const bool mine = j0 + IPT > 0 && j0 < nk;
        const bool full = j0 >= 0 && j0 + IPT <= nk;
        // Every load that does not depend on the rows goes out first, so its latency overlaps
        // the row-end staging and the scan: this thread's values and saved gathers (blocked)
        // and the bucket positions of the lane-consecutive scatter.
        float vv[IPT], xv[IPT];
        int bp[IPT], cc[IPT];
        if ((want_pv || SCATTER) && mine) load_values<V, IPT>(values + k0 + j0, vec_v, full, j0, nk, vv);
        if (want_dv && mine) load_values<float, IPT>(xg + k0 + j0, vec_xg, full, j0, nk, xv);
        if (SCATTER && mine) load_ints<IPT>(ci + k0 + j0, vec_ci, full, j0, nk, cc);
        if (want_pv) {
#pragma unroll
            for (int u = 0; u < IPT; ++u) {
                const int j = threadIdx.x + u * THREADS;
                bp[u] = j < nk ? (bucket_pos != nullptr ? __ldcs(bucket_pos + k0 + j) : k0 + j) : 0;
            }
        }
        for (int r = threadIdx.x; r < nr; r += THREADS) {
            const int e = __ldg(row_end + r0 + r) - k0;  // first nonzero of the next row, tile-local
            if (e >= 0 && e < nk) atomicAdd(&cnt[e + lead], 1);
        }
        __syncthreads();
        int c[IPT];
#pragma unroll
        for (int q = 0; q < IPT; q += 4) {
            const int4 t = *reinterpret_cast<const int4 *>(cnt + s0 + q);
            c[q] = t.x;
            c[q + 1] = t.y;
            c[q + 2] = t.z;
            c[q + 3] = t.w;
            *reinterpret_cast<int4 *>(cnt + s0 + q) = make_int4(0, 0, 0, 0);  // ready for the next tile
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
        if (mine) {
            float gq[IPT];
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const int row = r0 + base + c[q];
                gq[q] = (j0 + q >= 0 && j0 + q < nk && row < m) ? __ldg(g + row) : 0.f;
            }
            if (SCATTER) {
#pragma unroll
                for (int q = 0; q < IPT; ++q)
                    if (j0 + q >= 0 && j0 + q < nk) atomicAdd(dx_acc + cc[q], vv[q] * gq[q]);
            }
            if (want_pv) {
#pragma unroll
                for (int q = 0; q < IPT; q += 4)
                    *reinterpret_cast<float4 *>(s_pv + s0 + q) =
                        make_float4(vv[q] * gq[q], vv[q + 1] * gq[q + 1], vv[q + 2] * gq[q + 2], vv[q + 3] * gq[q + 3]);
            }
            if (want_dv) {
                float *dst = dv + k0 + j0;
                if (full && vec_dv) {
#pragma unroll
                    for (int q = 0; q < IPT; q += 4)
                        __stcs(reinterpret_cast<float4 *>(dst + q),
                               make_float4(gq[q] * xv[q], gq[q + 1] * xv[q + 1], gq[q + 2] * xv[q + 2],
                                           gq[q + 3] * xv[q + 3]));
                } else {
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
                        if (j0 + q >= 0 && j0 + q < nk) __stcs(dst + q, gq[q] * xv[q]);
                }
            }
        }
        if (want_pv) {
            __syncthreads();
#pragma unroll
            for (int u = 0; u < IPT; ++u) {
                const int j = threadIdx.x + u * THREADS;
                if (j < nk) pv[bp[u]] = s_pv[j + lead];
            }
        }
        __syncthreads();  // the counts, wsum and s_pv are reused by the next tile
    }
}

template <typename V, bool SCATTER>
static cudaError_t launch_csr_backward_t(int num_tiles, int m, int tile_items, const int *tile_row, const int *tile_nz,
                                         const int *row_end, const float *g, const V *values, const int *bucket_pos,
                                         float *pv, const float *xg, float *dv, const int *ci, float *dx_acc,
                                         cudaStream_t stream) {
    // One wave of resident CTAs (the kernel loops over tiles).  A tile's slots: its items plus
    // a lead of up to 3 must fit.
    auto launch = [&](auto kern, int threads) -> cudaError_t {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
        if (e != cudaSuccess) return e;
        long long grid = static_cast<long long>(per_sm > 0 ? per_sm : 1) * current_sm_count();
        if (grid > num_tiles) grid = num_tiles;
        kern<<<static_cast<int>(grid), threads, 0, stream>>>(num_tiles, m, tile_row, tile_nz, row_end, g, values,
                                                             bucket_pos, pv, xg, dv, ci, dx_acc);
        return cudaGetLastError();
    };
    if (tile_items + 3 <= 2048) return launch(csr_backward_kernel<V, 256, 8, SCATTER>, 256);
    if (tile_items + 3 <= 4096) return launch(csr_backward_kernel<V, 512, 8, SCATTER>, 512);
    return cudaErrorInvalidValue;
}

cudaError_t launch_csr_backward(lb_dtype vdt, int num_tiles, int m, int tile_items, const int *tile_row,
                                const int *tile_nz, const int *row_end, const float *g, const void *values,
                                const int *bucket_pos, float *pv, const float *xg, float *dv, cudaStream_t stream) {
    if (num_tiles <= 0) return cudaSuccess;
    if ((pv != nullptr && values == nullptr) || (dv != nullptr && xg == nullptr)) return cudaErrorInvalidValue;
    switch (vdt) {
        case LB_F32:
            return launch_csr_backward_t<float, false>(num_tiles, m, tile_items, tile_row, tile_nz, row_end, g,
                                                       static_cast<const float *>(values), bucket_pos, pv, xg, dv,
                                                       nullptr, nullptr, stream);
        case LB_BF16:
            return launch_csr_backward_t<__nv_bfloat16, false>(num_tiles, m, tile_items, tile_row, tile_nz, row_end, g,
                                                               static_cast<const __nv_bfloat16 *>(values), bucket_pos,
                                                               pv, xg, dv, nullptr, nullptr, stream);
        case LB_F16:
            return launch_csr_backward_t<__half, false>(num_tiles, m, tile_items, tile_row, tile_nz, row_end, g,
                                                        static_cast<const __half *>(values), bucket_pos, pv, xg, dv,
                                                        nullptr, nullptr, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_csr_backward_scatter(lb_dtype vdt, int num_tiles, int m, int tile_items, const int *tile_row,
                                        const int *tile_nz, const int *row_end, const float *g, const void *values,
                                        const int *ci, float *dx, const float *xg, float *dv, cudaStream_t stream) {
    if (num_tiles <= 0) return cudaSuccess;
    if (values == nullptr || ci == nullptr || dx == nullptr || (dv != nullptr && xg == nullptr))
        return cudaErrorInvalidValue;
    switch (vdt) {
        case LB_F32:
            return launch_csr_backward_t<float, true>(num_tiles, m, tile_items, tile_row, tile_nz, row_end, g,
                                                      static_cast<const float *>(values), nullptr, nullptr, xg, dv, ci,
                                                      dx, stream);
        case LB_BF16:
            return launch_csr_backward_t<__nv_bfloat16, true>(num_tiles, m, tile_items, tile_row, tile_nz, row_end, g,
                                                              static_cast<const __nv_bfloat16 *>(values), nullptr,
                                                              nullptr, xg, dv, ci, dx, stream);
        case LB_F16:
            return launch_csr_backward_t<__half, true>(num_tiles, m, tile_items, tile_row, tile_nz, row_end, g,
                                                       static_cast<const __half *>(values), nullptr, nullptr, xg, dv,
                                                       ci, dx, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_dvalues(int num_tiles, int m, int tile_items, const int *tile_row, const int *tile_nz,
                           const int *row_end, const int *ci, const float *g, const float *x, const float *xg,
                           float *dv, cudaStream_t stream) {
    if (xg == nullptr)
        return launch_tile_rows<false>(num_tiles, tile_items, tile_row, tile_nz, row_end, ci, g, x, dv, nullptr,
                                       stream);
    return launch_csr_backward(LB_F32, num_tiles, m, tile_items, tile_row, tile_nz, row_end, g, nullptr, nullptr,
                               nullptr, xg, dv, stream);
}

cudaError_t launch_tile_row_ids(int num_tiles, int tile_items, const int *tile_row, const int *tile_nz,
                                const int *row_end, int *rowid, cudaStream_t stream) {
    return launch_tile_rows<true>(num_tiles, tile_items, tile_row, tile_nz, row_end, nullptr, nullptr, nullptr,
                                  nullptr, rowid, stream);
}

}  // namespace lb
