// lb_backward.cu -- the per-nonzero passes over the forward merge-path partition: row ids of
// the nonzeros (for the transpose), dvalues gathering x, and the CSR-order backward pass
// (dvalues from saved gathers, the scaled values for dx in CSC buckets, or their float
// reductions into dx).
#include <cstdint>
#include <type_traits>

#include "lb_warp.cuh"

namespace lb {

// A gradient value in the values' 16-bit type (round to nearest even), as its bits.
template <typename T>
__device__ __forceinline__ uint32_t narrow_bits(float v) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value)
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    else
        return __half_as_ushort(__float2half_rn(v));
}

// Store one gradient value as T (FP32, or 16-bit rounded to nearest even).
template <typename T>
__device__ __forceinline__ void store_grad(void *base, long long k, float v) {
    if constexpr (std::is_same<T, float>::value)
        static_cast<float *>(base)[k] = v;
    else
        static_cast<unsigned short *>(base)[k] = static_cast<unsigned short>(narrow_bits<T>(v));
}

// ------------------------------------------------------------------------------------------
// Per-nonzero maps over the forward merge-path partition.  Each tile stages its row ends;
// each thread finds the row of its first nonzero by one binary search and walks forward over
// its IPT consecutive nonzeros (row ends are sorted), recording row ids in shared memory;
// a second, coalesced pass reads the column indices and writes the outputs.

template <int THREADS, int IPT, bool ROWID, typename DVT = float>
__global__ void __launch_bounds__(THREADS) tile_rows_kernel(int G, const int *__restrict__ tile_row,
                                                            const int *__restrict__ tile_nz,
                                                            const int *__restrict__ row_end,
                                                            const int *__restrict__ ci, const float *__restrict__ g,
                                                            const float *__restrict__ x, int n,
                                                            void *__restrict__ dv, int *__restrict__ rowid) {
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
                else {
                    const int c = __ldg(ci + k);
                    store_grad<DVT>(dv, k, LB_IN_RANGE(c, n) ? __ldg(g + row) * __ldg(x + c) : 0.f);
                }
            }
        }
        __syncthreads();
    }
}

template <bool ROWID, typename DVT = float>
static cudaError_t launch_tile_rows(int G, int tile_items, const int *tile_row, const int *tile_nz,
                                    const int *row_end, const int *ci, const float *g, const float *x, int n,
                                    void *dv, int *rowid, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    int grid = G;
    const int cap = current_sm_count() * 6;
    if (grid > cap) grid = cap;
    // The staged row ends must fit: a tile holds at most tile_items rows.
    if (tile_items <= 1024)
        tile_rows_kernel<256, 4, ROWID, DVT><<<grid, 256, 0, st>>>(G, tile_row, tile_nz, row_end, ci, g, x, n, dv, rowid);
    else if (tile_items <= 2048)
        tile_rows_kernel<256, 8, ROWID, DVT><<<grid, 256, 0, st>>>(G, tile_row, tile_nz, row_end, ci, g, x, n, dv, rowid);
    else if (tile_items <= 4096)
        tile_rows_kernel<256, 16, ROWID, DVT><<<grid, 256, 0, st>>>(G, tile_row, tile_nz, row_end, ci, g, x, n, dv, rowid);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// One streaming pass over the nonzeros in CSR order, warp tile by warp tile over the forward
// merge-path partition (every warp independent, no block-wide barrier):
//   pv[pos(k)] = values[k] * g[row(k)]   (pos = bucket_pos, or the identity), when pv is given;
//   dv[k]      = g[row(k)] * xg[k]        (the values gradient from saved gathers), when dv is;
//   dx[ci[k]] += values[k] * g[row(k)]    (float reductions, SCATTER only).
// Lane l owns the tile's slots [8 l, 8 l + 8); slot 0 sits 32 bytes aligned in the nonzero
// arrays (the tile's first nonzero at slot lead = k0 mod 8), so every lane moves its eight
// values, saved gathers and dvalues with one 256-bit (values: 128-bit when 16-bit) access.
// The rows come without a search: each row end inside the tile adds 1 to a per-slot count
// in the warp's shared memory, and a slot's row is r0 plus the inclusive prefix sum of the
// counts (in the lane, then across lanes by shuffles).  The scaled values leave through the
// warp's shared memory in a lane-consecutive pass, so that the bucket positions of
// neighbouring nonzeros (consecutive inside a bucket) coalesce.
struct CsrBackwardArgs {
    int G, m, nnz, n;  // n: columns (dx entries), checked against in the range-checked build
    const int *tile_row, *tile_nz, *row_end;
    const float *g;
    const void *values;
    const int *bucket_pos;  // null: pv in CSR order
    float *pv;              // null: no scaled values
    const float *xg;        // saved gathers (with dv)
    void *dv;               // null: no values gradient; FP32, or the values' type when dv_narrow
    int dv_narrow;          // dv holds the values' 16-bit type (rounded to nearest even)
    const int *ci;          // SCATTER: column indices
    float *dx;              // SCATTER: dx accumulated by float reductions
    int vec_v, vec_xg, vec_dv, vec_ci;  // the arrays' bases are 32-byte (16-bit values: 16-byte) aligned
};

// Per warp: per-slot row-end counts, then the padded buffer of scaled values.
template <int IPT>
__host__ __device__ constexpr int csr_warp_bytes() {
    return WarpTile<IPT>::SLOTS * 4 + WarpTile<IPT>::VALS * 4;
}

template <typename V, int IPT, bool SCATTER>
__global__ void __launch_bounds__(256) csr_backward_kernel(const CsrBackwardArgs a) {
    constexpr int SLOTS = WarpTile<IPT>::SLOTS;
    constexpr int WB = csr_warp_bytes<IPT>();
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int *cnt = reinterpret_cast<int *>(smem + wib * WB);
    float *buf = reinterpret_cast<float *>(smem + wib * WB + SLOTS * 4);
    const int nw = static_cast<int>(gridDim.x) * (blockDim.x >> 5);
    int t = static_cast<int>(blockIdx.x) * (blockDim.x >> 5) + wib;
    if (t >= a.G) return;
#pragma unroll
    for (int q = 0; q < IPT; q += 4) *reinterpret_cast<int4 *>(cnt + IPT * lane + q) = make_int4(0, 0, 0, 0);
    __syncwarp();
    const uint64_t pol = policy_evict_first();
    const bool want_pv = !SCATTER && a.pv != nullptr, want_dv = a.dv != nullptr;
    int bw = lane < 2 ? __ldg(a.tile_row + t + lane) : (lane < 4 ? __ldg(a.tile_nz + t + lane - 2) : 0);
    for (; t < a.G; t += nw) {
        const int r0 = __shfl_sync(0xffffffffu, bw, 0), r1 = __shfl_sync(0xffffffffu, bw, 1);
        const int k0 = __shfl_sync(0xffffffffu, bw, 2), k1 = __shfl_sync(0xffffffffu, bw, 3);
        if (t + nw < a.G)
            bw = lane < 2 ? __ldg(a.tile_row + t + nw + lane) : (lane < 4 ? __ldg(a.tile_nz + t + nw + lane - 2) : 0);
        const int nr = r1 - r0, nk = k1 - k0;
        if (r0 < 0 || nr < 0 || r1 > a.m || k0 < 0 || nk < 0 || k1 > a.nnz || nr + nk > WarpTile<IPT>::ITEMS)
            continue;  // malformed offsets (warp-uniform): nothing is read or written
        const int lead = k0 & 7;
        const int kb = k0 - lead;
        const int e0 = kb + IPT * lane;
        const uint32_t vm = slot_mask<IPT>(e0, k0, k1);
        const bool inb = e0 >= 0 && e0 + IPT <= a.nnz;  // the lane's eight elements exist
        // Every load that does not depend on the rows goes out first.
        float vv[IPT], xv[IPT];
        int cc[IPT], bp[IPT];
#pragma unroll
        for (int q = 0; q < IPT; ++q) vv[q] = xv[q] = 0.f, cc[q] = bp[q] = 0;
        if ((want_pv || SCATTER) && vm) {
            if (sizeof(V) == 4) {
                const float *v = static_cast<const float *>(a.values);
                if (a.vec_v && inb) {
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
                const unsigned short *v = static_cast<const unsigned short *>(a.values);
                if (a.vec_v && inb) {
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
        if (want_dv && vm) {
            if (a.vec_xg && inb) {
#pragma unroll
                for (int h = 0; h < IPT; h += 8) {
                    uint32_t r[8];
                    ld_stream8(a.xg + e0 + h, pol, r);
#pragma unroll
                    for (int q = 0; q < 8; ++q) xv[h + q] = __uint_as_float(r[q]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < IPT; ++q)
                    if ((vm >> q) & 1u) xv[q] = __ldg(a.xg + e0 + q);
            }
        }
        if (SCATTER && vm) {
            if (a.vec_ci && inb) {
#pragma unroll
                for (int h = 0; h < IPT; h += 8) {
                    uint32_t r[8];
                    ld_stream8(a.ci + e0 + h, pol, r);
#pragma unroll
                    for (int q = 0; q < 8; ++q) cc[h + q] = static_cast<int>(r[q]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < IPT; ++q)
                    if ((vm >> q) & 1u) cc[q] = __ldg(a.ci + e0 + q);
            }
        }
        if (want_pv) {  // lane-consecutive: slot j = 32 q + lane
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const int j = 32 * q + lane;
                if (j >= lead && j < lead + nk)
                    bp[q] = a.bucket_pos != nullptr ? __ldcs(a.bucket_pos + kb + j) : kb + j;
            }
        }
        // Rows: each row end inside the tile counts at the slot of the next row's first nonzero.
        for (int j = 0; j < nr; j += 32) {
            if (j + lane < nr) {
                const int e = __ldg(a.row_end + r0 + j + lane);
                if (e >= k0 && e < k1) atomicAdd(cnt + (e - kb), 1);
            }
        }
        __syncwarp();
        int c[IPT];
#pragma unroll
        for (int q = 0; q < IPT; q += 4) {
            const int4 cq = *reinterpret_cast<const int4 *>(cnt + IPT * lane + q);
            *reinterpret_cast<int4 *>(cnt + IPT * lane + q) = make_int4(0, 0, 0, 0);
            c[q] = cq.x, c[q + 1] = cq.y, c[q + 2] = cq.z, c[q + 3] = cq.w;
        }
#pragma unroll
        for (int q = 1; q < IPT; ++q) c[q] += c[q - 1];
        int incl = c[IPT - 1];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += u;
        }
        const int base = r0 + incl - c[IPT - 1];
        float gq[IPT];
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int row = base + c[q];
            gq[q] = (((vm >> q) & 1u) && row < a.m) ? __ldg(a.g + row) : 0.f;
        }
        if (want_dv && vm) {
            float d[IPT];
#pragma unroll
            for (int q = 0; q < IPT; ++q) d[q] = gq[q] * xv[q];
            if (sizeof(V) == 2 && a.dv_narrow) {  // the values' type: 16 bytes per lane
                unsigned short *dvn = static_cast<unsigned short *>(a.dv);
                if (vm == (1u << IPT) - 1u && a.vec_dv) {
#pragma unroll
                    for (int h = 0; h < IPT; h += 8) {
                        uint32_t w[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            w[i] = narrow_bits<V>(d[h + 2 * i]) | (narrow_bits<V>(d[h + 2 * i + 1]) << 16);
                        asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.b32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(
                                         dvn + e0 + h),
                                     "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "l"(pol)
                                     : "memory");
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
                        if ((vm >> q) & 1u) dvn[e0 + q] = static_cast<unsigned short>(narrow_bits<V>(d[q]));
                }
            } else {
                float *dvf = static_cast<float *>(a.dv);
                if (vm == (1u << IPT) - 1u && a.vec_dv) {
#pragma unroll
                    for (int h = 0; h < IPT; h += 8) st_stream8(dvf + e0 + h, pol, d + h);
                } else {
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
                        if ((vm >> q) & 1u) __stcs(dvf + e0 + q, d[q]);
                }
            }
        }
        if (SCATTER) {
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                if (((vm >> q) & 1u) && LB_IN_RANGE(cc[q], a.n)) atomicAdd(a.dx + cc[q], vv[q] * gq[q]);
        }
        if (want_pv) {
#pragma unroll
            for (int q = 0; q < IPT; q += 4)
                *reinterpret_cast<float4 *>(buf + ppad(IPT * lane + q)) =
                    make_float4(vv[q] * gq[q], vv[q + 1] * gq[q + 1], vv[q + 2] * gq[q + 2], vv[q + 3] * gq[q + 3]);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const int j = 32 * q + lane;
                if (j >= lead && j < lead + nk && LB_IN_RANGE(bp[q], a.nnz)) a.pv[bp[q]] = buf[ppad(j)];
            }
        }
        __syncwarp();  // the counts and the buffer are reused by the next tile
    }
}

template <typename V, int IPT, bool SCATTER>
static cudaError_t launch_csr_backward_ipt(CsrBackwardArgs a, cudaStream_t stream) {
    // One wave of resident warps (each loops over its tiles).
    auto kern = csr_backward_kernel<V, IPT, SCATTER>;
    constexpr int threads = 256;
    const size_t smem = static_cast<size_t>(threads / 32) * csr_warp_bytes<IPT>();
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    long long grid = static_cast<long long>(per_sm > 0 ? per_sm : 1) * current_sm_count();
    const long long need = (static_cast<long long>(a.G) + threads / 32 - 1) / (threads / 32);
    if (grid > need) grid = need;
    const size_t vb = (sizeof(V) == 4) ? 31u : 15u;
    a.vec_v = (reinterpret_cast<uintptr_t>(a.values) & vb) == 0;
    a.vec_xg = (reinterpret_cast<uintptr_t>(a.xg) & 31u) == 0;
    a.vec_dv = (reinterpret_cast<uintptr_t>(a.dv) & (a.dv_narrow ? 15u : 31u)) == 0;
    a.vec_ci = (reinterpret_cast<uintptr_t>(a.ci) & 31u) == 0;
    kern<<<static_cast<int>(grid), threads, smem, stream>>>(a);
    return cudaGetLastError();
}

// The warp tiles' size picks the slots per lane: tiles of merge_tile_items(8) or (16) items.
template <typename V, bool SCATTER>
static cudaError_t launch_csr_backward_t(CsrBackwardArgs a, int tile_items, cudaStream_t stream) {
    if (tile_items <= merge_tile_items(8)) return launch_csr_backward_ipt<V, 8, SCATTER>(a, stream);
    if (tile_items <= merge_tile_items(16)) return launch_csr_backward_ipt<V, 16, SCATTER>(a, stream);
    return cudaErrorInvalidValue;
}

cudaError_t launch_csr_backward(lb_dtype vdt, int num_tiles, int tile_items, int m, int nnz, const int *tile_row,
                                const int *tile_nz, const int *row_end, const float *g, const void *values,
                                const int *bucket_pos, float *pv, const float *xg, void *dv, bool dv_narrow,
                                cudaStream_t stream) {
    if (num_tiles <= 0) return cudaSuccess;
    if ((pv != nullptr && values == nullptr) || (dv != nullptr && xg == nullptr)) return cudaErrorInvalidValue;
    if (dv_narrow && vdt == LB_F32) return cudaErrorInvalidValue;
    CsrBackwardArgs a{};
    a.G = num_tiles, a.m = m, a.nnz = nnz;
    a.tile_row = tile_row, a.tile_nz = tile_nz, a.row_end = row_end, a.g = g, a.values = values;
    a.bucket_pos = bucket_pos, a.pv = pv, a.xg = xg, a.dv = dv, a.dv_narrow = dv_narrow ? 1 : 0;
    switch (vdt) {
        case LB_F32:
            return launch_csr_backward_t<float, false>(a, tile_items, stream);
        case LB_BF16:
            return launch_csr_backward_t<__nv_bfloat16, false>(a, tile_items, stream);
        case LB_F16:
            return launch_csr_backward_t<__half, false>(a, tile_items, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_csr_backward_scatter(lb_dtype vdt, int num_tiles, int tile_items, int m, int n, int nnz,
                                        const int *tile_row,
                                        const int *tile_nz, const int *row_end, const float *g, const void *values,
                                        const int *ci, float *dx, const float *xg, void *dv, bool dv_narrow,
                                        cudaStream_t stream) {
    if (num_tiles <= 0) return cudaSuccess;
    if (values == nullptr || ci == nullptr || dx == nullptr || (dv != nullptr && xg == nullptr))
        return cudaErrorInvalidValue;
    if (dv_narrow && vdt == LB_F32) return cudaErrorInvalidValue;
    CsrBackwardArgs a{};
    a.G = num_tiles, a.m = m, a.nnz = nnz;
    a.tile_row = tile_row, a.tile_nz = tile_nz, a.row_end = row_end, a.g = g, a.values = values;
    a.xg = xg, a.dv = dv, a.dv_narrow = dv_narrow ? 1 : 0, a.ci = ci, a.dx = dx, a.n = n;
    switch (vdt) {
        case LB_F32:
            return launch_csr_backward_t<float, true>(a, tile_items, stream);
        case LB_BF16:
            return launch_csr_backward_t<__nv_bfloat16, true>(a, tile_items, stream);
        case LB_F16:
            return launch_csr_backward_t<__half, true>(a, tile_items, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_dvalues(int num_tiles, int tile_items, const int *tile_row, const int *tile_nz,
                           const int *row_end, const int *ci, const float *g, const float *x, int n, void *dv,
                           lb_dtype dvdt, cudaStream_t stream) {
    switch (dvdt) {
        case LB_F32:
            return launch_tile_rows<false, float>(num_tiles, tile_items, tile_row, tile_nz, row_end, ci, g, x, n, dv,
                                                  nullptr, stream);
        case LB_BF16:
            return launch_tile_rows<false, __nv_bfloat16>(num_tiles, tile_items, tile_row, tile_nz, row_end, ci, g, x, n,
                                                          dv, nullptr, stream);
        case LB_F16:
            return launch_tile_rows<false, __half>(num_tiles, tile_items, tile_row, tile_nz, row_end, ci, g, x, n, dv,
                                                   nullptr, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_tile_row_ids(int num_tiles, int tile_items, const int *tile_row, const int *tile_nz,
                                const int *row_end, int *rowid, cudaStream_t stream) {
    return launch_tile_rows<true>(num_tiles, tile_items, tile_row, tile_nz, row_end, nullptr, nullptr, nullptr, 0,
                                  nullptr, rowid, stream);
}

}  // namespace lb
