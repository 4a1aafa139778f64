// lb_spmm.cu -- load-balanced SpMM, C = A B with B dense (n x kc, row-major), over the
// merge-path partition of A.
//
// The dissertation's SpMM is its SpMV with one more loop, over the columns of B (Ch.4 Sec.
// "Application Space", the SpMM listing); the schedules and their work split carry over
// unchanged.  Here the tiles are the forward merge-path tiles of the plan (rows + nonzeros in
// equal shares), the row left open at the end of a tile goes out as a carry of kc values, and
// a fixup adds the carries of each row in tile order, exactly as for SpMV.
//
// GB300 realisation.  Where SpMV gathers one 4-byte x per nonzero, SpMM gathers a row of B:
// kc contiguous floats, read as 16-byte vectors, so every gather request carries four useful
// values instead of one.  Per tile:
//   1. the tile's column indices and values are staged in shared memory (coalesced), and each
//      nonzero's row comes from per-slot row-end counts and a block scan (no search);
//   2. threads are arranged as (column quad q, nonzero range g): thread (q, g) walks range g's
//      nonzeros in order, accumulating B[col][4q .. 4q+3] * value per row, and writes rows that
//      start and end inside its range straight to C;
//   3. the first and last partial row of every range go through shared memory; the range where
//      a row first appears sums its partials forward through the ranges it spans and writes
//      the row to C, or to the tile's carry when it is the row left open at the tile's end.
//      Rows without nonzeros in the tile that end there are written as zeros.
// Summation order is fixed (nonzero order within a tile, tile order in the fixup), so results
// are deterministic.
#include "lb_internal.cuh"

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

__device__ __forceinline__ void fma4(float4 &acc, float v, float4 b) {
    acc.x = fmaf(v, b.x, acc.x);
    acc.y = fmaf(v, b.y, acc.y);
    acc.z = fmaf(v, b.z, acc.z);
    acc.w = fmaf(v, b.w, acc.w);
}

__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

}  // namespace

// NQ column quads per pass (a power of two, <= THREADS); NG = THREADS / NQ nonzero ranges.
template <typename V, int THREADS, int TMAX, bool VEC>
__global__ void __launch_bounds__(THREADS) spmm_kernel(int G, int m, int n, int kc, int nq, const int *__restrict__ tile_row,
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

// Fixup: C[r][:] += the carries of row r, summed in tile order with compensated addition.  A
// warp per run of equal carry rows, lanes over the columns.
__global__ void spmm_fixup_kernel(int G, int m, int kc, const int *__restrict__ carry_row,
                                  const float *__restrict__ carry_val, float *__restrict__ C) {
    const int lane = threadIdx.x & 31;
    const long long warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
    for (long long c = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; c < G; c += warps) {
        const int r = __ldg(carry_row + c);
        if (r >= m) continue;
        if (c > 0 && __ldg(carry_row + c - 1) == r) continue;
        long long end = c + 1;
        while (end < G && __ldg(carry_row + end) == r) ++end;
        for (int col = lane; col < kc; col += 32) {
            float s = 0.f, comp = 0.f;
            for (long long t = c; t < end; ++t) kbn_add(s, comp, __ldg(carry_val + t * kc + col));
            C[static_cast<long long>(r) * kc + col] += s + comp;
        }
    }
}

template <typename V, int TMAX, bool VEC>
static cudaError_t launch_spmm_t(int G, int m, int n, int kc, const int *tile_row, const int *tile_nz, const int *row_end,
                                 const int *ci, const V *values, const float *B, float *C, int *carry_row,
                                 float *carry_val, cudaStream_t st) {
    constexpr int THREADS = 256;
    const int kq = (kc + 3) / 4;
    int nq = 1;
    while (nq < kq && nq < 32) nq <<= 1;  // up to 32 quads (128 columns) per pass
    auto kern = spmm_kernel<V, THREADS, TMAX, VEC>;
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
static cudaError_t launch_spmm_v(int G, int m, int n, int kc, int tile_items, const int *tile_row, const int *tile_nz,
                                 const int *row_end, const int *ci, const void *values, const float *B, float *C,
                                 int *carry_row, float *carry_val, cudaStream_t st) {
    const V *v = static_cast<const V *>(values);
    const bool vec = kc % 4 == 0 && (reinterpret_cast<uintptr_t>(B) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(C) & 15u) == 0;
    if (tile_items > 2048) return cudaErrorInvalidValue;  // shared-memory staging holds 2048 items
    return vec ? launch_spmm_t<V, 2048, true>(G, m, n, kc, tile_row, tile_nz, row_end, ci, v, B, C, carry_row, carry_val,
                                              st)
               : launch_spmm_t<V, 2048, false>(G, m, n, kc, tile_row, tile_nz, row_end, ci, v, B, C, carry_row,
                                               carry_val, st);
}

cudaError_t launch_spmm(lb_dtype vdt, int G, int m, int n, int kc, int tile_items, const int *tile_row, const int *tile_nz,
                        const int *row_end, const int *ci, const void *values, const float *B, float *C,
                        int *carry_row, float *carry_val, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    switch (vdt) {
        case LB_F32:
            return launch_spmm_v<float>(G, m, n, kc, tile_items, tile_row, tile_nz, row_end, ci, values, B, C, carry_row,
                                        carry_val, st);
        case LB_BF16:
            return launch_spmm_v<__nv_bfloat16>(G, m, n, kc, tile_items, tile_row, tile_nz, row_end, ci, values, B, C,
                                                carry_row, carry_val, st);
        case LB_F16:
            return launch_spmm_v<__half>(G, m, n, kc, tile_items, tile_row, tile_nz, row_end, ci, values, B, C, carry_row,
                                         carry_val, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lb
