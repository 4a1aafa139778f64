// lb_nzsplit.cu -- the nonzero-splitting schedule: every tile gets the same number of
// nonzeros, rows cost nothing.
//
// The dissertation names two definitions of a work item for work-oriented scheduling (Ch.3
// Sec. "Work-Oriented"): nonzero splitting counts only the nonzeros (multiply-adds) as work,
// merge path counts the nonzeros and the rows.  With nonzero splitting a tile holds exactly T
// nonzeros however many rows they span, so empty rows are free to the partition but still
// have to be written: here y is cleared first and only rows with nonzeros are written, which
// is this schedule's cost on matrices with many empty rows.
//
// Per tile (T = 2048 nonzeros): the rows starting inside the tile add 1 to a per-slot count,
// and a block scan gives each nonzero's row; each thread walks its 8 consecutive nonzeros and
// writes the rows that start and end among them.  Rows spanning threads are summed by a
// segmented scan of the threads' last partial rows, in thread order, and written where they
// end.  The tile's first and last rows, which may continue in the neighbouring tiles, go out
// as two carries, and the fixup adds each row's carries in tile order: deterministic, no
// atomics on y.
#include <cstring>

#include "lb_internal.cuh"

namespace lb {

namespace {

constexpr int kNzThreads = 256;
constexpr int kNzIpt = 8;

// Row holding nonzero k: the last r with ro[r] <= k (0 <= k < nnz).
__device__ __forceinline__ int row_of_nonzero(const int *__restrict__ ro, int m, long long k) {
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(ro + mid) <= k)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void nz_partition_kernel(int G, int m, int nnz, int T, const int *__restrict__ ro, int *first_row,
                                    int *last_row) {
    for (long long c = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; c < G;
         c += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long k0 = c * T;
        const long long k1 = k0 + T < nnz ? k0 + T : nnz;
        first_row[c] = row_of_nonzero(ro, m, k0);
        last_row[c] = row_of_nonzero(ro, m, k1 - 1);
    }
}

// Eight consecutive values from a 16-byte-aligned address, widened to FP32.
__device__ __forceinline__ void load8_values(const float *p, float (&o)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p)), b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
template <typename H>
__device__ __forceinline__ void load8_values(const H *p, float (&o)[8]) {
    const uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        H lo, hi;
        const unsigned short bl = static_cast<unsigned short>(w[e] & 0xffffu), bh = static_cast<unsigned short>(w[e] >> 16);
        memcpy(&lo, &bl, 2);
        memcpy(&hi, &bh, 2);
        o[2 * e] = to_f32(lo);
        o[2 * e + 1] = to_f32(hi);
    }
}

template <typename V>
__global__ void __launch_bounds__(kNzThreads) nzsplit_kernel(int G, int m, int n, int nnz, const int *__restrict__ first_row,
                                                             const int *__restrict__ last_row,
                                                             const int *__restrict__ ro, const int *__restrict__ ci,
                                                             const V *__restrict__ values, const float *__restrict__ x,
                                                             float *__restrict__ y, int *__restrict__ carry_row,
                                                             float *__restrict__ carry_val) {
    constexpr int T = kNzThreads * kNzIpt;
    constexpr int WARPS = kNzThreads / 32;
    __shared__ __align__(16) int cnt[T];
    __shared__ int wsum[WARPS];
    __shared__ int s_tail[kNzThreads];    // each thread's last row (-1: no nonzeros)
    __shared__ int s_first[kNzThreads];   // each thread's first row
    __shared__ float s_tval[kNzThreads];  // scanned tail values
    __shared__ float w_val[WARPS];
    __shared__ int w_seg[WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(ci) & 15u) == 0 && (reinterpret_cast<uintptr_t>(values) & 15u) == 0;
    for (int i = tid; i < T; i += kNzThreads) cnt[i] = 0;
    __syncthreads();
    for (int tile = blockIdx.x; tile < G; tile += gridDim.x) {
        const long long k0 = static_cast<long long>(tile) * T;
        const int nk = static_cast<int>(k0 + T < nnz ? T : nnz - k0);
        const int r_first = __ldg(first_row + tile), r_last = __ldg(last_row + tile);
        // Gathers first: they do not depend on the rows.  A tile starts at a multiple of 2048
        // nonzeros, so a thread's 8 consecutive indices and values move as 16-byte vectors
        // when the arrays' bases allow it.
        const int j0 = tid * kNzIpt;
        float prod[kNzIpt];
        if (vec && j0 + kNzIpt <= nk) {
            int col[kNzIpt];
            float val[kNzIpt];
            const int4 *cp = reinterpret_cast<const int4 *>(ci + k0 + j0);
            const int4 c0 = __ldg(cp), c1 = __ldg(cp + 1);
            col[0] = c0.x; col[1] = c0.y; col[2] = c0.z; col[3] = c0.w;
            col[4] = c1.x; col[5] = c1.y; col[6] = c1.z; col[7] = c1.w;
            load8_values(values + k0 + j0, val);
#pragma unroll
            for (int q = 0; q < kNzIpt; ++q) prod[q] = LB_IN_RANGE(col[q], n) ? val[q] * __ldg(x + col[q]) : 0.f;
        } else {
#pragma unroll
            for (int q = 0; q < kNzIpt; ++q) {
                const int j = j0 + q;
                prod[q] = 0.f;
                if (j < nk) {
                    const int c = __ldg(ci + k0 + j);
                    if (LB_IN_RANGE(c, n)) prod[q] = to_f32(values[k0 + j]) * __ldg(x + c);
                }
            }
        }
        // Rows starting inside the tile (empty rows included: they share a start).
        for (long long r = r_first + 1 + tid; r <= r_last; r += kNzThreads) {
            const long long s = __ldg(ro + r) - k0;
            if (s > 0 && s < nk) atomicAdd(&cnt[s], 1);
        }
        __syncthreads();
        int c[kNzIpt];
#pragma unroll
        for (int q = 0; q < kNzIpt; q += 4) {
            const int4 t = *reinterpret_cast<const int4 *>(cnt + j0 + q);
            c[q] = t.x;
            c[q + 1] = t.y;
            c[q + 2] = t.z;
            c[q + 3] = t.w;
            *reinterpret_cast<int4 *>(cnt + j0 + q) = make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 1; q < kNzIpt; ++q) c[q] += c[q - 1];
        const int tot = c[kNzIpt - 1];
        int incl = tot;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int base = r_first + incl - tot;
        for (int w = 0; w < warp; ++w) base += wsum[w];
        // Walk this thread's nonzeros: rows that start and end here are complete.
        int cur = -1, first = -1;
        float acc = 0.f, facc = 0.f;
#pragma unroll
        for (int q = 0; q < kNzIpt; ++q) {
            if (j0 + q >= nk) break;
            const int row = base + c[q];
            if (row != cur) {
                if (cur >= 0) {
                    if (first < 0) {
                        first = cur;
                        facc = acc;
                    } else {
                        y[cur] = acc;
                    }
                }
                cur = row;
                acc = 0.f;
            }
            acc += prod[q];
        }
        // This thread's partial rows: its first row (f, a), and when another row follows, its
        // last row (l, b).  Rows spanning threads are summed by a segmented scan over the
        // threads in order; each row's total is written where its last segment lies.
        const bool active = j0 < nk;
        const bool has2 = first >= 0;
        const int f = has2 ? first : cur;
        const float a = has2 ? facc : acc;
        const int L = active ? cur : -1;  // the thread's tail row
        if (tid == 0) {  // the tile's two carries start empty
            carry_row[2 * tile] = r_first;
            carry_val[2 * tile] = 0.f;
            carry_row[2 * tile + 1] = r_last;
            carry_val[2 * tile + 1] = 0.f;
        }
        s_tail[tid] = L;
        __syncthreads();
        const int prevL = tid > 0 ? s_tail[tid - 1] : -1;
        const bool cont = active && !has2 && f == prevL;  // the tail continues the previous thread's
        // Segmented inclusive scan of the tail values, restarting where a tail does not continue.
        float tv = active ? acc : 0.f;
        bool seg = !cont;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float v_up = __shfl_up_sync(0xffffffffu, tv, off);
            const int s_up = __shfl_up_sync(0xffffffffu, static_cast<int>(seg), off);
            if (lane >= off && !seg) tv += v_up;
            if (lane >= off) seg = seg || s_up;
        }
        if (lane == 31) {
            w_val[warp] = tv;
            w_seg[warp] = seg ? 1 : 0;
        }
        __syncthreads();
        if (!seg) {  // no restart in this warp up to here: add the carry of the warps before
            float c = 0.f;
            for (int w = 0; w < warp; ++w) c = w_seg[w] ? w_val[w] : c + w_val[w];
            tv += c;
        }
        s_tval[tid] = tv;
        s_first[tid] = active ? f : -1;
        __syncthreads();
        if (active) {
            auto put = [&](int R, float v) {
                if (R == r_first)
                    carry_val[2 * tile] = v;  // may continue from the tile before
                else if (R == r_last)
                    carry_val[2 * tile + 1] = v;  // may continue into the tile after
                else
                    y[R] = v;
            };
            if (has2) put(f, a + (tid > 0 && prevL == f ? s_tval[tid - 1] : 0.f));  // the first row ends here
            const bool tail_ends = tid + 1 == kNzThreads || s_first[tid + 1] != L;
            if (tail_ends) put(L, tv);
        }
        __syncthreads();
    }
}

template <typename V>
cudaError_t launch_nzsplit_t(int G, int m, int n, int nnz, const int *first_row, const int *last_row, const int *ro,
                             const int *ci, const void *values, const float *x, float *y, int *carry_row,
                             float *carry_val, cudaStream_t st) {
    auto kern = nzsplit_kernel<V>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNzThreads, 0);
    if (e != cudaSuccess) return e;
    long long grid = static_cast<long long>(per_sm > 0 ? per_sm : 1) * current_sm_count();
    if (grid > G) grid = G;
    kern<<<static_cast<int>(grid), kNzThreads, 0, st>>>(G, m, n, nnz, first_row, last_row, ro, ci,
                                                         static_cast<const V *>(values), x, y, carry_row, carry_val);
    return cudaGetLastError();
}

}  // namespace

int nzsplit_tile_nonzeros() { return kNzThreads * kNzIpt; }

cudaError_t launch_nz_partition(int G, int m, int nnz, const int *ro, int *first_row, int *last_row,
                                cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    long long b = (static_cast<long long>(G) + 255) / 256;
    const long long cap = static_cast<long long>(current_sm_count()) * 16;
    nz_partition_kernel<<<static_cast<int>(b < cap ? b : cap), 256, 0, st>>>(G, m, nnz, nzsplit_tile_nonzeros(), ro,
                                                                           first_row, last_row);
    return cudaGetLastError();
}

cudaError_t launch_nzsplit(lb_dtype vdt, int G, int m, int n, int nnz, const int *first_row, const int *last_row,
                           const int *ro, const int *ci, const void *values, const float *x, float *y,
                           int *carry_row, float *carry_val, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(y, 0, static_cast<size_t>(m) * sizeof(float), st);
    if (e != cudaSuccess || G <= 0) return e;
    switch (vdt) {
        case LB_F32:
            e = launch_nzsplit_t<float>(G, m, n, nnz, first_row, last_row, ro, ci, values, x, y, carry_row, carry_val, st);
            break;
        case LB_BF16:
            e = launch_nzsplit_t<__nv_bfloat16>(G, m, n, nnz, first_row, last_row, ro, ci, values, x, y, carry_row,
                                                carry_val, st);
            break;
        case LB_F16:
            e = launch_nzsplit_t<__half>(G, m, n, nnz, first_row, last_row, ro, ci, values, x, y, carry_row, carry_val,
                                         st);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return launch_fixup(2 * G, m, carry_row, carry_val, y, st);
}

}  // namespace lb
