// lb_mapped.cu -- thread-mapped, group-mapped (4..32 lanes) and block-mapped SpMV.
//
// Thread-mapped (Ch.3 Sec. "Thread-Mapped"; Ch.4 Listing lst:thread-mapped and lst:spmv): a
// row per thread, rows strided by the grid, the row's nonzeros summed in order.
//
// Group-mapped (Ch.3 Sec. "Group-Mapped", Alg. alg:group-mapped; Ch.4 Sec. "Group-level load
// balancing"): a group of G threads owns G consecutive rows.  Each thread loads one row's
// length, the group forms the inclusive prefix sum, and the group then walks the group's
// nonzeros G at a time: thread t of a round takes nonzero kb + t, finds its row by a binary
// search in the prefix sum (upper bound: the first row whose running total exceeds the
// atom's index), and multiplies.  The paper's pseudocode assigns the product to y[row]; here
// each round reduces the products row by row (a segmented scan across the group) and the
// owner thread of each row accumulates the round's sum, so a row's sum is complete and
// deterministic without atomics.
//
// Sums across rounds (and along a thread-mapped row) use compensated addition, so the error
// bound stays that of a few roundings however long the row.
#include "lb_internal.cuh"

namespace lb {

// v[k] * x[ci[k]] for nonzero k (tested against nnz and n in the range-checked build).
template <typename V>
__device__ __forceinline__ float nz_product(const V *__restrict__ v, const int *__restrict__ ci,
                                           const float *__restrict__ x, long long k, int nnz, int n) {
    if (!LB_IN_RANGE(k, nnz)) return 0.f;
    const int c = __ldg(ci + k);
    return LB_IN_RANGE(c, n) ? to_f32(__ldg(v + k)) * __ldg(x + c) : 0.f;
}

template <typename V>
__global__ void __launch_bounds__(256) thread_mapped_kernel(int m, int n, int nnz, const int *__restrict__ ro,
                                                            const int *__restrict__ ci, const V *__restrict__ v,
                                                            const float *__restrict__ x, float *__restrict__ y) {
    for (long long row = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; row < m;
         row += static_cast<long long>(gridDim.x) * blockDim.x) {
        float s = 0.f, c = 0.f;
        const int e = __ldg(ro + row + 1);
        for (int k = __ldg(ro + row); k < e; ++k) kbn_add(s, c, nz_product(v, ci, x, k, nnz, n));
        y[row] = s + c;
    }
}

template <typename V, int G>
__global__ void __launch_bounds__(256) group_mapped_kernel(int m, int n, int nnz, const int *__restrict__ ro,
                                                           const int *__restrict__ ci, const V *__restrict__ v,
                                                           const float *__restrict__ x, float *__restrict__ y) {
    static_assert(G >= 2 && G <= 32 && (G & (G - 1)) == 0, "group size");
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const long long groups = static_cast<long long>(gridDim.x) * blockDim.x / G;
    for (long long grp = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) / G; grp * G < m;
         grp += groups) {
        const long long row = grp * G + gl;
        const int start = row < m ? __ldg(ro + row) : 0;
        const int len = row < m ? __ldg(ro + row + 1) - start : 0;
        int sc = len;  // inclusive prefix sum of row lengths over the group
#pragma unroll
        for (int off = 1; off < G; off <<= 1) {
            const int t = __shfl_up_sync(gmask, sc, off, G);
            if (gl >= off) sc += t;
        }
        const int total = __shfl_sync(gmask, sc, G - 1, G);
        const int base = __shfl_sync(gmask, start, 0, G);
        const int my_first = sc - len;
        float acc = 0.f, comp = 0.f;
        for (int kb = 0; kb < total; kb += G) {
            const int k = kb + gl;
            // Row of atom k: the first lane whose running total exceeds k.
            int lo = 0, hi = G - 1;
#pragma unroll
            for (int step = 1; step < G; step <<= 1) {
                const int mid = (lo + hi) >> 1;
                const int smid = __shfl_sync(gmask, sc, mid, G);
                if (smid > k)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            const int rl = lo;
            float p = 0.f;
            if (k < total) {
                const int nz = base + k;
                p = nz_product(v, ci, x, nz, nnz, n);
            }
            // Segmented inclusive scan of the round's products by row.
            float sp = p;
#pragma unroll
            for (int off = 1; off < G; off <<= 1) {
                const float t = __shfl_up_sync(gmask, sp, off, G);
                const int rt = __shfl_up_sync(gmask, rl, off, G);
                if (gl >= off && rt == rl) sp += t;
            }
            // The owner of each row reads the scan at its row's last atom in this round.
            const bool mine = len > 0 && my_first < kb + G && sc > kb;
            const int last = (sc < kb + G ? sc : kb + G) - 1;
            const int src = mine ? last - kb : 0;
            const float seg = __shfl_sync(gmask, sp, src, G);
            if (mine) kbn_add(acc, comp, seg);
        }
        if (row < m) y[row] = acc + comp;
    }
}

// Block-mapped: the group is the whole block (THREADS rows per block, shared-memory scans).
template <typename V, int THREADS>
__global__ void __launch_bounds__(THREADS) block_mapped_kernel(int m, int n, int nnz, const int *__restrict__ ro,
                                                               const int *__restrict__ ci, const V *__restrict__ v,
                                                               const float *__restrict__ x, float *__restrict__ y) {
    constexpr int WARPS = THREADS / 32;
    __shared__ int s_sc[THREADS];
    __shared__ float s_sp[THREADS];
    __shared__ int s_wi[WARPS];
    __shared__ float s_wv[WARPS];
    __shared__ int s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (long long row0 = static_cast<long long>(blockIdx.x) * THREADS; row0 < m;
         row0 += static_cast<long long>(gridDim.x) * THREADS) {
        const long long row = row0 + tid;
        const int start = row < m ? __ldg(ro + row) : 0;
        const int len = row < m ? __ldg(ro + row + 1) - start : 0;
        // Block inclusive scan of the lengths.
        int sc = len;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, sc, off);
            if (lane >= off) sc += t;
        }
        if (lane == 31) s_wi[warp] = sc;
        if (tid == 0) s_base = start;
        __syncthreads();
        int pre = 0;
        for (int w = 0; w < warp; ++w) pre += s_wi[w];
        sc += pre;
        s_sc[tid] = sc;
        __syncthreads();
        const int total = s_sc[THREADS - 1];
        const int base = s_base;
        const int my_first = sc - len;
        float acc = 0.f, comp = 0.f;
        for (int kb = 0; kb < total; kb += THREADS) {
            const int k = kb + tid;
            int lo = 0, hi = THREADS - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_sc[mid] > k)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            const int rl = lo;
            float p = 0.f;
            if (k < total) {
                const int nz = base + k;
                p = nz_product(v, ci, x, nz, nnz, n);
            }
            // Segmented inclusive scan over the block: (starts a row segment?, value).
            const int rprev = __shfl_up_sync(0xffffffffu, rl, 1);
            int fi = (lane == 0) ? 1 : (rprev != rl);
            float vi = p;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float vu = __shfl_up_sync(0xffffffffu, vi, off);
                const int fu = __shfl_up_sync(0xffffffffu, fi, off);
                if (lane >= off) {
                    if (!fi) vi = vu + vi;
                    fi |= fu;
                }
            }
            // Lane 0 of a warp starts a segment only if the previous warp's last row differs.
            const int first_rl = __shfl_sync(0xffffffffu, rl, 0);
            const int last_rl = __shfl_sync(0xffffffffu, rl, 31);
            if (lane == 31) {
                s_wv[warp] = vi;
                s_wi[warp] = last_rl;
            }
            __syncthreads();
            // Carry from earlier warps into this warp's first segment: rows are non-decreasing
            // across the block, so the earlier atoms of row first_rl are exactly the tail
            // segments of the earlier warps whose last row is first_rl.
            float pv = 0.f;
            for (int w = 0; w < warp; ++w)
                if (s_wi[w] == first_rl) pv += s_wv[w];
            // Lanes in this warp's first segment (no segment start before them) take pv.
            const unsigned starts = __ballot_sync(0xffffffffu, (lane == 0) ? 0 : (rprev != rl));
            const bool in_first = (starts & ((2u << lane) - 1u)) == 0;
            if (in_first) vi = pv + vi;
            s_sp[tid] = vi;
            __syncthreads();
            const bool mine = len > 0 && my_first < kb + THREADS && sc > kb;
            if (mine) {
                const int last = (sc < kb + THREADS ? sc : kb + THREADS) - 1;
                kbn_add(acc, comp, s_sp[last - kb]);
            }
            __syncthreads();
        }
        if (row < m) y[row] = acc + comp;
        __syncthreads();
    }
}

template <typename V>
static cudaError_t launch_mapped_t(lb_schedule s, const lb_tuning &t, int m, int n, int nnz, const int *ro, const int *ci,
                                   const V *v, const float *x, float *y, cudaStream_t st) {
    const int sms = current_sm_count();
    if (s == LB_SCHED_THREAD_MAPPED) {
        long long blocks = (static_cast<long long>(m) + 255) / 256;
        if (blocks > static_cast<long long>(sms) * 64) blocks = static_cast<long long>(sms) * 64;
        thread_mapped_kernel<V><<<static_cast<int>(blocks), 256, 0, st>>>(m, n, nnz, ro, ci, v, x, y);
        return cudaGetLastError();
    }
    if (s == LB_SCHED_BLOCK_MAPPED) {
        const int th = t.threads > 0 ? t.threads : 256;
        long long blocks = (static_cast<long long>(m) + th - 1) / th;
        if (blocks > static_cast<long long>(sms) * 32) blocks = static_cast<long long>(sms) * 32;
        if (th == 128)
            block_mapped_kernel<V, 128><<<static_cast<int>(blocks), 128, 0, st>>>(m, n, nnz, ro, ci, v, x, y);
        else if (th == 256)
            block_mapped_kernel<V, 256><<<static_cast<int>(blocks), 256, 0, st>>>(m, n, nnz, ro, ci, v, x, y);
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    const int g = (s == LB_SCHED_WARP_MAPPED) ? 32 : (t.group_size > 0 ? t.group_size : 32);
    long long blocks = (static_cast<long long>(m) + 255) / 256;  // 256 rows per block of 256 threads
    if (blocks > static_cast<long long>(sms) * 64) blocks = static_cast<long long>(sms) * 64;
    switch (g) {
        case 4:
            group_mapped_kernel<V, 4><<<static_cast<int>(blocks), 256, 0, st>>>(m, n, nnz, ro, ci, v, x, y);
            break;
        case 8:
            group_mapped_kernel<V, 8><<<static_cast<int>(blocks), 256, 0, st>>>(m, n, nnz, ro, ci, v, x, y);
            break;
        case 16:
            group_mapped_kernel<V, 16><<<static_cast<int>(blocks), 256, 0, st>>>(m, n, nnz, ro, ci, v, x, y);
            break;
        case 32:
            group_mapped_kernel<V, 32><<<static_cast<int>(blocks), 256, 0, st>>>(m, n, nnz, ro, ci, v, x, y);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_mapped(lb_schedule s, const lb_tuning &t, lb_dtype vdt, int m, int n, int nnz, const int *ro, const int *ci,
                          const void *v, const float *x, float *y, cudaStream_t stream) {
    if (m <= 0) return cudaSuccess;
    switch (vdt) {
        case LB_F32:
            return launch_mapped_t<float>(s, t, m, n, nnz, ro, ci, static_cast<const float *>(v), x, y, stream);
        case LB_BF16:
            return launch_mapped_t<__nv_bfloat16>(s, t, m, n, nnz, ro, ci, static_cast<const __nv_bfloat16 *>(v), x, y,
                                                  stream);
        case LB_F16:
            return launch_mapped_t<__half>(s, t, m, n, nnz, ro, ci, static_cast<const __half *>(v), x, y, stream);
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------------
// Thread-mapped over a batch (the row schedule of Ch.3 Sec. "Thread-Mapped", applied to the
// block-diagonal matrix of a batched plan), with the group-mapped remedy for its imbalance:
// a row longer than kLongRow nonzeros is not left to one lane but summed by the whole warp
// (Ch.3 Sec. "Group-Mapped" with the group a warp).  Each warp owns a contiguous range of
// rows, 32 at a time with consecutive rows on consecutive lanes; a lane sums its short row
// in order with compensated addition; the warp then takes the chunk's long rows one by one,
// each lane summing a strided share and a fixed shuffle tree joining them.  Every row is
// finished by one lane or one warp: no carries and no fixup.  The warps' row ranges come
// from the plan's merge-path partition (whole runs of its tiles, cut at the row ends the
// tiles' boundaries fall after), so each warp gets about the same rows + nonzeros.  The matrix
// of a row (for its column base) is found once per warp by binary search and then followed
// forward.

struct BatchRowsArgs {
    long long rows;           // rows of the block-diagonal matrix
    const int *ro;            // its offsets [rows + 1]
    const int *ci;            // local column indices (per matrix)
    const void *val;          // values
    const float *x;           // concatenated x
    long long x_len;          // its length
    float *y;                 // concatenated y [rows]
    int kc;                   // matrices with rows
    const int *mat_row_base;  // [kc + 1] first global row of each matrix
    const int *mat_col_base;  // [kc] offset of each matrix's x inside x
    int G;                    // merge-path tiles of the plan's partition
    const int *tile_row;      // [G + 1] row ends consumed before each tile boundary
};

constexpr int kLongRow = 32;

template <typename V>
__global__ void __launch_bounds__(256) batched_rows_kernel(const BatchRowsArgs a) {
    const V *__restrict__ v = static_cast<const V *>(a.val);
    const int lane = threadIdx.x & 31;
    const long long warp = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
    const long long per = (a.G + nwarps - 1) / nwarps;  // tiles per warp
    const long long t0 = warp * per, t1 = t0 + per < a.G ? t0 + per : a.G;
    if (t0 >= t1) return;
    const long long r_begin = __ldg(a.tile_row + t0);
    const long long r_end = t1 == a.G ? a.rows : __ldg(a.tile_row + t1);
    long long c = 0;  // chunks of 32 rows from r_begin
    const long long c_end = (r_end - r_begin + 31) >> 5;
    if (c >= c_end) return;
    // Matrix of the warp's first row: the last i with mat_row_base[i] <= row.
    int mi = 0;
    if (lane == 0) {
        int lo = 0, hi = a.kc - 1;
        const long long r = r_begin;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(a.mat_row_base + mid) <= r)
                lo = mid;
            else
                hi = mid - 1;
        }
        mi = lo;
    }
    mi = __shfl_sync(0xffffffffu, mi, 0);
    // Row offsets of the first chunk; each chunk loads the next chunk's while it works.
    auto load_ro = [&](long long cc, int &s, int &e) {
        const long long row = r_begin + (cc << 5) + lane;
        s = row < r_end ? __ldg(a.ro + row) : 0;
        e = row < r_end ? __ldg(a.ro + row + 1) : 0;
    };
    int s, e;
    load_ro(c, s, e);
    for (; c < c_end; ++c) {
        const long long row = r_begin + (c << 5) + lane;
        const bool in = row < r_end;
        int i = mi;
        if (in)
            while (i + 1 < a.kc && __ldg(a.mat_row_base + i + 1) <= row) ++i;
        mi = __shfl_sync(0xffffffffu, i, 31);  // rows only increase
        const int cb = in ? __ldg(a.mat_col_base + i) : 0;
        const bool lng = e - s > kLongRow;
        int ns = 0, ne = 0;
        if (c + 1 < c_end) load_ro(c + 1, ns, ne);
        // A short row: its lane sums it in order, two nonzeros' loads in flight at a time.
        float acc = 0.f, comp = 0.f;
        if (in && !lng) {
            int k = s;
            for (; k + 1 < e; k += 2) {
                const long long g0 = static_cast<long long>(__ldg(a.ci + k)) + cb;
                const long long g1 = static_cast<long long>(__ldg(a.ci + k + 1)) + cb;
                const float v0 = to_f32(__ldg(v + k)), v1 = to_f32(__ldg(v + k + 1));
                const float x0 = LB_IN_RANGE(g0, a.x_len) ? __ldg(a.x + g0) : 0.f;
                const float x1 = LB_IN_RANGE(g1, a.x_len) ? __ldg(a.x + g1) : 0.f;
                kbn_add(acc, comp, v0 * x0);
                kbn_add(acc, comp, v1 * x1);
            }
            if (k < e) {
                const long long g0 = static_cast<long long>(__ldg(a.ci + k)) + cb;
                if (LB_IN_RANGE(g0, a.x_len)) kbn_add(acc, comp, to_f32(__ldg(v + k)) * __ldg(a.x + g0));
            }
        }
        // Long rows: the whole warp, one row at a time, 128 nonzeros per step.
        for (unsigned lm = __ballot_sync(0xffffffffu, in && lng); lm; lm &= lm - 1) {
            const int src = __ffs(lm) - 1;
            const int rs = __shfl_sync(0xffffffffu, s, src), re = __shfl_sync(0xffffffffu, e, src);
            const int rcb = __shfl_sync(0xffffffffu, cb, src);
            float ps = 0.f, pc = 0.f;
            for (int k0 = rs; k0 < re; k0 += 128) {
                int kc4[4];
                float vv4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = k0 + 32 * u + lane;
                    kc4[u] = k < re ? __ldg(a.ci + k) : -1;
                    vv4[u] = k < re ? to_f32(__ldg(v + k)) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long gcol = static_cast<long long>(kc4[u]) + rcb;
                    if (kc4[u] >= 0 && LB_IN_RANGE(gcol, a.x_len)) kbn_add(ps, pc, vv4[u] * __ldg(a.x + gcol));
                }
            }
            float t = ps + pc;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == src) acc = t, comp = 0.f;
        }
        if (in) a.y[row] = acc + comp;
        s = ns;
        e = ne;
    }
}

cudaError_t launch_batched_rows(lb_dtype vdt, long long rows, const int *ro, const int *ci, const void *val,
                                const float *x, long long x_len, float *y, int kc, const int *mat_row_base,
                                const int *mat_col_base, int G, const int *tile_row, cudaStream_t stream) {
    if (rows <= 0 || kc <= 0 || G <= 0) return cudaSuccess;
    BatchRowsArgs a{rows, ro, ci, val, x, x_len, y, kc, mat_row_base, mat_col_base, G, tile_row};
    // One wave of resident warps, each a contiguous run of tiles.
    auto wave = [&](auto kern) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        long long blocks = static_cast<long long>(per_sm) * current_sm_count();
        const long long need = (static_cast<long long>(G) + 7) / 8;  // 8 warps per block, a tile or more each
        if (blocks > need) blocks = need;
        kern<<<static_cast<int>(blocks), 256, 0, stream>>>(a);
        return cudaGetLastError();
    };
    switch (vdt) {
        case LB_F32:
            return wave(batched_rows_kernel<float>);
        case LB_BF16:
            return wave(batched_rows_kernel<__nv_bfloat16>);
        case LB_F16:
            return wave(batched_rows_kernel<__half>);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lb
