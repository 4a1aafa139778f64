// lb_partition.cu -- merge-path partition, carry fixup, batched-plan helpers, validation.
#include <climits>
#include <mutex>

#include "lb_internal.cuh"

namespace lb {

int current_sm_count() {
    constexpr int kMaxDev = 64;
    static int cache[kMaxDev] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
    if (cache[dev] == 0) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = sms > 0 ? sms : 1;
    }
    return cache[dev];
}

// ------------------------------------------------------------------------------------------
// Merge-path partition (Alg. alg:work-oriented, the "2DSearch" for every tile boundary).
//
// Row end R_r sits at merge position K_r = r + offsets[r+1] (R_r precedes nonzero k exactly
// when offsets[r+1] <= k), and K_r increases strictly with r.  A boundary d has
// i(d) = #{r : K_r < d} row ends before it, so i(d) = r exactly for K_{r-1} < d <= K_r
// (K_{-1} = -1, K_m = W).  Instead of one binary search per boundary, every row r computes
// the boundaries c with d_c = min(c T, W) in that interval and writes (r, d_c - r) for them:
// one coalesced pass over the offsets, the same result bit for bit.  A warp shares the
// writes of its 32 rows, so a row spanning many tiles does not serialize one thread; each warp
// step loads four chunks of 32 rows' offsets before working on them.
__global__ void __launch_bounds__(256) partition_kernel(int m, long long W, int T, long long G, const int *offsets,
                                                        int *tile_row, int *tile_nz) {
    constexpr int U = 4;  // 32-row chunks per warp step, their offsets loaded together
    const int lane = threadIdx.x & 31;
    const long long warp = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const long long warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
    const unsigned Tu = static_cast<unsigned>(T);
    const int Gi = static_cast<int>(G);  // G < 2^31 (checked on the host)
    for (long long base0 = warp * 32 * U; base0 <= m; base0 += warps * 32 * U) {
        // Each lane loads offsets[r+1] of its row in every chunk; lane 0 also loads offsets[r]
        // of the step's first row, whose predecessor lies outside the step.
        int end_offs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long r = base0 + 32 * u + lane;
            end_offs[u] = (r < m) ? __ldg(offsets + r + 1) : 0;
        }
        const int start0 = (lane == 0 && base0 > 0 && base0 <= m) ? __ldg(offsets + base0) : 0;
        // Tile of the row end before the step's first row: K_{r-1} / T, or -1 before row 0.
        int q_carry = -1;
        if (base0 > 0) {
            const unsigned qc = static_cast<unsigned>((base0 - 1) + static_cast<long long>(start0)) / Tu;
            q_carry = qc < static_cast<unsigned>(Gi) ? static_cast<int>(qc) : Gi;
        }
        q_carry = __shfl_sync(0xffffffffu, q_carry, 0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long base = base0 + 32 * u;
            if (base > m) break;  // warp-uniform
            const long long r = base + lane;
            // Boundaries c with K_{r-1} < c T <= K_r (and c = G at row m) are those with
            // q(r-1) < c <= q(r), where q(r) = K_r / T (rounded down) and K_r = r + offsets[r+1]
            // fits 32 bits (m + nnz < 2^32); q(r) = G from row m on.  One division per row: q(r-1)
            // comes from the lane below.  Tile indices and counts are below G < 2^31.
            int q_cur = Gi;
            if (r < m) {
                const unsigned qc = static_cast<unsigned>(r + static_cast<long long>(end_offs[u])) / Tu;
                q_cur = qc < static_cast<unsigned>(Gi) ? static_cast<int>(qc) : Gi;  // malformed offsets: keep writes in [0, G]
            }
            int q_prev = __shfl_up_sync(0xffffffffu, q_cur, 1);
            if (lane == 0) q_prev = q_carry;
            q_carry = __shfl_sync(0xffffffffu, q_cur, 31);
            const int c_lo = q_prev + 1;
            const int n_c = r <= m && q_cur > q_prev ? q_cur - q_prev : 0;
            if (__ballot_sync(0xffffffffu, n_c > 0) == 0u) continue;  // no boundary in these 32 rows (most)
            // Exclusive prefix of the per-lane boundary counts.
            int incl = n_c;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += t;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            const int excl = incl - n_c;
            for (int q0 = 0; q0 < total; q0 += 32) {  // warp-uniform trip count
                const int q = q0 + lane;
                // Owner: the last lane whose exclusive prefix is <= q.
                int lo = 0, hi = 31;
#pragma unroll
                for (int step = 0; step < 5; ++step) {
                    const int mid = (lo + hi + 1) >> 1;
                    const int e_mid = __shfl_sync(0xffffffffu, excl, mid);
                    if (e_mid <= q)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                const int e_own = __shfl_sync(0xffffffffu, excl, lo);
                const int c_own = __shfl_sync(0xffffffffu, c_lo, lo);
                if (q >= total) continue;
                const long long c = static_cast<long long>(c_own) + (q - e_own);
                const long long row = base + lo;
                const long long d = c * T < W ? c * T : W;
                if (!LB_IN_RANGE(c, G + 1)) continue;
                tile_row[c] = static_cast<int>(row);
                tile_nz[c] = static_cast<int>(d - row);
            }
        }
    }
}

cudaError_t launch_partition(int m, long long nnz, const int *offsets, int tile_items, int *tile_row, int *tile_nz,
                             cudaStream_t stream) {
    const long long W = static_cast<long long>(m) + nnz;
    const long long G = (W + tile_items - 1) / tile_items;
    if (G >= INT_MAX) return cudaErrorInvalidValue;  // the kernel counts tiles in 32 bits
    // A warp per four 32-row chunks (their loads in flight together), grid-strided beyond
    // 16 blocks per SM (several waves: a warp held up by a row spanning many tiles leaves the
    // SM to the next wave's blocks).
    long long blocks = (static_cast<long long>(m) + 1 + 1023) / 1024;
    const long long cap = static_cast<long long>(current_sm_count()) * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    partition_kernel<<<static_cast<int>(blocks), 256, 0, stream>>>(m, W, tile_items, G, offsets, tile_row, tile_nz);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Fixup ("Fix-up" procedure of Alg. alg:work-oriented): y[r] += the carries of row r.
//
// Carry rows are non-decreasing in tile order, so the carries of a row form one run.  A warp
// takes 32 consecutive carries at a time (one coalesced load of rows and values): the runs that
// start and end among them are summed by one segmented shuffle scan and added to y by their
// last lane; the run that starts among them and continues past them (at most one per warp
// step) is summed by the whole warp, which finds the run's end with galloping and 32-way probes
// and sums it with compensated per-lane sums (eight loads in flight per lane) and a fixed
// shuffle tree.  A run that began before the 32 carries belongs to the warp step where it
// began.  Every sum has a fixed order, so the result is deterministic, and there are no
// atomics.  Carry rows outside [0, m) (the -1 of a skipped malformed tile) are skipped.
__global__ void __launch_bounds__(256) fixup_kernel(int G, int m, const int *carry_row, const float *carry_val,
                                                    float *y) {
    const int lane = threadIdx.x & 31;
    const long long warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
    for (long long c0 = ((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32; c0 < G;
         c0 += warps * 32) {
        const long long c = c0 + lane;
        const int r = c < G ? __ldg(carry_row + c) : -1;
        const float v = c < G ? __ldg(carry_val + c) : 0.f;
        const bool valid = static_cast<unsigned>(r) < static_cast<unsigned>(m);
        int prev = __shfl_up_sync(0xffffffffu, r, 1);
        if (lane == 0) prev = c0 > 0 ? __ldg(carry_row + c0 - 1) : -1;
        int next = __shfl_down_sync(0xffffffffu, r, 1);
        if (lane == 31) next = c + 1 < G ? __ldg(carry_row + c + 1) : -1;
        const bool start = lane == 0 || prev != r;  // a segment of equal rows begins here
        const bool head = valid && prev != r;        // a run begins here (not before c0)
        // Segmented inclusive scan of the values over segments of equal rows.
        const uint32_t starts = __ballot_sync(0xffffffffu, start) & (0xffffffffu >> (31 - lane));
        const int seg = 31 - __clz(starts);  // lane 0 always starts a segment
        float s = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float u = __shfl_up_sync(0xffffffffu, s, off);
            if (lane - off >= seg) s += u;
        }
        // A run that starts and ends among these carries: its last lane adds it.
        const int seg_head = __shfl_sync(0xffffffffu, head ? 1 : 0, seg);
        if (valid && next != r && seg_head) y[r] += s;
        // The run that holds lane 31 and continues past it, when it began among these carries:
        // the whole warp sums it.
        const int r31 = __shfl_sync(0xffffffffu, r, 31), n31 = __shfl_sync(0xffffffffu, next, 31);
        const int seg31 = __shfl_sync(0xffffffffu, seg, 31);
        const bool head31 = __shfl_sync(0xffffffffu, head ? 1 : 0, seg31) != 0;
        if (static_cast<unsigned>(r31) < static_cast<unsigned>(m) && n31 == r31 && head31) {
            const long long cs = c0 + seg31;
            const int rs = r31;
            // The run's end: galloping probes (lane l probes cs + 2^l), then 32-way narrowing.
            const long long probe = cs + (1ll << lane);
            const unsigned run_mask = __ballot_sync(0xffffffffu, probe < G && __ldg(carry_row + probe) == rs);
            const int L = __popc(run_mask);  // probes 1, 2, .., 2^(L-1) are inside the run
            long long lo = L == 0 ? cs : cs + (1ll << (L - 1));
            long long hi = cs + (1ll << L);
            if (hi > G) hi = G;
            while (hi - lo > 1) {
                const long long step = (hi - lo + 31) / 32;
                const long long q = lo + (lane + 1) * step;
                const int cnt = __popc(__ballot_sync(0xffffffffu, q < hi && __ldg(carry_row + q) == rs));
                const long long new_lo = lo + cnt * step;
                long long new_hi = new_lo + step;
                if (new_hi > hi) new_hi = hi;
                lo = new_lo;
                hi = new_hi;
            }
            const long long end = hi;  // carries [cs, end) belong to row rs
            float sum = 0.f, comp = 0.f;
            long long q = cs + lane;
            for (; q + 7 * 32 < end; q += 8 * 32) {
                float u[8];
#pragma unroll
                for (int h = 0; h < 8; ++h) u[h] = __ldg(carry_val + q + 32 * h);
#pragma unroll
                for (int h = 0; h < 8; ++h) kbn_add(sum, comp, u[h]);
            }
            for (; q < end; q += 32) kbn_add(sum, comp, __ldg(carry_val + q));
            float t = sum + comp;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0) y[rs] += t;
        }
    }
}

cudaError_t launch_fixup(int num_tiles, int num_rows, const int *carry_row, const float *carry_val, float *y,
                         cudaStream_t stream) {
    if (num_tiles <= 0) return cudaSuccess;
    long long blocks = (static_cast<long long>(num_tiles) + 255) / 256;  // a warp per 32 carries
    const long long cap = static_cast<long long>(current_sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    fixup_kernel<<<static_cast<int>(blocks), 256, 0, stream>>>(num_tiles, num_rows, carry_row, carry_val, y);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Batched plans: the block-diagonal matrix diag(A_0, .., A_{K-1}) (Ch.6 Sec. "Multi-GPU Load
// Balancing": merge-path keeps its structure one level up, a "set of sets").

// ro_global[0] = 0; for row r of matrix i, ro_global[row_base[i] + r + 1] =
// nz_base[i] + ro_concat[ro_pos[i] + r + 1].  One block per matrix, threads over its rows.
__global__ void __launch_bounds__(256) block_diag_offsets_kernel(int count, const int *ro_pos, const int *row_base,
                                                                 const int *nz_base, const int *ro_concat,
                                                                 int *ro_global) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ro_global[0] = 0;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const int rb = row_base[i], m_i = row_base[i + 1] - rb, nb = nz_base[i];
        const int *src = ro_concat + ro_pos[i] + 1;
        for (int r = threadIdx.x; r < m_i; r += blockDim.x) ro_global[rb + r + 1] = nb + src[r];
    }
}

cudaError_t launch_block_diag_offsets(int count, const int *ro_pos, const int *row_base, const int *nz_base,
                                      const int *ro_concat, int total_rows, int *ro_global, cudaStream_t stream) {
    (void)total_rows;
    int blocks = count < current_sm_count() * 8 ? count : current_sm_count() * 8;
    if (blocks < 1) blocks = 1;
    block_diag_offsets_kernel<<<blocks, 256, 0, stream>>>(count, ro_pos, row_base, nz_base, ro_concat, ro_global);
    return cudaGetLastError();
}

// tile_mat[c] = the matrix holding nonzero tile_nz[c]: the last i with mat_nz_base[i] <= k,
// clamped to [0, count - 1].
__global__ void tile_matrix_kernel(int G, const int *tile_nz, int count, const int *mat_nz_base, int *tile_mat) {
    for (long long c = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; c <= G;
         c += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int k = tile_nz[c];
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (mat_nz_base[mid] <= k)
                lo = mid;
            else
                hi = mid - 1;
        }
        tile_mat[c] = lo;
    }
}

cudaError_t launch_tile_matrix(int num_tiles, const int *tile_nz, int count, const int *mat_nz_base, int *tile_mat,
                               cudaStream_t stream) {
    const long long n = static_cast<long long>(num_tiles) + 1;
    int blocks = static_cast<int>((n + 255) / 256);
    if (blocks > current_sm_count() * 8) blocks = current_sm_count() * 8;
    tile_matrix_kernel<<<blocks, 256, 0, stream>>>(num_tiles, tile_nz, count, mat_nz_base, tile_mat);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// CSR validation: ORs problem bits into *status (never traps).
__global__ void validate_offsets_kernel(int m, int nnz, const int *ro, int *status) {
    for (long long r = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; r <= m;
         r += static_cast<long long>(gridDim.x) * blockDim.x) {
        int bits = 0;
        const int v = ro[r];
        if (r == 0 && v != 0) bits |= 1;
        if (r < m && ro[r + 1] < v) bits |= 2;
        if (r == m && v != nnz) bits |= 4;
        if (bits) atomicOr(status, bits);
    }
}

// Each warp checks a contiguous chunk of the nonzeros, 128 at a time (four per lane,
// coalesced): the column range, and an increase over the predecessor except where a row
// starts.  The row starts of each 128-entry window come from walking the row offsets
// alongside (a merge of the two sorted sequences): the warp finds the first offset at or past
// its chunk once by a binary search, then reads the offsets lane-parallel, window by window.
// Row boundaries are only trustworthy when the offsets passed; whatever they hold, every read
// stays inside ro[0..m] and the walk ends.
__global__ void validate_columns_kernel(int m, int n, int nnz, const int *__restrict__ ro,
                                        const int *__restrict__ ci, int check_sorted, int *status) {
    constexpr int W = 4;  // 32-entry words per window
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
    const long long warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
    const long long chunk = ((static_cast<long long>(nnz) + warps - 1) / warps + 32 * W - 1) / (32 * W) * (32 * W);
    const long long K0 = warp * chunk;
    const long long K1 = K0 + chunk < nnz ? K0 + chunk : nnz;
    int bits = 0;
    if (K0 < K1) {
        long long r = 0, hi = m;  // first r in [0, m] with ro[r] >= K0
        while (r < hi) {
            const long long mid = (r + hi) >> 1;
            if (__ldg(ro + mid) < K0) r = mid + 1;
            else hi = mid;
        }
        for (long long K = K0; K < K1; K += 32 * W) {
            int c[W], p[W];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const long long k = K + 32 * j + lane;
                c[j] = k < K1 ? __ldg(ci + k) : 0;
                p[j] = (k < K1 && k > 0) ? __ldg(ci + k - 1) : 0;
            }
            unsigned starts[W] = {};  // bit i of word j: a row starts at nonzero K + 32 j + i
            for (;;) {
                const long long rr = r + lane;
                const long long s = rr <= m ? __ldg(ro + rr) : LLONG_MAX;
                const long long d = s - K;
                const bool in = d >= 0 && d < 32 * W;
#pragma unroll
                for (int j = 0; j < W; ++j)
                    starts[j] |= __reduce_or_sync(0xffffffffu, (in && (d >> 5) == j) ? 1u << (d & 31) : 0u);
                const int cnt = __popc(__ballot_sync(0xffffffffu, rr <= m && d < 32 * W));
                r += cnt;
                if (cnt < 32) break;
            }
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const long long k = K + 32 * j + lane;
                if (k < K1) {
                    if (c[j] < 0 || c[j] >= n) bits |= 8;
                    if (check_sorted && k > 0 && !((starts[j] >> lane) & 1u) && c[j] <= p[j]) bits |= 16;
                }
            }
        }
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    if (lane == 0 && bits) atomicOr(status, bits);
}

// ------------------------------------------------------------------------------------------
// COO input (the framework's COO view, Ch.4 Sec. "Implementing Sparse Data Structures"): row
// offsets of a row-sorted COO matrix, ro[r] = #{k : row_idx[k] < r} (a lower bound per row),
// so that (ro, col_idx, values) is the same matrix in CSR and every schedule applies
// unchanged.  A check pass ORs 1 into *status for a row index outside [0, m) and 2 for a
// decrease; the offsets are only meaningful when it stays 0.
__global__ void coo_check_kernel(int m, int nnz, const int *__restrict__ row_idx, int *status) {
    int bits = 0;
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < nnz;
         k += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int r = __ldg(row_idx + k);
        if (r < 0 || r >= m) bits |= 1;
        if (k > 0 && r < __ldg(row_idx + k - 1)) bits |= 2;
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0 && bits) atomicOr(status, bits);
}

__global__ void coo_offsets_kernel(int m, int nnz, const int *__restrict__ row_idx, int *__restrict__ ro) {
    for (long long r = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; r <= m;
         r += static_cast<long long>(gridDim.x) * blockDim.x) {
        long long lo = 0, hi = nnz;  // first k with row_idx[k] >= r
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (__ldg(row_idx + mid) < r)
                lo = mid + 1;
            else
                hi = mid;
        }
        ro[r] = static_cast<int>(lo);
    }
}

cudaError_t launch_coo_offsets(int m, int nnz, const int *row_idx, int *row_offsets, int *d_status,
                               cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    const long long cap = static_cast<long long>(current_sm_count()) * 16;
    if (nnz > 0) {
        long long b = (static_cast<long long>(nnz) + 255) / 256;
        coo_check_kernel<<<static_cast<int>(b < cap ? b : cap), 256, 0, stream>>>(m, nnz, row_idx, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    long long b = (static_cast<long long>(m) + 1 + 255) / 256;
    coo_offsets_kernel<<<static_cast<int>(b < cap ? b : cap), 256, 0, stream>>>(m, nnz, row_idx, row_offsets);
    return cudaGetLastError();
}

cudaError_t launch_validate(int m, int n, int nnz, const int *ro, const int *ci, int check_sorted, int *d_status,
                            cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    int blocks = static_cast<int>((static_cast<long long>(m) + 1 + 255) / 256);
    if (blocks > current_sm_count() * 16) blocks = current_sm_count() * 16;
    if (blocks < 1) blocks = 1;
    validate_offsets_kernel<<<blocks, 256, 0, stream>>>(m, nnz, ro, d_status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (m > 0 && nnz > 0) {
        // Warps of 128-entry windows, at least 16 windows each until the grid is full.
        long long wblocks = (static_cast<long long>(nnz) + 8 * 128 * 16 - 1) / (8 * 128 * 16);
        if (wblocks > current_sm_count() * 8) wblocks = current_sm_count() * 8;
        validate_columns_kernel<<<static_cast<int>(wblocks), 256, 0, stream>>>(m, n, nnz, ro, ci, check_sorted,
                                                                                d_status);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace lb
