// lb_transpose.cu -- CSC plan (stable transpose), the value buckets, and the scans they need.
//
// The CSC view lets merge-path run over columns (Ch.4 Sec. "Implementing Sparse Data
// Structures": CSR, CSC and COO all map to atoms and tiles; Sec. "Merge-path load
// balancing": any format that can count atoms per tile).  The transpose must be stable --
// inside a column, entries keep increasing CSR index, hence increasing row -- so that the
// transposed SpMV sums every column in a fixed order.  It is built once per sparsity
// structure with a least-significant-digit radix sort of (column, CSR index) pairs: 8-bit
// digits, per-block digit counts, one exclusive scan over (digit, block), then a scatter in
// which every element's rank among equal digits of its block comes from warp match masks; a
// block orders its tile by digit in shared memory and writes it out digit run by digit run.
// Every step is a pure function of its input, so the plan is bit-exact and deterministic.
#include <cstdlib>
#include <cstring>

#include "lb_internal.cuh"

namespace lb {

// ------------------------------------------------------------------------------------------
// Exclusive scan of int arrays (three kernels; in place allowed).

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const int *in, long long n, int *sums) {
    __shared__ int s_w[kScanThreads / 32];
    const long long base = static_cast<long long>(blockIdx.x) * kScanChunk;
    int s = 0;
    for (int i = threadIdx.x; i < kScanChunk; i += kScanThreads) {
        const long long k = base + i;
        if (k < n) s += in[k];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += s_w[w];
        sums[blockIdx.x] = t;
    }
}

// Exclusive scan of `sums` in place by one block of 1024 threads.
__global__ void __launch_bounds__(1024) scan_sums_kernel(int *sums, int nb) {
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + tid;
        const int v = i < nb ? sums[i] : 0;
        int incl = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        int pre = 0;
        for (int w = 0; w < warp; ++w) pre += s_w[w];
        const int carry = s_carry;
        if (i < nb) sums[i] = carry + pre + incl - v;
        __syncthreads();
        if (tid == 1023) s_carry = carry + pre + incl;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int *in, int *out, long long n,
                                                                  const int *sums) {
    __shared__ int s_w[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long base = static_cast<long long>(blockIdx.x) * kScanChunk + static_cast<long long>(tid) * kScanItems;
    int v[kScanItems];
    int tot = 0;
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
        const long long k = base + u;
        v[u] = k < n ? in[k] : 0;
        tot += v[u];
    }
    int incl = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    int run = (sums != nullptr ? sums[blockIdx.x] : 0) + incl - tot;  // null: a single chunk
    for (int w = 0; w < warp; ++w) run += s_w[w];
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
        const long long k = base + u;
        if (k < n) out[k] = run;
        run += v[u];
    }
}

// Exclusive scan of n ints; `sums` needs ceil(n / 2048) ints of scratch.
cudaError_t exclusive_scan(const int *in, int *out, long long n, int *sums, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int nb = static_cast<int>((n + kScanChunk - 1) / kScanChunk);
    if (nb == 1) {  // one chunk: one block scans it, with no chunk sums
        scan_apply_kernel<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
        return cudaGetLastError();
    }
    scan_reduce_kernel<<<nb, kScanThreads, 0, st>>>(in, n, sums);
    scan_sums_kernel<<<1, 1024, 0, st>>>(sums, nb);
    scan_apply_kernel<<<nb, kScanThreads, 0, st>>>(in, out, n, sums);
    return cudaGetLastError();
}

long long scan_scratch_ints(long long n) { return (n + kScanChunk - 1) / kScanChunk + 1; }

// ------------------------------------------------------------------------------------------
// Radix sort of (key, value) pairs by key, stable.

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

__global__ void __launch_bounds__(kRsThreads) radix_hist_kernel(const int *keys, int n, int shift, int nblocks,
                                                                int *hist) {
    __shared__ int cnt[256];
    for (int d = threadIdx.x; d < 256; d += kRsThreads) cnt[d] = 0;
    __syncthreads();
    const long long base = static_cast<long long>(blockIdx.x) * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        const long long k = base + i;
        if (k < n) atomicAdd(&cnt[(keys[k] >> shift) & 255], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kRsThreads) hist[static_cast<long long>(d) * nblocks + blockIdx.x] = cnt[d];
}

// vals_in == nullptr means the identity (value = position); keys_out == nullptr skips the keys
// (the last pass needs only the values).  Each tile is ordered by digit in shared memory first
// (stable: in tile order within a digit), then written out run by run, so the stores of one
// digit's run are consecutive in memory.
__global__ void __launch_bounds__(kRsThreads) radix_scatter_kernel(const int *keys_in, const int *vals_in,
                                                                   int *keys_out, int *vals_out, int n, int shift,
                                                                   int nblocks, const int *offsets) {
    static_assert(kRsThreads == 256, "one thread per digit in the digit scan");
    __shared__ int s_key[kRsTile];
    __shared__ int s_val[kRsTile];
    __shared__ int wc[kRsWarps][256];
    __shared__ int cnt[256];    // digit counts, then the running local position of each digit
    __shared__ int lbase[256];  // where each digit's run starts in the tile
    __shared__ int goff[256];   // where it starts in the output
    __shared__ int wsum[kRsWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long base = static_cast<long long>(blockIdx.x) * kRsTile;
    cnt[tid] = 0;
    goff[tid] = offsets[static_cast<long long>(tid) * nblocks + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) wc[w][tid] = 0;
    __syncthreads();
    int key[kRsItems], val[kRsItems];
#pragma unroll
    for (int u = 0; u < kRsItems; ++u) {
        const long long p = base + static_cast<long long>(u) * kRsThreads + tid;
        const bool valid = p < n;
        key[u] = valid ? keys_in[p] : 0;
        val[u] = valid ? (vals_in ? vals_in[p] : static_cast<int>(p)) : 0;
        if (valid) atomicAdd(&cnt[(key[u] >> shift) & 255], 1);
    }
    __syncthreads();
    {
        // Exclusive scan of the tile's digit counts, one digit per thread.
        const int c = cnt[tid];
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int b = incl - c;
        for (int w = 0; w < warp; ++w) b += wsum[w];
        lbase[tid] = b;
        cnt[tid] = b;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int u = 0; u < kRsItems; ++u) {
        const long long p = base + static_cast<long long>(u) * kRsThreads + tid;
        const bool valid = p < n;
        const int d = valid ? ((key[u] >> shift) & 255) : (256 + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        const int count = __popc(peers);
        const bool leader = (31 - __clz(peers)) == lane;
        if (valid && leader) wc[warp][d] = count;
        __syncthreads();
        if (valid) {
            int pos = cnt[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wc[w][d];
            s_key[pos] = key[u];
            s_val[pos] = val[u];
        }
        __syncthreads();
        if (valid && leader) {
            atomicAdd(&cnt[d], count);
            wc[warp][d] = 0;
        }
        __syncthreads();
    }
    const long long left = static_cast<long long>(n) - base;
    const int tile_n = left < kRsTile ? static_cast<int>(left) : kRsTile;
    for (int i = tid; i < tile_n; i += kRsThreads) {
        const int k = s_key[i];
        const int d = (k >> shift) & 255;
        const long long gp = static_cast<long long>(goff[d]) + (i - lbase[d]);
        if (keys_out != nullptr) keys_out[gp] = k;
        vals_out[gp] = s_val[i];
    }
}

__global__ void iota_kernel(int *out, int n) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        out[i] = static_cast<int>(i);
}

__global__ void count_columns_kernel(const int *ci, int nnz, int *counts) {
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < nnz;
         k += static_cast<long long>(gridDim.x) * blockDim.x)
        atomicAdd(&counts[ci[k]], 1);
}

__global__ void gather_kernel(const int *src, const int *idx, int *dst, int n) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        dst[i] = src[idx[i]];
}

// ------------------------------------------------------------------------------------------

cudaError_t build_transpose(int m, int n, int nnz, const int *ro, const int *ci, int num_tiles, int tile_items,
                            const int *tile_row, const int *tile_nz, TransposeOut out, cudaStream_t st) {
    (void)m;
    cudaError_t e;
    const int sms = current_sm_count();
    // Column offsets: counts, then an exclusive scan over n + 1 entries (co[n] = nnz).
    if ((e = cudaMemsetAsync(out.col_offsets, 0, (static_cast<size_t>(n) + 1) * sizeof(int), st)) != cudaSuccess)
        return e;
    if (nnz == 0) return cudaSuccess;
    const int nblocks = static_cast<int>((static_cast<long long>(nnz) + kRsTile - 1) / kRsTile);
    const long long hist_n = 256ll * nblocks;
    long long scan_n = hist_n > static_cast<long long>(n) + 1 ? hist_n : static_cast<long long>(n) + 1;
    const size_t ints = static_cast<size_t>(nnz) * 3 + static_cast<size_t>(hist_n) +
                        static_cast<size_t>(scan_scratch_ints(scan_n));
    int *work = nullptr;
    if ((e = dev_malloc_async(reinterpret_cast<void **>(&work), ints * sizeof(int), st)) != cudaSuccess) return e;
    int *rowid = work;
    int *keys_a = rowid + nnz;
    int *vals_a = keys_a + nnz;
    int *hist = vals_a + nnz;
    int *sums = hist + hist_n;
    int *keys_b = out.row_idx;  // row_idx is written last, so it can hold keys meanwhile

    const int grid = sms * 8;
    count_columns_kernel<<<grid, 256, 0, st>>>(ci, nnz, out.col_offsets);
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    if ((e = exclusive_scan(out.col_offsets, out.col_offsets, static_cast<long long>(n) + 1, sums, st)) !=
        cudaSuccess)
        goto done;
    if ((e = launch_tile_row_ids(num_tiles, tile_items, tile_row, tile_nz, ro + 1, rowid, st)) != cudaSuccess)
        goto done;
    {
        int bits = 0;
        while (bits < 31 && (1ll << bits) < n) ++bits;
        const int passes = (bits + 7) / 8;
        if (passes == 0) {
            iota_kernel<<<grid, 256, 0, st>>>(out.perm, nnz);
        } else {
            const int *kin = ci;
            const int *vin = nullptr;
            for (int p = 0; p < passes; ++p) {
                int *kout = (p + 1 == passes) ? nullptr : ((p & 1) ? keys_b : keys_a);  // last pass: values only
                int *vout = ((passes - 1 - p) % 2 == 0) ? out.perm : vals_a;
                radix_hist_kernel<<<nblocks, kRsThreads, 0, st>>>(kin, nnz, 8 * p, nblocks, hist);
                if ((e = exclusive_scan(hist, hist, hist_n, sums, st)) != cudaSuccess) goto done;
                radix_scatter_kernel<<<nblocks, kRsThreads, 0, st>>>(kin, vin, kout, vout, nnz, 8 * p, nblocks, hist);
                if ((e = cudaGetLastError()) != cudaSuccess) goto done;
                kin = kout;
                vin = vout;
            }
        }
        gather_kernel<<<grid, 256, 0, st>>>(rowid, out.perm, out.row_idx, nnz);
        e = cudaGetLastError();
    }
done:
    cudaError_t e2 = dev_free_async(work, st);
    return e != cudaSuccess ? e : e2;
}

// ------------------------------------------------------------------------------------------
// Bringing CSR-ordered data into CSC order, every call, without random HBM accesses.
//
// The transposed product needs, for CSC entry p, data of CSR entry perm[p]: a random
// permutation of an array far larger than L2.  Gathering it directly costs one DRAM sector
// per nonzero.  Instead the CSC entries are cut into buckets of 2^shift consecutive entries
// (each bucket's data fit comfortably in L2), and each call (1) streams the CSR-ordered data
// once into bucket order -- CSR entries of one bucket keep their CSR order, so every bucket
// receives one sequential stream of writes -- and (2) lets the transposed kernel gather from
// the bucket being worked on, which stays resident in L2 while the persistent CTAs sweep
// through it.  Both maps are fixed per structure, so results stay deterministic.

int value_bucket_shift(long long nnz) {
    int shift = 23;  // 8M entries: 32 MB of FP32 values
    // LBSPMV_VALUE_BUCKET_SHIFT (8..30) overrides the bucket size, so tests can exercise
    // many buckets on small matrices.
    if (const char *env = getenv("LBSPMV_VALUE_BUCKET_SHIFT")) {
        const int v = atoi(env);
        if (v >= 8 && v <= 30) shift = v;
    }
    while (shift < 30 && ((nnz + (1ll << shift) - 1) >> shift) > 256) ++shift;
    return shift;
}

__global__ void scatter_inverse_kernel(const int *src, int *dst, int n) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        dst[src[i]] = static_cast<int>(i);
}

cudaError_t build_value_buckets(int nnz, int shift, const int *perm, int *bucket_pos, int *bucket_perm,
                                cudaStream_t st) {
    if (nnz <= 0) return cudaSuccess;
    cudaError_t e;
    const int nblocks = static_cast<int>((static_cast<long long>(nnz) + kRsTile - 1) / kRsTile);
    const long long hist_n = 256ll * nblocks;
    const size_t ints = 2 * static_cast<size_t>(nnz) + static_cast<size_t>(hist_n) +
                        static_cast<size_t>(scan_scratch_ints(hist_n));
    int *work = nullptr;
    if ((e = dev_malloc_async(reinterpret_cast<void **>(&work), ints * sizeof(int), st)) != cudaSuccess) return e;
    int *pinv = work;            // CSR entry -> CSC position
    int *order = pinv + nnz;     // bucket order -> CSR entry
    int *hist = order + nnz;
    int *sums = hist + hist_n;
    const int grid = current_sm_count() * 8;
    scatter_inverse_kernel<<<grid, 256, 0, st>>>(perm, pinv, nnz);
    // One stable counting pass on the bucket number pinv >> shift (< 256 buckets).
    radix_hist_kernel<<<nblocks, kRsThreads, 0, st>>>(pinv, nnz, shift, nblocks, hist);
    if ((e = cudaGetLastError()) == cudaSuccess) e = exclusive_scan(hist, hist, hist_n, sums, st);
    if (e == cudaSuccess) {
        radix_scatter_kernel<<<nblocks, kRsThreads, 0, st>>>(pinv, nullptr, nullptr, order, nnz, shift, nblocks, hist);
        scatter_inverse_kernel<<<grid, 256, 0, st>>>(order, bucket_pos, nnz);  // bucket_pos[order[q]] = q
        gather_kernel<<<grid, 256, 0, st>>>(bucket_pos, perm, bucket_perm, nnz);  // bucket_perm[p] = bucket_pos[perm[p]]
        e = cudaGetLastError();
    }
    cudaError_t e2 = dev_free_async(work, st);
    return e != cudaSuccess ? e : e2;
}

}  // namespace lb
