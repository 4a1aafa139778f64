// lb_graph.cu -- single-source shortest paths (and BFS) over a CSR graph on the same
// load-balancing machinery.
//
// The dissertation expresses SSSP with its load-balanced schedules (Ch.4 Sec. "Application
// Space", the SSSP listing): every edge of the current frontier is an atom; relaxing it
// computes the neighbour's tentative distance, lowers the neighbour's distance with an
// atomic minimum, and adds the neighbour to the next frontier when the distance dropped; the
// host loops until the frontier is empty (one synchronization per iteration, to read the next
// frontier's size).  Here the frontier's edges are split evenly over
// the threads (the work-oriented schedule applied to the frontier): the frontier vertices'
// degrees are scanned, and thread e relaxes edge e, finding its vertex by a binary search
// over the scan.  A vertex enters the next frontier once per iteration (a stamp with the
// iteration number, raised atomically).  Distances are FP32; they are non-negative, so their
// bit patterns order like the values and an integer atomic minimum applies.  The final
// distances are the fixpoint dist[v] = min over edges (u, v) of dist[u] + w(u, v), the same
// whatever order the relaxations run in.
//
// With weights, the frontier is split by distance (the near-far method: Davidson, Baxter,
// Garland and Owens, "Work-efficient parallel GPU methods for single-source shortest paths",
// IPDPS 2014): a vertex whose new distance lies below the current split point joins the next
// frontier; one at or beyond it is only marked far.  When the near frontier runs empty, the
// split point advances by delta and the marked vertices below it form the next frontier (a
// pass over all vertices); the split jumps to the smallest marked distance when no marked
// vertex lies below it.  Vertices are thus mostly relaxed once their distance is near final,
// instead of once per improvement as in the plain frontier loop.  delta is the mean edge
// weight times 8 over the mean degree (the cited paper's rule has 32; 8 relaxed the 4M-vertex
// power-law graph fastest, fewer buckets costing more re-relaxations and more buckets more
// iterations); unit weights (BFS) use no split, one level per iteration.
#include <cmath>
#include <cstring>
#include <limits>

#include "lb_internal.cuh"

namespace lb {

namespace {

constexpr int kGraphThreads = 256;
constexpr unsigned kInfBits = 0x7f800000u;  // +inf

__global__ void sssp_init_kernel(int n, int source, float *dist, int *stamp, int *frontier) {
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < n;
         v += static_cast<long long>(gridDim.x) * blockDim.x) {
        dist[v] = v == source ? 0.f : __uint_as_float(kInfBits);
        stamp[v] = v == source ? 0 : -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) frontier[0] = source;
}

// deg[i] = out-degree of frontier vertex i, deg[fsize] = 0 (the scan's last entry becomes the
// edge count), and the next frontier's counter cleared for the relaxation that follows.
__global__ void frontier_degrees_kernel(int fsize, const int *__restrict__ frontier, const int *__restrict__ ro,
                                        int *__restrict__ deg, int *__restrict__ next_count) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < fsize;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int u = __ldg(frontier + i);
        deg[i] = __ldg(ro + u + 1) - __ldg(ro + u);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        deg[fsize] = 0;
        *next_count = 0;
    }
}

// Relax edges [0, total) of the frontier; pre[i] = first edge of frontier vertex i.  A
// neighbour whose distance drops below `split` joins the next frontier; one whose distance
// drops to `split` or beyond is marked far.
__global__ void __launch_bounds__(kGraphThreads) relax_kernel(int n, int fsize, int iter, float split,
                                                              const int *__restrict__ frontier,
                                                              const int *__restrict__ pre, const int *__restrict__ ro,
                                                              const int *__restrict__ ci, const float *__restrict__ w,
                                                              float *dist, int *stamp, int *far, int *next,
                                                              int *next_count) {
    const long long total = __ldg(pre + fsize);  // the frontier's edge count (end of the scan)
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        int lo = 0, hi = fsize - 1;  // last i with pre[i] <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(pre + mid) <= e)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int u = __ldg(frontier + lo);
        const long long k = __ldg(ro + u) + (e - __ldg(pre + lo));
        const int v = __ldg(ci + k);
        if (!LB_IN_RANGE(v, n)) continue;
        const float nd = dist[u] + (w ? __ldg(w + k) : 1.f);
        const int old = atomicMin(reinterpret_cast<int *>(dist) + v, __float_as_int(nd));
        if (nd < __int_as_float(old)) {
            if (!(nd < split))
                far[v] = 1;
            else if (atomicMax(stamp + v, iter) < iter)
                next[atomicAdd(next_count, 1)] = v;
        }
    }
}

// The next frontier from the far marks: vertices marked far whose distance lies below
// `split` (unmarked, stamped with `iter`); the others stay marked, counted in cnt[1], their
// smallest distance (as bits: distances are non-negative) in cnt[2].
__global__ void far_split_kernel(int n, int iter, float split, const float *dist, int *stamp, int *far, int *next,
                                 int *cnt) {
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < n;
         v += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (!far[v]) continue;
        const float d = dist[v];
        if (d < split) {
            far[v] = 0;
            if (atomicMax(stamp + v, iter) < iter) next[atomicAdd(cnt, 1)] = static_cast<int>(v);
        } else {
            atomicAdd(cnt + 1, 1);
            atomicMin(cnt + 2, __float_as_int(d));
        }
    }
}

// Sum of the weights (for delta), in double: block sums added atomically.
__global__ void weight_sum_kernel(long long nnz, const float *__restrict__ w, double *sum) {
    __shared__ double part[kGraphThreads / 32];
    double s = 0.0;
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < nnz;
         k += static_cast<long long>(gridDim.x) * blockDim.x)
        s += static_cast<double>(__ldg(w + k));
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kGraphThreads / 32; ++i) t += part[i];
        atomicAdd(sum, t);
    }
}

}  // namespace

cudaError_t run_sssp(int n, int nnz, const int *ro, const int *ci, const float *w, int source, float *dist,
                     int *iterations, cudaStream_t st) {
    *iterations = 0;
    if (n <= 0) return cudaSuccess;
    // Workspace: two frontiers, stamps, far marks, degrees / their scan, scan scratch, three
    // counters and the weight sum (a double, 8-byte aligned).
    const long long scratch = scan_scratch_ints(static_cast<long long>(n) + 1);
    const size_t ints = 5 * (static_cast<size_t>(n) + 1) + static_cast<size_t>(scratch) + 4 + 4;
    int *work = nullptr;
    cudaError_t e = dev_malloc_async(reinterpret_cast<void **>(&work), ints * sizeof(int), st);
    if (e != cudaSuccess) return e;
    int *f_cur = work;
    int *f_next = f_cur + n + 1;
    int *stamp = f_next + n + 1;
    int *far = stamp + n + 1;
    int *pre = far + n + 1;
    int *sums = pre + n + 1;
    int *d_cnt = sums + scratch;  // [0] next frontier size, [1] far vertices left, [2] their min distance bits
    double *d_wsum = reinterpret_cast<double *>(work + ((static_cast<size_t>(d_cnt - work) + 4 + 1) & ~size_t{1}));
    int *h_cnt = nullptr;
    e = cudaMallocHost(reinterpret_cast<void **>(&h_cnt), 4 * sizeof(int) + sizeof(double));
    const int sms = current_sm_count();
    auto blocks = [&](long long items) {
        long long b = (items + kGraphThreads - 1) / kGraphThreads;
        const long long cap = static_cast<long long>(sms) * 16;
        return static_cast<int>(b < 1 ? 1 : (b > cap ? cap : b));
    };
    if (e == cudaSuccess) {
        sssp_init_kernel<<<blocks(n), kGraphThreads, 0, st>>>(n, source, dist, stamp, f_cur);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(far, 0, (static_cast<size_t>(n) + 1) * sizeof(int), st);
    // The split point: none for unit weights; otherwise delta = mean weight * 8 / mean degree.
    float split = std::numeric_limits<float>::infinity(), delta = split;
    if (e == cudaSuccess && w != nullptr && nnz > 0) {
        double *h_sum = reinterpret_cast<double *>(h_cnt + 4);
        e = cudaMemsetAsync(d_wsum, 0, sizeof(double), st);
        if (e == cudaSuccess) {
            weight_sum_kernel<<<blocks(nnz), kGraphThreads, 0, st>>>(nnz, w, d_wsum);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_sum, d_wsum, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            const double d = (*h_sum / nnz) * 8.0 / (static_cast<double>(nnz) / n);
            if (d > 0.0 && d < 1e30) delta = static_cast<float>(d), split = delta;
        }
    }
    const bool split_on = std::isfinite(split);
    int fsize = 1, tick = 0;
    const long long tick_limit = 4ll * (static_cast<long long>(n) + 16);  // host-side guard
    while (e == cudaSuccess && tick < tick_limit) {
        // Near iterations: relax the frontier until no distance below the split drops.
        while (e == cudaSuccess && fsize > 0 && tick < tick_limit) {
            ++tick;
            frontier_degrees_kernel<<<blocks(fsize), kGraphThreads, 0, st>>>(fsize, f_cur, ro, pre, d_cnt);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            // Scan fsize + 1 entries (pre[fsize] = 0): pre[fsize] is the frontier's edge count.
            if ((e = exclusive_scan(pre, pre, static_cast<long long>(fsize) + 1, sums, st)) != cudaSuccess) break;
            // The edge count stays on the device; the relaxation reads it and strides over it.
            relax_kernel<<<sms * 16, kGraphThreads, 0, st>>>(n, fsize, tick, split, f_cur, pre, ro, ci, w, dist, stamp,
                                                             far, f_next, d_cnt);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(h_cnt, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
            fsize = h_cnt[0];
            int *t = f_cur;
            f_cur = f_next;
            f_next = t;
            ++*iterations;
        }
        if (e != cudaSuccess || !split_on) break;
        // Advance the split; the far vertices below it form the next frontier.  With none below
        // it, jump to the smallest far distance; with none left at all, done.
        for (;;) {
            split += delta;
            ++tick;
            // Counts to zero; the minimum to the bits 0x7f7f7f7f (about 3.4e38, above any finite
            // distance the far marks can hold).
            if ((e = cudaMemsetAsync(d_cnt, 0, 2 * sizeof(int), st)) != cudaSuccess) break;
            if ((e = cudaMemsetAsync(d_cnt + 2, 0x7f, sizeof(int), st)) != cudaSuccess) break;
            far_split_kernel<<<blocks(n), kGraphThreads, 0, st>>>(n, tick, split, dist, stamp, far, f_cur, d_cnt);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(h_cnt, d_cnt, 3 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
            fsize = h_cnt[0];
            if (fsize > 0 || h_cnt[1] == 0) break;
            float far_min;
            std::memcpy(&far_min, &h_cnt[2], sizeof(float));
            if (far_min >= split) split = far_min;  // the loop adds delta again
        }
        if (e != cudaSuccess || fsize == 0) break;
    }
    if (h_cnt) cudaFreeHost(h_cnt);
    cudaError_t e2 = dev_free_async(work, st);
    return e != cudaSuccess ? e : e2;
}

}  // namespace lb
