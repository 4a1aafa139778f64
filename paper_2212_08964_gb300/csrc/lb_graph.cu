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

__global__ void frontier_degrees_kernel(int fsize, const int *__restrict__ frontier, const int *__restrict__ ro,
                                        int *__restrict__ deg) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < fsize;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int u = __ldg(frontier + i);
        deg[i] = __ldg(ro + u + 1) - __ldg(ro + u);
    }
}

// Relax edges [0, total) of the frontier; pre[i] = first edge of frontier vertex i.
__global__ void __launch_bounds__(kGraphThreads) relax_kernel(int n, int fsize, int iter, const int *__restrict__ frontier,
                                                              const int *__restrict__ pre, const int *__restrict__ ro,
                                                              const int *__restrict__ ci, const float *__restrict__ w,
                                                              float *dist, int *stamp, int *next, int *next_count) {
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
        if (nd < __int_as_float(old) && atomicMax(stamp + v, iter) < iter) next[atomicAdd(next_count, 1)] = v;
    }
}

}  // namespace

cudaError_t run_sssp(int n, int nnz, const int *ro, const int *ci, const float *w, int source, float *dist,
                     int *iterations, cudaStream_t st) {
    *iterations = 0;
    if (n <= 0) return cudaSuccess;
    // Workspace: two frontiers, stamps, degrees / their scan, scan scratch, the next count.
    const long long scratch = scan_scratch_ints(static_cast<long long>(n) + 1);
    const size_t ints = 4 * (static_cast<size_t>(n) + 1) + static_cast<size_t>(scratch) + 1;
    int *work = nullptr;
    cudaError_t e = dev_malloc_async(reinterpret_cast<void **>(&work), ints * sizeof(int), st);
    if (e != cudaSuccess) return e;
    int *f_cur = work;
    int *f_next = f_cur + n + 1;
    int *stamp = f_next + n + 1;
    int *pre = stamp + n + 1;
    int *sums = pre + n + 1;
    int *d_count = sums + scratch;
    int *h_count = nullptr;
    e = cudaMallocHost(reinterpret_cast<void **>(&h_count), sizeof(int));
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
    int fsize = 1;
    for (int iter = 1; e == cudaSuccess && fsize > 0 && iter <= n + 1; ++iter) {
        frontier_degrees_kernel<<<blocks(fsize), kGraphThreads, 0, st>>>(fsize, f_cur, ro, pre);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        // pre[fsize] = 0 then scan fsize + 1 entries: pre[fsize] is the frontier's edge count.
        if ((e = cudaMemsetAsync(pre + fsize, 0, sizeof(int), st)) != cudaSuccess) break;
        if ((e = exclusive_scan(pre, pre, static_cast<long long>(fsize) + 1, sums, st)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(d_count, 0, sizeof(int), st)) != cudaSuccess) break;
        // The edge count stays on the device; the relaxation reads it and strides over it.
        relax_kernel<<<sms * 16, kGraphThreads, 0, st>>>(n, fsize, iter, f_cur, pre, ro, ci, w, dist, stamp, f_next,
                                                         d_count);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(h_count, d_count, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        fsize = *h_count;
        int *t = f_cur;
        f_cur = f_next;
        f_next = t;
        *iterations = iter;
    }
    (void)nnz;
    if (h_count) cudaFreeHost(h_count);
    cudaError_t e2 = dev_free_async(work, st);
    return e != cudaSuccess ? e : e2;
}

}  // namespace lb
