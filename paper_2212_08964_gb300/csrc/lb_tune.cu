// lb_tune.cu -- measured choice of schedule and launch shape (the autotuner's timing core).
//
// The dissertation picks a schedule by a fixed rule of matrix size (Ch.4 Sec. "Improved
// Performance Response": merge-path unless rows or columns < 500 and nonzeros < 10000).  A
// rule cannot see row-length skew or the hardware, so the autotuner measures instead: every
// candidate schedule and launch shape runs y = A x on the caller's matrix, timed with CUDA
// events on the caller's stream, and the candidates come back sorted by time.  The host side
// (shape classes, the table of winners) lives with the Python binding.
#include <algorithm>
#include <vector>

#include "lb_internal.cuh"

namespace {

struct Candidate {
    lb_schedule s;
    lb_tuning t;
};

// Every schedule and launch shape this library implements.
std::vector<Candidate> all_candidates() {
    std::vector<Candidate> c;
    const int merge[][2] = {{256, 8}, {128, 16}, {256, 16}, {384, 8}, {512, 8}};
    for (const auto &mp : merge) c.push_back({LB_SCHED_MERGE_PATH, {mp[0], mp[1], 0}});
    c.push_back({LB_SCHED_THREAD_MAPPED, {0, 0, 0}});
    c.push_back({LB_SCHED_WARP_MAPPED, {0, 0, 32}});
    for (int gs : {4, 8, 16}) c.push_back({LB_SCHED_GROUP_MAPPED, {0, 0, gs}});
    for (int th : {128, 256}) c.push_back({LB_SCHED_BLOCK_MAPPED, {th, 0, 0}});
    c.push_back({LB_SCHED_NONZERO_SPLIT, {0, 0, 0}});
    return c;
}

// Mean milliseconds of `reps` calls of fn, after one untimed call; events on `stream`.
template <typename F>
cudaError_t time_calls(F fn, int reps, cudaStream_t stream, float *ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    lb_status st = LB_OK;
    if (e == cudaSuccess) st = fn();
    if (e == cudaSuccess && st == LB_OK) e = cudaEventRecord(a, stream);
    for (int r = 0; r < reps && e == cudaSuccess && st == LB_OK; ++r) st = fn();
    if (e == cudaSuccess && st == LB_OK) e = cudaEventRecord(b, stream);
    if (e == cudaSuccess && st == LB_OK) e = cudaEventSynchronize(b);
    float total = 0.f;
    if (e == cudaSuccess && st == LB_OK) e = cudaEventElapsedTime(&total, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st != LB_OK && e == cudaSuccess) e = cudaErrorUnknown;
    *ms = total / static_cast<float>(reps);
    return e;
}

}  // namespace

extern "C" int lb_tune_candidates(void) { return static_cast<int>(all_candidates().size()); }

extern "C" lb_status lb_tune(int m, int n, int nnz, const int *row_offsets, const int *col_idx, const void *values,
                             lb_dtype vdt, const float *x, float *y, int reps, lb_tune_result *results, int capacity,
                             int *count, cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!count || !results || capacity < 0 || reps <= 0) return LB_ERR_INVALID_ARG;
    *count = 0;
    if (m <= 0 || n <= 0 || nnz <= 0 || !row_offsets || !col_idx || !values || !x || !y) return LB_ERR_INVALID_ARG;
    if (vdt != LB_F32 && vdt != LB_BF16 && vdt != LB_F16) return LB_ERR_INVALID_ARG;
    std::vector<lb_tune_result> out;
    for (const Candidate &c : all_candidates()) {
        lb_plan *p = nullptr;
        lb_status st = lb_plan_create(m, n, nnz, row_offsets, c.s, &c.t, stream, &p);
        if (st == LB_ERR_INVALID_ARG) continue;  // shape not applicable
        if (st != LB_OK) return st;
        float ms = 0.f;
        cudaError_t e =
            time_calls([&]() { return lb_spmv_planned(p, col_idx, values, vdt, x, y, stream); }, reps, stream, &ms);
        lb_schedule rs;
        lb_tuning rt;
        lb_plan_info(p, &rs, &rt, nullptr, nullptr);
        lb_plan_destroy(p);
        if (e != cudaSuccess) return LB_ERR_CUDA;
        out.push_back({rs, rt, ms});
    }
    std::stable_sort(out.begin(), out.end(),
                     [](const lb_tune_result &a, const lb_tune_result &b) { return a.ms < b.ms; });
    const int k = std::min(capacity, static_cast<int>(out.size()));
    for (int i = 0; i < k; ++i) results[i] = out[i];
    *count = k;
    return LB_OK;
}

extern "C" lb_status lb_tune_batched(int count_m, const int *h_m, const int *h_n, const int *h_nnz,
                                     const int *row_offsets_concat, const int *col_idx_concat,
                                     const void *values_concat, lb_dtype vdt, const float *x_concat,
                                     float *y_concat, int reps, lb_tune_result *results, int capacity, int *count,
                                     cudaStream_t stream) {
    LB_NVTX_RANGE();
    if (!count || !results || capacity < 0 || reps <= 0) return LB_ERR_INVALID_ARG;
    *count = 0;
    if (count_m <= 0 || !h_m || !h_n || !h_nnz || !row_offsets_concat || !col_idx_concat || !values_concat ||
        !x_concat || !y_concat)
        return LB_ERR_INVALID_ARG;
    std::vector<lb_tune_result> out;
    std::vector<Candidate> cands;
    cands.push_back({LB_SCHED_THREAD_MAPPED, lb_tuning{0, 0, 0}});
    for (const Candidate &c : all_candidates())
        if (c.s == LB_SCHED_MERGE_PATH) cands.push_back(c);  // the batch schedules: rows, or one merge path
    for (const Candidate &c : cands) {
        lb_batched_plan *p = nullptr;
        lb_status st = lb_batched_plan_create(count_m, h_m, h_n, h_nnz, row_offsets_concat, c.s, &c.t, stream, &p);
        if (st != LB_OK) return st;
        float ms = 0.f;
        cudaError_t e = time_calls(
            [&]() { return lb_spmv_batched(p, col_idx_concat, values_concat, vdt, x_concat, y_concat, stream); }, reps,
            stream, &ms);
        lb_batched_plan_destroy(p);
        if (e != cudaSuccess) return LB_ERR_CUDA;
        out.push_back({c.s, c.t, ms});
    }
    std::stable_sort(out.begin(), out.end(),
                     [](const lb_tune_result &a, const lb_tune_result &b) { return a.ms < b.ms; });
    const int k = std::min(capacity, static_cast<int>(out.size()));
    for (int i = 0; i < k; ++i) results[i] = out[i];
    *count = k;
    return LB_OK;
}
