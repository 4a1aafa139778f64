// Merge-path SpMV instances with __nv_bfloat16 values (one translation unit per value type so the
// library compiles in parallel).
#include "lb_merge.cuh"

namespace lb {

cudaError_t launch_merge_bf16(int mode, int threads, int ipt, const MergeArgs &a, cudaStream_t s, cudaEvent_t eb,
                             cudaEvent_t ea) {
    return dispatch_merge<__nv_bfloat16>(mode, threads, ipt, a, s, eb, ea);
}

cudaError_t prepare_merge_bf16(int threads, int ipt) { return prepare_merge_plain<__nv_bfloat16>(threads, ipt); }

}  // namespace lb
