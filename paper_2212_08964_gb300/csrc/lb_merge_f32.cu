// Merge-path SpMV instances with float values (one translation unit per value type so the
// library compiles in parallel).
#include "lb_merge.cuh"

namespace lb {

cudaError_t launch_merge_f32(int mode, int threads, int ipt, const MergeArgs &a, cudaStream_t s, cudaEvent_t eb,
                             cudaEvent_t ea) {
    return dispatch_merge<float>(mode, threads, ipt, a, s, eb, ea);
}

cudaError_t prepare_merge_f32(int threads, int ipt) { return prepare_merge_plain<float>(threads, ipt); }

}  // namespace lb
