// Merge-path SpMV instances with __half values (one translation unit per value type so the
// library compiles in parallel).
#include "lb_merge.cuh"

namespace lb {

cudaError_t launch_merge_f16(int mode, int threads, int ipt, const MergeArgs &a, cudaStream_t s, cudaEvent_t eb,
                             cudaEvent_t ea) {
    return dispatch_merge<__half>(mode, threads, ipt, a, s, eb, ea);
}

cudaError_t prepare_merge_f16(int threads, int ipt) { return prepare_merge_plain<__half>(threads, ipt); }

}  // namespace lb
