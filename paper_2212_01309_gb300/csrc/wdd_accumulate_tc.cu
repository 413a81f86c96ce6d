// Tensor-core phase accumulation (split FP16 precision): not built yet.
#include "wdd_internal.h"

namespace wdd {

bool split_path_available() { return false; }

cudaError_t prepare_split_kernels() { return cudaSuccess; }

cudaError_t launch_accumulate_split(const wdd_plan*, const float*, const int32_t*, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace wdd
