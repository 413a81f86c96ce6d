// Merging an exported accumulator into a plan (checkpoint/resume and partition merge).
//
// Live WDD is linear in the frames (Eq. 14): the accumulator H of a set of frames is the sum of
// the accumulators of any partition of it, and the hit counters add the same way (the merge by
// summation of partial results, Sect. 6.3).  So the state of a plan is its accumulator (read back
// with wdd_copy_array(WDD_ARRAY_ACCUM), which first accumulates any staged frames), its hit
// counters and its frame count; adding that state to a fresh plan of the same parameters resumes
// the acquisition, and adding the states of plans that saw disjoint frames gives the plan of
// all of them.
//
// The addition is one kernel on the plan's stream that reads the exported accumulator where it
// lies (device memory, or pinned host memory over the host link), so a merge neither allocates
// nor waits for other work on the device.

#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "wdd_internal.h"

namespace wdd {
namespace {

// H[t] += X[t] over the S x K accumulator.
__global__ void add_accum_kernel(float2* __restrict__ H, const float2* __restrict__ X,
                                 int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = H[t], b = X[t];
        H[t] = make_float2(a.x + b.x, a.y + b.y);
    }
}

wdd_status sfail(wdd_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

}  // namespace
}  // namespace wdd

using namespace wdd;

wdd_status wdd_merge_state(wdd_plan* P, const void* accum, const uint32_t* hits,
                           int64_t frames_seen) {
    if (!P || !accum || !hits) return sfail(WDD_ERR_INVALID_ARG, "plan, accum or hits is NULL");
    if (P->finished)
        return sfail(WDD_ERR_STATE, "plan already finalized (wdd_reset it to take a state)");
    if (frames_seen < 0) return sfail(WDD_ERR_INVALID_ARG, "frames_seen must be non-negative");
    int64_t total = 0;
    for (int v = 0; v < P->S; ++v) total += hits[v];
    if (total != frames_seen)
        return sfail(WDD_ERR_INVALID_ARG, "hit counters do not add up to frames_seen");
    for (int v = 0; v < P->S; ++v)
        if ((uint64_t)P->hits[v] + hits[v] > 0xFFFFFFFFull)
            return sfail(WDD_ERR_INVALID_ARG, "hit counter overflow");
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, accum) != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    const float2* X = nullptr;
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)
        X = static_cast<const float2*>(accum);
    else if (attr.type == cudaMemoryTypeHost)
        X = static_cast<const float2*>(attr.devicePointer ? attr.devicePointer : accum);
    if (!X) return sfail(WDD_ERR_INVALID_ARG, "accum must be in device or pinned host memory");
    const int64_t n = (int64_t)P->S * P->K;
    const int64_t blocks = std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 16);
    // in stream order after everything the plan has enqueued (every use of the accumulator is
    // on the plan's stream); staged frames are added by a later flush, which commutes with this
    add_accum_kernel<<<(unsigned)blocks, kThreads, 0, P->stream>>>(P->d_H, X, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sfail(WDD_ERR_CUDA, std::string("merge: ") + cudaGetErrorString(e));
    ++P->launches_total;
    for (int v = 0; v < P->S; ++v) {
        if (P->hits[v] == 0u && hits[v] != 0u) ++P->covered;
        P->hits[v] += hits[v];
    }
    P->frames_seen += frames_seen;
    return WDD_OK;
}
