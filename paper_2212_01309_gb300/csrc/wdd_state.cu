// Merging an exported accumulator into a plan (checkpoint/resume and partition merge).
//
// Live WDD is linear in the frames (Eq. 14): the accumulator H of a set of frames is the sum of
// the accumulators of any partition of it, and the hit counters add the same way (the merge by
// summation of partial results, Sect. 6.3).  So the state of a plan is its accumulator (read back
// with wdd_copy_array(WDD_ARRAY_ACCUM), which first accumulates any staged frames), its hit
// counters and its frame count; adding that state to a fresh plan of the same parameters resumes
// the acquisition, and adding the states of plans that saw disjoint frames gives the plan of
// all of them.

#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "wdd_internal.h"

namespace wdd {
namespace {

// H[t] += X[t]
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
    if (frames_seen < 0) return sfail(WDD_ERR_INVALID_ARG, "frames_seen must be non-negative");
    int64_t total = 0;
    for (int v = 0; v < P->S; ++v) total += hits[v];
    if (total != frames_seen)
        return sfail(WDD_ERR_INVALID_ARG, "hit counters do not add up to frames_seen");
    for (int v = 0; v < P->S; ++v)
        if ((uint64_t)P->hits[v] + hits[v] > 0xFFFFFFFFull)
            return sfail(WDD_ERR_INVALID_ARG, "hit counter overflow");
    const size_t n = (size_t)P->S * P->K;
    // order after every queued use of the accumulator
    cudaError_t e = cudaDeviceSynchronize();
    float2* tmp = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&tmp, 8 * n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(e == cudaErrorMemoryAllocation ? WDD_ERR_OUT_OF_MEMORY : WDD_ERR_CUDA,
                     std::string("merge buffer: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(tmp, accum, 8 * n, cudaMemcpyDefault);
    if (e == cudaSuccess) {
        const int64_t blocks = std::min<int64_t>(((int64_t)n + kThreads - 1) / kThreads, 152 * 32);
        add_accum_kernel<<<(unsigned)blocks, kThreads>>>(P->d_H, tmp, (int64_t)n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(tmp);
    if (e != cudaSuccess) return sfail(WDD_ERR_CUDA, std::string("merge: ") + cudaGetErrorString(e));
    for (int v = 0; v < P->S; ++v) {
        if (P->hits[v] == 0u && hits[v] != 0u) ++P->covered;
        P->hits[v] += hits[v];
    }
    P->frames_seen += frames_seen;
    return WDD_OK;
}
