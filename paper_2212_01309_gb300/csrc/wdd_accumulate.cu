// Phase accumulation on the SIMT cores in FP32 (the plain path):
//   H[v, k] += sum_b E[v, s_b] c_b[k],   E[v, s] = exp(-2 pi i (v_y s_y / S_y + v_x s_x / S_x))
// which is Eq. 14 restricted to the frames at hand (Algorithm 2: the subset of F_2D for
// each s built from the two 1-D DFT matrices).  The phase factor is never read from HBM: its
// exact integer index m = (v_y s_y mod S_y) * (lcm / S_y) + (v_x s_x mod S_x) * (lcm / S_x)
// (mod lcm) selects an entry of an lcm-long table of exp(-2 pi i m / lcm) built in FP64.
//
// Tiling: a CTA owns a 64 (v) x 64 (k) tile of H and streams the staged frames through shared
// memory in chunks of 16; each thread keeps a 4 x 4 block of complex accumulators.

#include "wdd_internal.h"

namespace wdd {

namespace {

constexpr int kTV = 64, kTK = 64, kTB = 16;

__global__ void __launch_bounds__(kThreads)
accumulate_fp32_kernel(const float* __restrict__ c, const int32_t* __restrict__ idx, int n,
                       int S, int Sy, int Sx, int K, int lcm, const float2* __restrict__ tw,
                       float2* __restrict__ H) {
    __shared__ __align__(16) float2 sE[kTB][kTV];
    __shared__ __align__(16) float sC[kTB][kTK];
    const int v0 = blockIdx.x * kTV;
    const int k0 = blockIdx.y * kTK;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int my = lcm / Sy, mx = lcm / Sx;

    // E generation: this thread fills column vv of sE for rows bb = ty0, ty0 + 4, ...
    const int vv = threadIdx.x % kTV;
    const int bq = threadIdx.x / kTV;  // 0..3
    const int vg = v0 + vv;
    const int vy = (vg < S) ? vg / Sx : 0;
    const int vx = (vg < S) ? vg % Sx : 0;

    float ar[4][4], ai[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { ar[i][j] = 0.f; ai[i][j] = 0.f; }

    for (int b0 = 0; b0 < n; b0 += kTB) {
        // coefficients chunk (coalesced along k)
        for (int t = threadIdx.x; t < kTB * kTK; t += blockDim.x) {
            int bb = t / kTK, kk = t % kTK;
            int b = b0 + bb, k = k0 + kk;
            sC[bb][kk] = (b < n && k < K) ? __ldg(c + (size_t)b * K + k) : 0.f;
        }
        // phase factors
#pragma unroll
        for (int q = 0; q < kTB / 4; ++q) {
            int bb = bq + 4 * q;
            int b = b0 + bb;
            float2 e = make_float2(0.f, 0.f);
            if (b < n && vg < S) {
                int s = __ldg(idx + b);
                int sy = s / Sx, sx = s - sy * Sx;
                int m = ((vy * sy) % Sy) * my + ((vx * sx) % Sx) * mx;
                if (m >= lcm) m -= lcm;
                e = __ldg(tw + m);
            }
            sE[bb][vv] = e;
        }
        __syncthreads();
#pragma unroll 4
        for (int bb = 0; bb < kTB; ++bb) {
            float4 e01 = *reinterpret_cast<const float4*>(&sE[bb][ty * 4]);
            float4 e23 = *reinterpret_cast<const float4*>(&sE[bb][ty * 4 + 2]);
            float4 cc = *reinterpret_cast<const float4*>(&sC[bb][tx * 4]);
            float er[4] = {e01.x, e01.z, e23.x, e23.z};
            float ei[4] = {e01.y, e01.w, e23.y, e23.w};
            float cv[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    ar[i][j] = fmaf(er[i], cv[j], ar[i][j]);
                    ai[i][j] = fmaf(ei[i], cv[j], ai[i][j]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int v = v0 + ty * 4 + i;
        if (v >= S) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int k = k0 + tx * 4 + j;
            if (k < K) {
                float2 h = H[(size_t)v * K + k];
                h.x += ar[i][j];
                h.y += ai[i][j];
                H[(size_t)v * K + k] = h;
            }
        }
    }
}

}  // namespace

cudaError_t launch_accumulate_fp32(const wdd_plan* P, const float* c, const int32_t* idx, int n,
                                   cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    dim3 grid((P->S + kTV - 1) / kTV, (P->K + kTK - 1) / kTK);
    accumulate_fp32_kernel<<<grid, kThreads, 0, st>>>(c, idx, n, P->S, P->Sy, P->Sx, P->K,
                                                      P->lcm, P->d_tw, P->d_H);
    return cudaGetLastError();
}

}  // namespace wdd
