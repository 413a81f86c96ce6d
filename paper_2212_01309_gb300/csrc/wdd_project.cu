// Frame ingest and projection onto the reduced basis (Sect. 5 operator H; Algorithm 2, step 1):
//   c_b[k] = component_k( sum_{i,j} By[i, ly_k] I_b[i, j] Bx[j, lx_k] )
// computed separably: T = I Bx per row block, then By^T T.  Frames are read in their stored
// type (uint16, float32, float64) straight from device memory or pinned host memory with 16-byte
// vector loads and converted to FP32 in registers; nothing is staged in HBM.
//
// The scan indices of the launch arrive as a by-value parameter block and are stored next to
// the staged coefficients for the phase accumulation, so a push needs no host-to-device copy.
//
// For the split-precision path the kernel also keeps a running maximum of |c| per coefficient
// (float bits compared as unsigned integers), from which the accumulation picks its scales.
//
// Grid: (frames, row blocks).  Each CTA reduces kProjRows detector rows.  When a frame spans more
// than one row block, every CTA writes its partial coefficients to a scratch slot and the last
// CTA to arrive (per-frame arrival counter) adds the partials in row-block order, so the result
// does not depend on CTA scheduling.

#include "wdd_internal.h"

namespace wdd {

namespace {

template <typename FT>
__device__ __forceinline__ float to_f(FT v) { return (float)v; }

// Loads `count` consecutive frame elements starting at src into dst (float), vectorised when
// src is 16-byte aligned.
template <typename FT>
__device__ __forceinline__ void load_rows(const FT* __restrict__ src, float* dst, int count) {
    constexpr int V = 16 / sizeof(FT);
    const bool aligned = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && (count % V == 0);
    if (aligned) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        int nv = count / V;
        for (int t = threadIdx.x; t < nv; t += blockDim.x) {
            uint4 q = __ldg(s4 + t);
            const FT* e = reinterpret_cast<const FT*>(&q);
#pragma unroll
            for (int u = 0; u < V; ++u) dst[t * V + u] = to_f(e[u]);
        }
    } else {
        for (int t = threadIdx.x; t < count; t += blockDim.x) dst[t] = to_f(src[t]);
    }
}

template <typename FT, bool CPLX>
__global__ void __launch_bounds__(kThreads)
project_kernel(const FT* __restrict__ frames, int Ny, int Nx, int Ly, int Lx, int K,
               const float2* __restrict__ By, const float2* __restrict__ Bx,
               const int2* __restrict__ ktab, float* __restrict__ cpart,
               unsigned* __restrict__ count, float* __restrict__ c_out, int nrb,
               const IndexBlock ids, int32_t* __restrict__ idx_out, unsigned* __restrict__ colmax) {
    extern __shared__ float sm[];
    const int b = blockIdx.x;
    const int rb = blockIdx.y;
    const int i0 = rb * kProjRows;
    const int rows = min(kProjRows, Ny - i0);
    constexpr int CW = CPLX ? 2 : 1;  // floats per basis value

    float* sBx = sm;                              // Nx * Lx * CW
    float* sI = sBx + (size_t)Nx * Lx * CW;       // kProjRows * Nx
    float* sT = sI + (size_t)kProjRows * Nx;      // kProjRows * Lx * CW
    if (rb == 0 && threadIdx.x == 0) idx_out[b] = ids.s[b];  // scan index for the accumulation

    for (int t = threadIdx.x; t < Nx * Lx; t += blockDim.x) {
        float2 v = Bx[t];
        if (CPLX) { sBx[2 * t] = v.x; sBx[2 * t + 1] = v.y; }
        else sBx[t] = v.x;
    }
    const FT* src = frames + (size_t)b * Ny * Nx + (size_t)i0 * Nx;
    load_rows<FT>(src, sI, rows * Nx);
    __syncthreads();

    // T[r][lx] = sum_j I[r][j] Bx[j][lx]
    for (int t = threadIdx.x; t < rows * Lx; t += blockDim.x) {
        int r = t / Lx, lx = t % Lx;
        const float* ir = sI + (size_t)r * Nx;
        if (CPLX) {
            float ar = 0.f, ai = 0.f;
            for (int j = 0; j < Nx; ++j) {
                float x = ir[j];
                ar = fmaf(x, sBx[2 * (j * Lx + lx)], ar);
                ai = fmaf(x, sBx[2 * (j * Lx + lx) + 1], ai);
            }
            sT[2 * t] = ar;
            sT[2 * t + 1] = ai;
        } else {
            float a = 0.f;
            for (int j = 0; j < Nx; ++j) a = fmaf(ir[j], sBx[j * Lx + lx], a);
            sT[t] = a;
        }
    }
    __syncthreads();

    // partial c[k] over this CTA's rows: component of sum_r By[i0+r][ly] T[r][lx]
    float* dst = (nrb == 1) ? (c_out + (size_t)b * K) : (cpart + ((size_t)b * nrb + rb) * K);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        int2 e = ktab[k];
        int ly = e.x / Lx, lx = e.x % Lx;
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) {
            float2 by = __ldg(By + (size_t)(i0 + r) * Ly + ly);
            if (CPLX) {
                float tr = sT[2 * (r * Lx + lx)], ti = sT[2 * (r * Lx + lx) + 1];
                // (by.x + i by.y)(tr + i ti): real part or imaginary part
                acc = (e.y == 0) ? fmaf(by.x, tr, fmaf(-by.y, ti, acc))
                                 : fmaf(by.x, ti, fmaf(by.y, tr, acc));
            } else {
                acc = fmaf(by.x, sT[r * Lx + lx], acc);
            }
        }
        dst[k] = acc;
        if (nrb == 1 && colmax) atomicMax(colmax + k, __float_as_uint(fabsf(acc)));
    }
    if (nrb == 1) return;

    // deterministic cross-CTA reduction: the last CTA of frame b adds partials in order
    __shared__ unsigned s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(count + b, 1u);
        s_last = (prev == (unsigned)(nrb - 1)) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float acc = 0.f;
        for (int q = 0; q < nrb; ++q) acc += __ldcg(cpart + ((size_t)b * nrb + q) * K + k);
        c_out[(size_t)b * K + k] = acc;
        if (colmax) atomicMax(colmax + k, __float_as_uint(fabsf(acc)));
    }
    if (threadIdx.x == 0) count[b] = 0u;  // ready for the next launch (stream ordered)
}

template <typename FT>
cudaError_t launch_typed(const wdd_plan* P, const FT* frames, int n, const IndexBlock& ids,
                         float* c_out, int32_t* idx_out, cudaStream_t st) {
    dim3 grid(n, P->rb);
    int CW = P->complex_basis ? 2 : 1;
    size_t smem = sizeof(float) * ((size_t)P->Nx * P->Lx * CW + (size_t)kProjRows * P->Nx +
                                   (size_t)kProjRows * P->Lx * CW);
    if (P->complex_basis) {
        project_kernel<FT, true><<<grid, kThreads, smem, st>>>(
            frames, P->Ny, P->Nx, P->Ly, P->Lx, P->K, P->d_By32, P->d_Bx32, P->d_ktab,
            P->d_cpart, P->d_count, c_out, P->rb, ids, idx_out, P->d_colmax);
    } else {
        project_kernel<FT, false><<<grid, kThreads, smem, st>>>(
            frames, P->Ny, P->Nx, P->Ly, P->Lx, P->K, P->d_By32, P->d_Bx32, P->d_ktab,
            P->d_cpart, P->d_count, c_out, P->rb, ids, idx_out, P->d_colmax);
    }
    return cudaGetLastError();
}

template <typename FT>
cudaError_t prepare_typed() {
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(project_kernel<FT, true>));
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(project_kernel<FT, false>));
    return e;
}

}  // namespace

cudaError_t prepare_project_kernels() {
    cudaError_t e = prepare_typed<uint16_t>();
    if (e == cudaSuccess) e = prepare_typed<float>();
    if (e == cudaSuccess) e = prepare_typed<double>();
    return e;
}

cudaError_t launch_project(const wdd_plan* P, const void* frames, int dtype, int n,
                           const IndexBlock& ids, float* c_out, int32_t* idx_out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > kLaunchFrames) return cudaErrorInvalidValue;
    switch (dtype) {
        case WDD_FRAME_U16:
            return launch_typed(P, static_cast<const uint16_t*>(frames), n, ids, c_out, idx_out, st);
        case WDD_FRAME_F32:
            return launch_typed(P, static_cast<const float*>(frames), n, ids, c_out, idx_out, st);
        case WDD_FRAME_F64:
            return launch_typed(P, static_cast<const double*>(frames), n, ids, c_out, idx_out, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace wdd
