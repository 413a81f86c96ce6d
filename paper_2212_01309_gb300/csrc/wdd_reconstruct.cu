// Snapshot reconstruction (Algorithm 2, after the frame loop; Eq. 3):
//   o_v = sum_k W_v[k] H[v, k]                 (Hadamard product with K_v, summed over every element)
//   O   = conj( IDFT2( o / sqrt(o_0) ) )        (numpy ifft2 normalisation 1/S)
//   phase = atan2(Im O, Re O)
// The deconvolution reads H and W once (HBM bound); the inverse DFT runs
// row-column on the S_y x S_x spectrum with exact integer twiddle indices.

#include <mutex>

#include "wdd_internal.h"

namespace wdd {

namespace {

// One warp per scan frequency.  FP32 with four independent partial sums per lane, added in a
// fixed order (FP64 arithmetic is slow on this part and K <= 4096 terms need no more).
__global__ void deconvolve_kernel(const float2* __restrict__ W, const float2* __restrict__ H,
                                  float2* __restrict__ o, int S, int K) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= S) return;
    const float2* w = W + (size_t)warp * K;
    const float2* h = H + (size_t)warp * K;
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    int k = lane, q = 0;
    for (; k < K; k += 32, q = (q + 1) & 3) {
        const float2 a = __ldg(w + k);
        const float2 b = __ldcg(h + k);
        re[q] = fmaf(a.x, b.x, fmaf(-a.y, b.y, re[q]));
        im[q] = fmaf(a.x, b.y, fmaf(a.y, b.x, im[q]));
    }
    float sr = (re[0] + re[1]) + (re[2] + re[3]);
    float si = (im[0] + im[1]) + (im[2] + im[3]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, off);
        si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    if (lane == 0) o[warp] = make_float2(sr, si);
}

// 1 / sqrt(z) with the principal square root; 1 when z == 0.  The root is formed without
// cancellation: t = sqrt((|z| + |x|) / 2) gives the larger component and y / (2 t) the other,
// so a rounded |z| slightly below |x| cannot produce the square root of a negative number.
__device__ double2 inv_principal_sqrt(float2 zf) {
    double x = zf.x, y = zf.y;
    if (x == 0.0 && y == 0.0) return make_double2(1.0, 0.0);
    double r = hypot(x, y);
    double t = sqrt(0.5 * (r + fabs(x)));
    double sr, si;
    if (x >= 0.0) {
        sr = t;
        si = y / (2.0 * t);
    } else {
        sr = fabs(y) / (2.0 * t);
        si = copysign(t, y);
    }
    double d = sr * sr + si * si;
    return make_double2(sr / d, -si / d);
}

// pass 1: X[vy][x] = sum_vx (o[vy][vx] / sqrt(o_0)) exp(+2 pi i vx x / Sx); one CTA per row
__global__ void idft_rows_kernel(const float2* __restrict__ o, const float2* __restrict__ twx,
                                 float2* __restrict__ X, int Sy, int Sx) {
    extern __shared__ float2 sm2[];
    float2* srow = sm2;        // Sx
    float2* stw = sm2 + Sx;    // Sx
    const int vy = blockIdx.x;
    double2 sc = inv_principal_sqrt(o[0]);
    float scr = (float)sc.x, sci = (float)sc.y;
    for (int t = threadIdx.x; t < Sx; t += blockDim.x) {
        float2 a = o[(size_t)vy * Sx + t];
        srow[t] = make_float2(a.x * scr - a.y * sci, a.x * sci + a.y * scr);
        stw[t] = twx[t];
    }
    __syncthreads();
    for (int x = threadIdx.x; x < Sx; x += blockDim.x) {
        float re = 0.f, im = 0.f;
        int m = 0;
        for (int vx = 0; vx < Sx; ++vx) {
            float2 a = srow[vx], w = stw[m];
            re = fmaf(a.x, w.x, fmaf(-a.y, w.y, re));
            im = fmaf(a.x, w.y, fmaf(a.y, w.x, im));
            m += x;
            if (m >= Sx) m -= Sx;
        }
        X[(size_t)vy * Sx + x] = make_float2(re, im);
    }
}

// pass 2: O[y][x] = conj( sum_vy X[vy][x] exp(+2 pi i vy y / Sy) ) / S; one CTA per column
__global__ void idft_cols_kernel(const float2* __restrict__ X, const float2* __restrict__ twy,
                                 float2* __restrict__ obj, float* __restrict__ phase, int Sy,
                                 int Sx) {
    extern __shared__ float2 sm2[];
    float2* scol = sm2;        // Sy
    float2* stw = sm2 + Sy;    // Sy
    const int x = blockIdx.x;
    for (int t = threadIdx.x; t < Sy; t += blockDim.x) {
        scol[t] = X[(size_t)t * Sx + x];
        stw[t] = twy[t];
    }
    __syncthreads();
    const float inv = 1.0f / (float)((double)Sy * (double)Sx);
    for (int y = threadIdx.x; y < Sy; y += blockDim.x) {
        float re = 0.f, im = 0.f;
        int m = 0;
        for (int vy = 0; vy < Sy; ++vy) {
            float2 a = scol[vy], w = stw[m];
            re = fmaf(a.x, w.x, fmaf(-a.y, w.y, re));
            im = fmaf(a.x, w.y, fmaf(a.y, w.x, im));
            m += y;
            if (m >= Sy) m -= Sy;
        }
        float2 r = make_float2(re * inv, -im * inv);
        obj[(size_t)y * Sx + x] = r;
        if (phase) phase[(size_t)y * Sx + x] = atan2f(r.y, r.x);
    }
}

}  // namespace

cudaError_t launch_deconvolve(const wdd_plan* P, cudaStream_t st) {
    int warps_per_block = kThreads / 32;
    int blocks = (P->S + warps_per_block - 1) / warps_per_block;
    deconvolve_kernel<<<blocks, kThreads, 0, st>>>(P->d_W, P->d_H, P->d_o, P->S, P->K);
    return cudaGetLastError();
}

namespace {

// Twiddles exp(+2 pi i m / n) for both scan axes (the same expression as the plan's tables).
__global__ void idft_tables_kernel(float2* twy, int Sy, float2* twx, int Sx) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < Sy) {
        double s, c;
        sincospi(2.0 * (double)t / (double)Sy, &s, &c);
        twy[t] = make_float2((float)c, (float)s);
    }
    if (t < Sx) {
        double s, c;
        sincospi(2.0 * (double)t / (double)Sx, &s, &c);
        twx[t] = make_float2((float)c, (float)s);
    }
}

// ---- reconstruction without allocation ---------------------------------------------------
// Scratch for wdd_reconstruct_noalloc: spectrum (S), inverse-DFT intermediate (S) and the two
// twiddle tables, in one file-scope device array that every call shares.  Each call writes all
// of the scratch it reads, so nothing needs clearing between calls.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static void* g_noalloc_ptr[kMaxDevices];   // device address of the scratch, per device
static std::mutex g_noalloc_mutex;

}  // namespace

cudaError_t noalloc_scratch(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        // the host-side symbol is only a stand-in: the kernel needs the device address
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = prepare_reconstruct_kernels();
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return cudaSuccess;
}

size_t noalloc_scratch_limit() { return kNoAllocScratchBytes; }

cudaError_t launch_reconstruct_noalloc(void* scratch, const float2* W, const float2* H, int Sy,
                                       int Sx, int K, float2* obj, float* phase, cudaStream_t st) {
    const int S = Sy * Sx;
    float2* o = static_cast<float2*>(scratch);
    float2* X = o + S;
    float2* twy = X + S;
    float2* twx = twy + Sy;
    const int nt = Sy > Sx ? Sy : Sx;
    idft_tables_kernel<<<(nt + kThreads - 1) / kThreads, kThreads, 0, st>>>(twy, Sy, twx, Sx);
    deconvolve_kernel<<<(S + kThreads / 32 - 1) / (kThreads / 32), kThreads, 0, st>>>(W, H, o, S, K);
    idft_rows_kernel<<<Sy, kThreads, 2 * sizeof(float2) * Sx, st>>>(o, twx, X, Sy, Sx);
    idft_cols_kernel<<<Sx, kThreads, 2 * sizeof(float2) * Sy, st>>>(X, twy, obj, phase, Sy, Sx);
    return cudaGetLastError();
}

cudaError_t prepare_reconstruct_kernels() {
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(idft_rows_kernel));
    if (e == cudaSuccess) e = allow_max_dynamic_smem(reinterpret_cast<const void*>(idft_cols_kernel));
    return e;
}

cudaError_t launch_idft_tables(float2* twy, int Sy, float2* twx, int Sx, cudaStream_t st) {
    const int nt = Sy > Sx ? Sy : Sx;
    idft_tables_kernel<<<(nt + kThreads - 1) / kThreads, kThreads, 0, st>>>(twy, Sy, twx, Sx);
    return cudaGetLastError();
}

cudaError_t launch_idft(const float2* o, const float2* twx, const float2* twy, float2* tmp, int Sy,
                        int Sx, float2* obj, float* phase, cudaStream_t st) {
    idft_rows_kernel<<<Sy, kThreads, 2 * sizeof(float2) * Sx, st>>>(o, twx, tmp, Sy, Sx);
    idft_cols_kernel<<<Sx, kThreads, 2 * sizeof(float2) * Sy, st>>>(tmp, twy, obj, phase, Sy, Sx);
    return cudaGetLastError();
}

cudaError_t launch_inverse_dft(const wdd_plan* P, float2* obj, float* phase, cudaStream_t st) {
    idft_rows_kernel<<<P->Sy, kThreads, 2 * sizeof(float2) * P->Sx, st>>>(P->d_o, P->d_twx,
                                                                         P->d_tmp, P->Sy, P->Sx);
    idft_cols_kernel<<<P->Sx, kThreads, 2 * sizeof(float2) * P->Sy, st>>>(P->d_tmp, P->d_twy, obj,
                                                                         phase, P->Sy, P->Sx);
    return cudaGetLastError();
}

}  // namespace wdd
