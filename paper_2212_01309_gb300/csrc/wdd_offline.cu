// Classical (offline) WDD on the GPU: Eq. 2 and Eq. 3 over the whole 4-D dataset.
//
//   G(v, q)  = sum_s exp(-2 pi i q_v . r_s) I_s(q)         forward FFT over both scan axes
//   G'(v, r) = IFFT_q( ifftshift_q G(v, .) )                 inverse FFT over the detector
//   W_O      = G' conj(W_P) / (|W_P|^2 + eps_eff),  W_P = IFFT_q( ifftshift_q Y_v )
//   o_v      = sum_r W_O(v, r)                                (F_r(W_O) at q = 0)
//
// followed by the normalisation by sqrt(o_0) and the conjugated inverse DFT shared with the live
// path.  Every transform is a batch of 1-D transforms staged through shared memory: radix-2
// decimation in time for power-of-two lengths (inputs placed in bit-reversed order as they are
// loaded) and a direct DFT with exact integer twiddle indices for other lengths, in FP32 with
// twiddles built in FP64.  Each pass reads and writes HBM once; the detector pass keeps one scan
// frequency's whole detector plane in shared memory when it fits and multiplies by the Wiener
// kernel on the way out, so G' never reaches HBM.  Larger detectors take a row pass and a column
// pass, the second one fused with the product and a per-block partial sum.
//
// The Wiener kernel conj(W_P) / (|W_P|^2 + eps_eff) is built once per plan: Y_v in FP64 exactly
// as the live plan evaluates it (the analytic probe at the shifted point), the same detector
// transform in FP32, eps_eff = epsilon * max |W_P|^2 (relative, reading R5) and the division.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "wdd_device.cuh"
#include "wdd_internal.h"

struct wdd_offline_plan {
    wdd_params p{};
    int Sy = 0, Sx = 0, S = 0, Ny = 0, Nx = 0, npix = 0;
    double lambda = 0, R = 0, eps_eff = 0;
    int n_active = 0;
    int fused = 0;               // 1: one CTA holds a whole detector plane
    int rb = 0, cp = 0, ncb = 0; // two-pass detector transform: rows per CTA, columns per CTA, blocks
    float2* d_G = nullptr;       // [S][Ny][Nx] scan spectrum (work array)
    float2* d_K = nullptr;       // [S][Ny][Nx] Wiener kernel conj(W_P) / (|W_P|^2 + eps_eff)
    uint8_t* d_mask = nullptr;   // [S]
    double* d_qy = nullptr;      // [Sy] probe shift per frequency row, detector pixels
    double* d_qx = nullptr;      // [Sx]
    float2* d_tw_sy = nullptr;   // [Sy] exp(-2 pi i j / Sy)
    float2* d_tw_sx = nullptr;   // [Sx]
    float2* d_tw_dy = nullptr;   // [Ny] exp(-2 pi i j / Ny) (conjugated for the inverse)
    float2* d_tw_dx = nullptr;   // [Nx]
    float2* d_twy_inv = nullptr; // [Sy] exp(+2 pi i j / Sy) (final inverse DFT)
    float2* d_twx_inv = nullptr; // [Sx]
    float2* d_o = nullptr;       // [S] spectrum o_v
    float2* d_tmp = nullptr;     // [S] inverse-DFT intermediate
    float2* d_part = nullptr;    // [S][ncb] partial sums of the two-pass detector transform
    unsigned* d_max = nullptr;   // [1] max |W_P|^2 (float bits)
    // probe reconstruction (Sect. 10): K built from an object estimate instead of the probe
    int swapped = 0;
    double2* d_Ey = nullptr;     // [Sy][Ny][Sy] scan-y sums at detector row i - cy - qy[vy]
    double2* d_Ey0 = nullptr;    // [Ny][Sy] the same without the shift
    double2* d_Ex = nullptr;     // [Sx][Nx][Sx]
    double2* d_Ex0 = nullptr;    // [Nx][Sx]
    double2* d_T = nullptr;      // [Sx][Sy][Nx] x sums of the object estimate per x shift
    double2* d_T0 = nullptr;     // [Sy][Nx]
    double2* d_Psi0 = nullptr;   // [Ny][Nx] object spectrum at the detector pixels
    float* d_vmax = nullptr;     // [S] max_r |W_O(v, r)|^2
    std::vector<wdd::DevBuf> allocs;
    int64_t device_bytes = 0;
};

namespace wdd {
namespace {

constexpr int kOffThreads = 256;
constexpr int kDetThreads = 512;
constexpr int kScanLineElems = 8192;    // elements staged per scan-axis CTA (64 KB)
constexpr int kFusedPow2Pix = 16384;    // detector planes up to 128 KB take the fused pass
constexpr int kFusedDftPix = 12288;     // two buffers for the direct DFT

wdd_status off_fail(wdd_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

wdd_status off_cuda_fail(cudaError_t e, const char* where) {
    return off_fail(WDD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int log2_exact(int n) {  // log2(n) for powers of two, else -1
    if (n <= 0 || (n & (n - 1))) return -1;
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

__device__ __forceinline__ int brev_bits(int j, int logn) {
    return logn > 0 ? (int)(__brev((unsigned)j) >> (32 - logn)) : 0;
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 as_c(uint16_t v) { return make_float2((float)v, 0.f); }
__device__ __forceinline__ float2 as_c(float v) { return make_float2(v, 0.f); }
__device__ __forceinline__ float2 as_c(double v) { return make_float2((float)v, 0.f); }
__device__ __forceinline__ float2 as_c(float2 v) { return v; }

// In-place radix-2 decimation-in-time transforms of `lines` lines of length 2^logn held in
// shared memory in bit-reversed order: element i of line l at buf[l * ls + i * es].
// tw[j] = exp(-2 pi i j / n) for j < n / 2; INV uses the conjugate (no 1/n factor).
// line_fastest: consecutive threads take consecutive lines (bank-conflict free when es > 1).
template <bool INV>
__device__ void fft_lines_pow2(float2* buf, int logn, int lines, int es, int ls, const float2* tw,
                               bool line_fastest) {
    if (logn <= 0) return;
    const int half = 1 << (logn - 1);
    const int total = lines * half;
    for (int s = 0; s < logn; ++s) {
        const int h = 1 << s;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            int l, t;
            if (line_fastest) {
                l = b % lines;
                t = b / lines;
            } else {
                l = b >> (logn - 1);
                t = b & (half - 1);
            }
            const int k = t & (h - 1);
            const int i0 = ((t >> s) << (s + 1)) + k;
            float2 w = tw[k << (logn - 1 - s)];
            if (INV) w.y = -w.y;
            float2* p0 = buf + (size_t)l * ls + (size_t)i0 * es;
            float2* p1 = p0 + (size_t)h * es;
            const float2 a = *p0;
            const float2 c = cmulf(w, *p1);
            *p0 = make_float2(a.x + c.x, a.y + c.y);
            *p1 = make_float2(a.x - c.x, a.y - c.y);
        }
        __syncthreads();
    }
}

// One output of a direct DFT of length n: sum_m in[m * es] w^(j m), w = exp(-/+ 2 pi i / n),
// with the exact twiddle index (j m) mod n into tw[j] = exp(-2 pi i j / n), j < n.
template <bool INV>
__device__ __forceinline__ float2 dft_point(const float2* in, int es, int n, int j,
                                            const float2* tw) {
    float re = 0.f, im = 0.f;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const float2 a = in[(size_t)i * es];
        float2 w = tw[m];
        if (INV) w.y = -w.y;
        re = fmaf(a.x, w.x, fmaf(-a.y, w.y, re));
        im = fmaf(a.x, w.y, fmaf(a.y, w.x, im));
        m += j;
        if (m >= n) m -= n;
    }
    return make_float2(re, im);
}

// Fixed-order block reductions (valid in thread 0).
__device__ float2 block_sum2(float2 v, float2* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float2 s = make_float2(0.f, 0.f);
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = make_float2(s.x + red[w].x, s.y + red[w].y);
    return s;
}

__device__ float block_max(float v, float* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float m = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    return m;
}

// exp(-2 pi i j / n), j < n, FP64-built.
__global__ void twiddle_kernel(float2* tw, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s, c;
    sincospi(2.0 * (double)j / (double)n, &s, &c);
    tw[j] = make_float2((float)c, (float)-s);
}

// Forward transform along one scan axis for a block of P detector pixels.  Line `o`
// (blockIdx.y) starts at o * outer_stride; element j of the axis sits j * es further; the P
// pixels are contiguous (coalesced).  src may be the frames (first axis) or dst itself.
template <typename T, bool PW2>
__global__ void __launch_bounds__(kOffThreads)
scan_axis_kernel(const T* src, float2* dst, const float2* __restrict__ tw_g, int n, int logn,
                 int P, int npix, int64_t outer_stride, int64_t es) {
    extern __shared__ float2 sm[];
    float2* tw = sm;        // n
    float2* buf = sm + n;   // n * P
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = tw_g[t];
    const int q0 = blockIdx.x * P;
    const int np = min(P, npix - q0);
    const int64_t base = (int64_t)blockIdx.y * outer_stride + q0;
    for (int t = threadIdx.x; t < n * P; t += blockDim.x) {
        const int j = t / P, p = t - (t / P) * P;
        float2 v = make_float2(0.f, 0.f);
        if (p < np) v = as_c(src[base + (int64_t)j * es + p]);
        const int pos = PW2 ? brev_bits(j, logn) : j;
        buf[pos * P + p] = v;
    }
    __syncthreads();
    if (PW2) {
        fft_lines_pow2<false>(buf, logn, P, P, 1, tw, true);
        for (int t = threadIdx.x; t < n * P; t += blockDim.x) {
            const int j = t / P, p = t - (t / P) * P;
            if (p < np) dst[base + (int64_t)j * es + p] = buf[t];
        }
    } else {
        for (int t = threadIdx.x; t < n * P; t += blockDim.x) {
            const int j = t / P, p = t - (t / P) * P;
            if (p < np) dst[base + (int64_t)j * es + p] = dft_point<false>(buf + p, P, n, j, tw);
        }
    }
}

// Whole detector plane of one scan frequency (blockIdx.x) in shared memory: ifftshift on load,
// inverse 2-D transform, then
//   MODE 0: o_v = scale * sum_r G'(r) K(r)   (inactive v: 0)
//   MODE 1: plane = scale * G' written back in place, max |.|^2 folded into *maxbits.
template <int MODE, bool PW2>
__global__ void __launch_bounds__(kDetThreads)
det_fused_kernel(float2* G, const float2* __restrict__ K, const uint8_t* __restrict__ mask,
                 float2* __restrict__ o, unsigned* __restrict__ maxbits,
                 const float2* __restrict__ twy_g, const float2* __restrict__ twx_g, int Ny,
                 int Nx, int logy, int logx, float scale) {
    extern __shared__ float2 sm[];
    __shared__ float2 red2[kDetThreads / 32];
    __shared__ float redf[kDetThreads / 32];
    const int npix = Ny * Nx;
    const int nty = PW2 ? Ny / 2 : Ny, ntx = PW2 ? Nx / 2 : Nx;
    float2* twy = sm;
    float2* twx = twy + nty;
    float2* A = twx + ntx;
    float2* B = A + npix;   // direct-DFT path only
    const int v = blockIdx.x;
    if (MODE == 0 && !mask[v]) {
        if (threadIdx.x == 0) o[v] = make_float2(0.f, 0.f);
        return;
    }
    for (int t = threadIdx.x; t < nty; t += blockDim.x) twy[t] = twy_g[t];
    for (int t = threadIdx.x; t < ntx; t += blockDim.x) twx[t] = twx_g[t];
    float2* g = G + (size_t)v * npix;
    const int hy = Ny / 2, hx = Nx / 2;
    for (int e = threadIdx.x; e < npix; e += blockDim.x) {
        const int qy = e / Nx, qx = e - (e / Nx) * Nx;
        int jy = qy - hy, jx = qx - hx;
        if (jy < 0) jy += Ny;
        if (jx < 0) jx += Nx;
        if (PW2) {
            jy = brev_bits(jy, logy);
            jx = brev_bits(jx, logx);
        }
        A[jy * Nx + jx] = g[e];
    }
    __syncthreads();
    float2 acc = make_float2(0.f, 0.f);
    float mx = 0.f;
    const float2* kv = K + (size_t)v * npix;
    if (PW2) {
        fft_lines_pow2<true>(A, logx, Ny, 1, Nx, twx, false);   // rows
        fft_lines_pow2<true>(A, logy, Nx, Nx, 1, twy, true);    // columns
        for (int e = threadIdx.x; e < npix; e += blockDim.x) {
            const float2 val = A[e];
            if (MODE == 0) {
                const float2 k = kv[e];
                acc.x = fmaf(val.x, k.x, fmaf(-val.y, k.y, acc.x));
                acc.y = fmaf(val.x, k.y, fmaf(val.y, k.x, acc.y));
            } else {
                const float2 w = make_float2(val.x * scale, val.y * scale);
                g[e] = w;
                mx = fmaxf(mx, w.x * w.x + w.y * w.y);
            }
        }
    } else {
        for (int e = threadIdx.x; e < npix; e += blockDim.x) {
            const int jy = e / Nx, rx = e - (e / Nx) * Nx;
            B[e] = dft_point<true>(A + (size_t)jy * Nx, 1, Nx, rx, twx);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < npix; e += blockDim.x) {
            const int ry = e / Nx, rx = e - (e / Nx) * Nx;
            const float2 val = dft_point<true>(B + rx, Nx, Ny, ry, twy);
            if (MODE == 0) {
                const float2 k = kv[e];
                acc.x = fmaf(val.x, k.x, fmaf(-val.y, k.y, acc.x));
                acc.y = fmaf(val.x, k.y, fmaf(val.y, k.x, acc.y));
            } else {
                const float2 w = make_float2(val.x * scale, val.y * scale);
                g[e] = w;
                mx = fmaxf(mx, w.x * w.x + w.y * w.y);
            }
        }
    }
    if (MODE == 0) {
        const float2 s = block_sum2(acc, red2);
        if (threadIdx.x == 0) o[v] = make_float2(s.x * scale, s.y * scale);
    } else {
        const float m = block_max(mx, redf);
        if (threadIdx.x == 0) atomicMax(maxbits, __float_as_uint(m));
    }
}

// Two-pass detector transform, pass 1: ifftshift along x and the inverse transform of RB rows
// (blockIdx.y) of one scan frequency (blockIdx.x), in place.  The y shift waits for pass 2.
template <bool PW2>
__global__ void __launch_bounds__(kOffThreads)
det_rows_kernel(float2* G, const float2* __restrict__ twx_g, int Ny, int Nx, int logx, int RB) {
    extern __shared__ float2 sm[];
    const int ntx = PW2 ? Nx / 2 : Nx;
    float2* twx = sm;
    float2* buf = sm + ntx;
    for (int t = threadIdx.x; t < ntx; t += blockDim.x) twx[t] = twx_g[t];
    const int y0 = blockIdx.y * RB;
    const int nr = min(RB, Ny - y0);
    float2* g = G + (size_t)blockIdx.x * Ny * Nx + (size_t)y0 * Nx;
    const int hx = Nx / 2;
    for (int t = threadIdx.x; t < nr * Nx; t += blockDim.x) {
        const int r = t / Nx, qx = t - (t / Nx) * Nx;
        int jx = qx - hx;
        if (jx < 0) jx += Nx;
        if (PW2) jx = brev_bits(jx, logx);
        buf[r * Nx + jx] = g[t];
    }
    __syncthreads();
    if (PW2) {
        fft_lines_pow2<true>(buf, logx, nr, 1, Nx, twx, false);
        for (int t = threadIdx.x; t < nr * Nx; t += blockDim.x) g[t] = buf[t];
    } else {
        for (int t = threadIdx.x; t < nr * Nx; t += blockDim.x) {
            const int r = t / Nx, rx = t - (t / Nx) * Nx;
            g[t] = dft_point<true>(buf + (size_t)r * Nx, 1, Nx, rx, twx);
        }
    }
}

// Pass 2: ifftshift along y and the inverse transform of P columns (blockIdx.y) of one scan
// frequency (blockIdx.x); MODE 0 multiplies by K and writes the block's partial sum
// part[v][blockIdx.y] (inactive v: 0), MODE 1 writes scale * G' back and folds max |.|^2.
template <int MODE, bool PW2>
__global__ void __launch_bounds__(kOffThreads)
det_cols_kernel(float2* G, const float2* __restrict__ K, const uint8_t* __restrict__ mask,
                float2* __restrict__ part, unsigned* __restrict__ maxbits,
                const float2* __restrict__ twy_g, int Ny, int Nx, int logy, int P, float scale) {
    extern __shared__ float2 sm[];
    __shared__ float2 red2[kOffThreads / 32];
    __shared__ float redf[kOffThreads / 32];
    const int v = blockIdx.x;
    const int ncb = gridDim.y;
    if (MODE == 0 && !mask[v]) {
        if (threadIdx.x == 0) part[(size_t)v * ncb + blockIdx.y] = make_float2(0.f, 0.f);
        return;
    }
    const int nty = PW2 ? Ny / 2 : Ny;
    float2* twy = sm;
    float2* buf = sm + nty;
    for (int t = threadIdx.x; t < nty; t += blockDim.x) twy[t] = twy_g[t];
    const int c0 = blockIdx.y * P;
    const int np = min(P, Nx - c0);
    const size_t npix = (size_t)Ny * Nx;
    float2* g = G + (size_t)v * npix;
    const int hy = Ny / 2;
    for (int t = threadIdx.x; t < Ny * P; t += blockDim.x) {
        const int i = t / P, p = t - (t / P) * P;
        int jy = i - hy;
        if (jy < 0) jy += Ny;
        if (PW2) jy = brev_bits(jy, logy);
        buf[jy * P + p] = p < np ? g[(size_t)i * Nx + c0 + p] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (PW2) fft_lines_pow2<true>(buf, logy, P, P, 1, twy, true);
    float2 acc = make_float2(0.f, 0.f);
    float mx = 0.f;
    const float2* kv = K + (size_t)v * npix;
    for (int t = threadIdx.x; t < Ny * P; t += blockDim.x) {
        const int ry = t / P, p = t - (t / P) * P;
        if (p >= np) continue;
        const float2 val = PW2 ? buf[t] : dft_point<true>(buf + p, P, Ny, ry, twy);
        const size_t e = (size_t)ry * Nx + c0 + p;
        if (MODE == 0) {
            const float2 k = kv[e];
            acc.x = fmaf(val.x, k.x, fmaf(-val.y, k.y, acc.x));
            acc.y = fmaf(val.x, k.y, fmaf(val.y, k.x, acc.y));
        } else {
            const float2 w = make_float2(val.x * scale, val.y * scale);
            g[e] = w;
            mx = fmaxf(mx, w.x * w.x + w.y * w.y);
        }
    }
    if (MODE == 0) {
        const float2 s = block_sum2(acc, red2);
        if (threadIdx.x == 0) part[(size_t)v * ncb + blockIdx.y] = s;
    } else {
        const float m = block_max(mx, redf);
        if (threadIdx.x == 0) atomicMax(maxbits, __float_as_uint(m));
    }
}

// o_v = scale * sum_b part[v][b] in block order (inactive v: 0).
__global__ void det_reduce_kernel(const float2* __restrict__ part, const uint8_t* __restrict__ mask,
                                  float2* __restrict__ o, int S, int ncb, float scale) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= S) return;
    float2 s = make_float2(0.f, 0.f);
    if (mask[v])
        for (int b = 0; b < ncb; ++b) {
            const float2 a = part[(size_t)v * ncb + b];
            s.x += a.x;
            s.y += a.y;
        }
    o[v] = make_float2(s.x * scale, s.y * scale);
}

// Y_v(q) = p(q) conj p(q + q_v) on the detector grid (Algorithm 1, Eq. 2), q_v the scan-axis
// shift turned by the scan rotation (rc, rs), evaluated in FP64 as the live plan does, stored
// as complex64 [S][Ny][Nx].
__global__ void probe_autocorr_kernel(float2* __restrict__ Y, const double* __restrict__ qy,
                                      const double* __restrict__ qx, int Sx, int Ny, int Nx,
                                      double cy, double cx, double R2, double coef, double rc,
                                      double rs, int64_t total) {
    const int64_t npix = (int64_t)Ny * Nx;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(t / npix);
        const int e = (int)(t - (int64_t)v * npix);
        const int i = e / Nx, j = e - (e / Nx) * Nx;
        const double sa = qy[v / Sx], sb = qx[v % Sx];
        const double shy = __dsub_rn(__dmul_rn(rc, sa), __dmul_rn(rs, sb));
        const double shx = __dadd_rn(__dmul_rn(rs, sa), __dmul_rn(rc, sb));
        const double ky = (double)i - cy, kx = (double)j - cx;
        const double k2 = __dadd_rn(__dmul_rn(ky, ky), __dmul_rn(kx, kx));
        const double2 a = probe_at(k2, R2, coef);
        float2 y = make_float2(0.f, 0.f);
        if (a.x != 0.0 || a.y != 0.0) {
            const double ky2 = __dadd_rn(ky, shy), kx2 = __dadd_rn(kx, shx);
            const double k2s = __dadd_rn(__dmul_rn(ky2, ky2), __dmul_rn(kx2, kx2));
            const double2 b = probe_at(k2s, R2, coef);
            y = make_float2((float)(a.x * b.x + a.y * b.y), (float)(a.y * b.x - a.x * b.y));
        }
        Y[t] = y;
    }
}

// K = conj(W_P) / (|W_P|^2 + eps) in place; inactive frequencies get 0.
__global__ void wiener_kernel(float2* __restrict__ K, const uint8_t* __restrict__ mask,
                              int64_t npix, int64_t total, float eps) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(t / npix);
        const float2 w = K[t];
        if (!mask[v]) {
            K[t] = make_float2(0.f, 0.f);
            continue;
        }
        const float d = w.x * w.x + w.y * w.y + eps;
        K[t] = make_float2(w.x / d, -w.y / d);
    }
}

// ---- probe reconstruction (Sect. 10): the deconvolution with the roles swapped.  The Wiener
// kernel is built from Omega_v(q) = Psi(q) conj Psi(q - q_v), Psi the spectrum of an object
// estimate given on the scan grid, evaluated at detector-pixel frequencies as the trigonometric
// sum over the scan positions.  Without a scan rotation that sum separates into one sum per
// scan axis, which is what the tables below hold.  The sums run in FP64: away from its peaks
// Psi is a small result of S unit-size terms, and FP32 sums left 1e-3 errors in the probe of a
// weak phase object where FP64 sums leave 2e-7; Omega is rounded to FP32 once, for the
// detector transform.

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // c + a b
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// E[(v * n + i) * ns + s] = exp(-2 pi i frac(((i - c - q[v]) * dks) * s)) for v < nv, i < n,
// s < ns: one axis of the trigonometric sum at detector-pixel frequency i - c - q[v] (q == NULL:
// no shift, nv = 1).  dks = dk * scan step; the phase is reduced to one turn.
__global__ void axis_dtft_table_kernel(double2* __restrict__ E, const double* __restrict__ q,
                                       int nv, int n, int ns, double c, double dks) {
    const int64_t total = (int64_t)nv * n * ns;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(t % ns);
        const int64_t r = t / ns;
        const int i = (int)(r % n);
        const int v = (int)(r / n);
        const double k = (double)i - c - (q ? q[v] : 0.0);
        const double ph = (k * dks) * (double)s;
        const double f = ph - floor(ph);
        double sn, cs;
        sincospi(-2.0 * f, &sn, &cs);
        E[t] = make_double2(cs, sn);
    }
}

// T[(u * Sy + sy) * Nx + j] = sum_sx O[sy][sx] Ex[(u * Nx + j) * Sx + sx] for u < nu: the sums of
// the object estimate along scan x at every x shift u and detector column j.
__global__ void obj_xsum_kernel(const float2* __restrict__ O, const double2* __restrict__ Ex,
                                double2* __restrict__ T, int nu, int Sy, int Sx, int Nx) {
    const int64_t total = (int64_t)nu * Sy * Nx;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % Nx);
        const int64_t r = t / Nx;
        const int sy = (int)(r % Sy);
        const int u = (int)(r / Sy);
        const float2* o = O + (size_t)sy * Sx;
        const double2* e = Ex + ((size_t)u * Nx + j) * Sx;
        double2 acc = make_double2(0.0, 0.0);
        for (int sx = 0; sx < Sx; ++sx) {
            const float2 ov = o[sx];
            acc = cfma(make_double2(ov.x, ov.y), e[sx], acc);
        }
        T[t] = acc;
    }
}

// Psi0[i][j] = sum_sy Ey0[i][sy] T0[sy][j]: the object spectrum at detector pixel (i, j).
__global__ void psi0_kernel(const double2* __restrict__ Ey0, const double2* __restrict__ T0,
                            double2* __restrict__ Psi0, int Sy, int Ny, int Nx) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Ny * Nx) return;
    const int i = t / Nx, j = t - (t / Nx) * Nx;
    double2 a = make_double2(0.0, 0.0);
    for (int sy = 0; sy < Sy; ++sy) a = cfma(Ey0[(size_t)i * Sy + sy], T0[(size_t)sy * Nx + j], a);
    Psi0[t] = a;
}

// K[v][i][j] = Psi0[i][j] conj Psi_v(i, j), Psi_v(i, j) = sum_sy Ey[vy][i][sy] T[vx][sy][j]: the
// object spectrum at the detector pixel moved by -q_v; rounded to complex64.
__global__ void omega_kernel(float2* __restrict__ K, const double2* __restrict__ Ey,
                             const double2* __restrict__ T, const double2* __restrict__ Psi0,
                             int Sy, int Sx, int Ny, int Nx, int64_t total) {
    const int64_t npix = (int64_t)Ny * Nx;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(t / npix);
        const int e = (int)(t - (int64_t)v * npix);
        const int i = e / Nx, j = e - (e / Nx) * Nx;
        const int vy = v / Sx, vx = v - (v / Sx) * Sx;
        const double2* ey = Ey + ((size_t)vy * Ny + i) * Sy;
        const double2* tv = T + (size_t)vx * Sy * Nx + j;
        double2 b = make_double2(0.0, 0.0);
        for (int sy = 0; sy < Sy; ++sy) b = cfma(ey[sy], tv[(size_t)sy * Nx], b);
        const double2 a = Psi0[e];
        K[t] = make_float2((float)(a.x * b.x + a.y * b.y), (float)(a.y * b.x - a.x * b.y));
    }
}

// vmax[v] = max over plane v of |K|^2; one CTA per scan frequency.
__global__ void __launch_bounds__(kOffThreads)
plane_max_kernel(const float2* __restrict__ K, float* __restrict__ vmax, int npix) {
    __shared__ float redf[kOffThreads / 32];
    const float2* k = K + (size_t)blockIdx.x * npix;
    float m = 0.f;
    for (int e = threadIdx.x; e < npix; e += blockDim.x) {
        const float2 w = k[e];
        m = fmaxf(m, w.x * w.x + w.y * w.y);
    }
    m = block_max(m, redf);
    if (threadIdx.x == 0) vmax[blockIdx.x] = m;
}

// K = conj(W_O) / (|W_O|^2 + eps_v) in place, eps_v = eps * vmax[v] (relative, per frequency) or
// eps (absolute); inactive frequencies and planes that are zero everywhere get 0.
__global__ void wiener_pf_kernel(float2* __restrict__ K, const uint8_t* __restrict__ mask,
                                 const float* __restrict__ vmax, int64_t npix, int64_t total,
                                 float eps, int absolute) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(t / npix);
        const float2 w = K[t];
        if (!mask[v]) {
            K[t] = make_float2(0.f, 0.f);
            continue;
        }
        const float ev = absolute ? eps : eps * vmax[v];
        const float d = w.x * w.x + w.y * w.y + ev;
        K[t] = d > 0.f ? make_float2(w.x / d, -w.y / d) : make_float2(0.f, 0.f);
    }
}

// dst[y][x] = src[-y][-x] (indices mod Sy, Sx), with its phase: the probe IFFT2(conj(p / sqrt(p_0)))
// from the conjugated inverse DFT conj(IFFT2(p / sqrt(p_0))) that the object path computes.
__global__ void negate_index_kernel(const float2* __restrict__ src, float2* __restrict__ dst,
                                    float* __restrict__ phase, int Sy, int Sx) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Sy * Sx) return;
    const int y = t / Sx, x = t - (t / Sx) * Sx;
    const int sy = y ? Sy - y : 0, sx = x ? Sx - x : 0;
    const float2 val = src[(size_t)sy * Sx + sx];
    dst[t] = val;
    if (phase) phase[t] = atan2f(val.y, val.x);
}

// ---- four-step transforms: a 1-D transform of n = N1 N2 points as N2 register DFTs of N1
// points, a twiddle w_n^(j2 k1), and N1 register DFTs of N2 points, with one shared-memory round
// trip in between (X[k1 + N1 k2] = sum_j2 w_N2^(j2 k2) w_n^(j2 k1) sum_j1 w_N1^(j1 k1) x[j1 N2 + j2]).

// In-register DFT of M = 2^m points, natural order in and out (radix-2 decimation in time after a
// compile-time bit reversal); w_M^t = tw[t * tws] from the table tw[j] = exp(-2 pi i j / n),
// tws = n / M; INV conjugates the twiddles.
template <int M, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&x)[M], const float2* tw, int tws) {
#pragma unroll
    for (int i = 0; i < M; ++i) {
        int r = 0;
#pragma unroll
        for (int b = 1, t = i; b < M; b <<= 1, t >>= 1) r = (r << 1) | (t & 1);
        if (r > i) {
            const float2 t = x[i];
            x[i] = x[r];
            x[r] = t;
        }
    }
#pragma unroll
    for (int h = 1; h < M; h <<= 1) {
#pragma unroll
        for (int k = 0; k < h; ++k) {
            float2 w = tw[k * (M / (2 * h)) * tws];
            if (INV) w.y = -w.y;
#pragma unroll
            for (int i0 = k; i0 < M; i0 += 2 * h) {
                const float2 a = x[i0];
                const float2 c = k == 0 ? x[i0 + h] : cmulf(w, x[i0 + h]);
                x[i0] = make_float2(a.x + c.x, a.y + c.y);
                x[i0 + h] = make_float2(a.x - c.x, a.y - c.y);
            }
        }
    }
}

// Forward transform of n = N1 N2 points along one scan axis for a block of P pixels (same
// addressing as scan_axis_kernel).  Step 1 reads its N1 points straight from global memory.
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(kOffThreads)
scan_axis4_kernel(const T* src, float2* dst, const float2* __restrict__ tw_g, int P, int npix,
                  int64_t outer_stride, int64_t es) {
    constexpr int n = N1 * N2;
    extern __shared__ float2 sm[];
    float2* tw = sm;        // n
    float2* buf = sm + n;   // [k1][j2][P]
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = tw_g[t];
    __syncthreads();
    const int q0 = blockIdx.x * P;
    const int np = min(P, npix - q0);
    const int64_t base = (int64_t)blockIdx.y * outer_stride + q0;
    for (int task = threadIdx.x; task < N2 * P; task += blockDim.x) {
        const int j2 = task / P, p = task - (task / P) * P;
        float2 x[N1];
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1)
            x[j1] = p < np ? as_c(src[base + (int64_t)(j1 * N2 + j2) * es + p])
                           : make_float2(0.f, 0.f);
        dft_reg<N1, false>(x, tw, N2);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            const float2 y = (k1 == 0 || j2 == 0) ? x[k1] : cmulf(x[k1], tw[j2 * k1]);
            buf[(k1 * N2 + j2) * P + p] = y;
        }
    }
    __syncthreads();
    for (int task = threadIdx.x; task < N1 * P; task += blockDim.x) {
        const int k1 = task / P, p = task - (task / P) * P;
        float2 y[N2];
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) y[j2] = buf[(k1 * N2 + j2) * P + p];
        dft_reg<N2, false>(y, tw, N1);
        if (p < np) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) dst[base + (int64_t)(k1 + N1 * k2) * es + p] = y[k2];
        }
    }
}

// Square detector planes of N = N1 N2 pixels (one scan frequency per CTA), four-step: columns
// first, straight from global memory with the ifftshift of both axes folded into the loads, then
// rows, every step in place in a padded plane (row stride N + N/16 + 1, a pad every 16 entries:
// conflict-free for the access orders below).  After the column steps, plane row q holds output
// row ry = q / N2 + N1 (q % N2); the row steps produce output column rx = k1 + N1 k2 directly,
// so the Wiener kernel is read in order.  MODE as in det_fused_kernel.
template <int MODE, int N1, int N2>
__global__ void __launch_bounds__(kDetThreads)
det_fused4_kernel(float2* G, const float2* __restrict__ K, const uint8_t* __restrict__ mask,
                  float2* __restrict__ o, unsigned* __restrict__ maxbits,
                  const float2* __restrict__ tw_g, float scale) {
    constexpr int N = N1 * N2;
    constexpr int RS = N + N / 16 + 1;
    extern __shared__ float2 sm[];
    __shared__ float2 red2[kDetThreads / 32];
    __shared__ float redf[kDetThreads / 32];
    float2* tw = sm;        // N
    float2* A = sm + N;     // N * RS
    const int v = blockIdx.x;
    if (MODE == 0 && !mask[v]) {
        if (threadIdx.x == 0) o[v] = make_float2(0.f, 0.f);
        return;
    }
    for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = tw_g[t];
    __syncthreads();
    float2* g = G + (size_t)v * N * N;
    auto pos = [](int row, int e) { return row * RS + e + (e >> 4); };
    constexpr int H = N / 2;
    // columns, step 1: shifted row j = j1 N2 + j2 is stored row (j + N/2) mod N
    for (int task = threadIdx.x; task < N * N2; task += blockDim.x) {
        const int c = task % N, j2 = task / N;
        const int col = (c + H) & (N - 1);
        float2 x[N1];
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) x[j1] = g[(size_t)(((j1 * N2 + j2) + H) & (N - 1)) * N + col];
        dft_reg<N1, true>(x, tw, N2);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            float2 w = tw[j2 * k1];
            w.y = -w.y;
            A[pos(k1 * N2 + j2, c)] = (k1 == 0 || j2 == 0) ? x[k1] : cmulf(x[k1], w);
        }
    }
    __syncthreads();
    // columns, step 2 (in place: reads and writes plane rows k1 N2 + 0 .. N2 - 1)
    for (int task = threadIdx.x; task < N * N1; task += blockDim.x) {
        const int c = task % N, k1 = task / N;
        float2 y[N2];
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) y[j2] = A[pos(k1 * N2 + j2, c)];
        dft_reg<N2, true>(y, tw, N1);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) A[pos(k1 * N2 + k2, c)] = y[k2];
    }
    __syncthreads();
    // rows, step 1 (in place: entries j1 N2 + j2 of plane row q)
    for (int task = threadIdx.x; task < N * N2; task += blockDim.x) {
        const int q = task % N, j2 = task / N;
        float2 x[N1];
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) x[j1] = A[pos(q, j1 * N2 + j2)];
        dft_reg<N1, true>(x, tw, N2);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            float2 w = tw[j2 * k1];
            w.y = -w.y;
            A[pos(q, k1 * N2 + j2)] = (k1 == 0 || j2 == 0) ? x[k1] : cmulf(x[k1], w);
        }
    }
    __syncthreads();
    // rows, step 2, consumed directly
    float2 acc = make_float2(0.f, 0.f);
    float mx = 0.f;
    const float2* kv = K + (size_t)v * N * N;
    for (int task = threadIdx.x; task < N * N1; task += blockDim.x) {
        const int k1 = task % N1, q = task / N1;
        float2 y[N2];
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) y[j2] = A[pos(q, k1 * N2 + j2)];
        dft_reg<N2, true>(y, tw, N1);
        const int ry = q / N2 + N1 * (q % N2);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const size_t e = (size_t)ry * N + k1 + N1 * k2;
            const float2 val = y[k2];
            if (MODE == 0) {
                const float2 k = kv[e];
                acc.x = fmaf(val.x, k.x, fmaf(-val.y, k.y, acc.x));
                acc.y = fmaf(val.x, k.y, fmaf(val.y, k.x, acc.y));
            } else {
                const float2 w = make_float2(val.x * scale, val.y * scale);
                g[e] = w;
                mx = fmaxf(mx, w.x * w.x + w.y * w.y);
            }
        }
    }
    if (MODE == 0) {
        const float2 s = block_sum2(acc, red2);
        if (threadIdx.x == 0) o[v] = make_float2(s.x * scale, s.y * scale);
    } else {
        const float m = block_max(mx, redf);
        if (threadIdx.x == 0) atomicMax(maxbits, __float_as_uint(m));
    }
}

// Two-pass detector transform for planes too large for one CTA, four-step version (power-of-
// two sides of 256 .. 1024).  Pass 1: the ifftshift along x and the inverse transform of RB rows
// of one scan frequency, in place; shared rows padded as in det_fused4_kernel.
template <int N1, int N2>
__global__ void __launch_bounds__(kOffThreads)
det_rows4_kernel(float2* G, const float2* __restrict__ tw_g, int Ny, int RB) {
    constexpr int N = N1 * N2;   // Nx
    constexpr int RS = N + N / 16 + 1;
    extern __shared__ float2 sm[];
    float2* tw = sm;        // N
    float2* A = sm + N;     // RB * RS
    for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = tw_g[t];
    __syncthreads();
    const int y0 = blockIdx.y * RB;
    const int nr = min(RB, Ny - y0);
    float2* g = G + (size_t)blockIdx.x * Ny * N + (size_t)y0 * N;
    auto pos = [](int r, int e) { return r * RS + e + (e >> 4); };
    constexpr int H = N / 2;
    for (int task = threadIdx.x; task < nr * N2; task += blockDim.x) {
        const int j2 = task % N2, r = task / N2;
        float2 x[N1];
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) x[j1] = g[(size_t)r * N + (((j1 * N2 + j2) + H) & (N - 1))];
        dft_reg<N1, true>(x, tw, N2);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            float2 w = tw[j2 * k1];
            w.y = -w.y;
            A[pos(r, k1 * N2 + j2)] = (k1 == 0 || j2 == 0) ? x[k1] : cmulf(x[k1], w);
        }
    }
    __syncthreads();
    for (int task = threadIdx.x; task < nr * N1; task += blockDim.x) {
        const int k1 = task % N1, r = task / N1;
        float2 y[N2];
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) y[j2] = A[pos(r, k1 * N2 + j2)];
        dft_reg<N2, true>(y, tw, N1);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) g[(size_t)r * N + k1 + N1 * k2] = y[k2];
    }
}

// Pass 2: the ifftshift along y and the inverse transform of P columns of one scan frequency;
// MODE 0 multiplies by K and writes the block's partial sum part[v][blockIdx.y] (inactive v:
// 0), MODE 1 writes scale * G' back and folds max |.|^2 (as det_cols_kernel).
template <int MODE, int N1, int N2>
__global__ void __launch_bounds__(kOffThreads)
det_cols4_kernel(float2* G, const float2* __restrict__ K, const uint8_t* __restrict__ mask,
                 float2* __restrict__ part, unsigned* __restrict__ maxbits,
                 const float2* __restrict__ tw_g, int Nx, int P, float scale) {
    constexpr int N = N1 * N2;   // Ny
    extern __shared__ float2 sm[];
    __shared__ float2 red2[kOffThreads / 32];
    __shared__ float redf[kOffThreads / 32];
    const int v = blockIdx.x;
    const int ncb = gridDim.y;
    if (MODE == 0 && !mask[v]) {
        if (threadIdx.x == 0) part[(size_t)v * ncb + blockIdx.y] = make_float2(0.f, 0.f);
        return;
    }
    float2* tw = sm;        // N
    float2* buf = sm + N;   // [k1][j2][P]
    for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = tw_g[t];
    __syncthreads();
    const int c0 = blockIdx.y * P;
    const int np = min(P, Nx - c0);
    const size_t npix = (size_t)N * Nx;
    float2* g = G + (size_t)v * npix;
    constexpr int H = N / 2;
    for (int task = threadIdx.x; task < N2 * P; task += blockDim.x) {
        const int j2 = task / P, p = task - (task / P) * P;
        float2 x[N1];
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1)
            x[j1] = p < np ? g[(size_t)(((j1 * N2 + j2) + H) & (N - 1)) * Nx + c0 + p]
                           : make_float2(0.f, 0.f);
        dft_reg<N1, true>(x, tw, N2);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            float2 w = tw[j2 * k1];
            w.y = -w.y;
            buf[(k1 * N2 + j2) * P + p] = (k1 == 0 || j2 == 0) ? x[k1] : cmulf(x[k1], w);
        }
    }
    __syncthreads();
    float2 acc = make_float2(0.f, 0.f);
    float mx = 0.f;
    const float2* kv = K + (size_t)v * npix;
    for (int task = threadIdx.x; task < N1 * P; task += blockDim.x) {
        const int k1 = task / P, p = task - (task / P) * P;
        float2 y[N2];
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) y[j2] = buf[(k1 * N2 + j2) * P + p];
        dft_reg<N2, true>(y, tw, N1);
        if (p >= np) continue;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const size_t e = (size_t)(k1 + N1 * k2) * Nx + c0 + p;
            const float2 val = y[k2];
            if (MODE == 0) {
                const float2 k = kv[e];
                acc.x = fmaf(val.x, k.x, fmaf(-val.y, k.y, acc.x));
                acc.y = fmaf(val.x, k.y, fmaf(val.y, k.x, acc.y));
            } else {
                const float2 w = make_float2(val.x * scale, val.y * scale);
                g[e] = w;
                mx = fmaxf(mx, w.x * w.x + w.y * w.y);
            }
        }
    }
    if (MODE == 0) {
        const float2 sres = block_sum2(acc, red2);
        if (threadIdx.x == 0) part[(size_t)v * ncb + blockIdx.y] = sres;
    } else {
        const float m = block_max(mx, redf);
        if (threadIdx.x == 0) atomicMax(maxbits, __float_as_uint(m));
    }
}

// ---- host side ---------------------------------------------------------------------------

int scan_pixels_per_cta(int n) {
    int P = 64;
    while (P > 4 && n * P > kScanLineElems) P >>= 1;
    return P;
}

size_t scan_smem(int n) { return sizeof(float2) * ((size_t)n + (size_t)n * scan_pixels_per_cta(n)); }

bool fused_fits(int Ny, int Nx) {
    const int npix = Ny * Nx;
    if (log2_exact(Ny) >= 0 && log2_exact(Nx) >= 0) return npix <= kFusedPow2Pix;
    return npix <= kFusedDftPix;
}

size_t fused_smem(int Ny, int Nx) {
    const bool pw2 = log2_exact(Ny) >= 0 && log2_exact(Nx) >= 0;
    const size_t npix = (size_t)Ny * Nx;
    return sizeof(float2) * ((pw2 ? Ny / 2 + Nx / 2 : Ny + Nx) + (pw2 ? npix : 2 * npix));
}

// Rows per CTA / columns per CTA of the two-pass detector transform (64 KB of staging).
int rows_per_cta(int Nx) { return std::max(1, kScanLineElems / Nx); }
int cols_per_cta(int Ny) {
    int P = 64;
    while (P > 1 && Ny * P > kScanLineElems) P >>= 1;
    return P;
}

// Sizes with a four-step transform: n = N1 N2 with register DFTs of at most 32 points.
#define WDD_FOUR_STEP_SIZES(X) X(32, 8, 4) X(64, 8, 8) X(128, 16, 8) X(256, 16, 16) \
    X(512, 32, 16) X(1024, 32, 32)
#define WDD_DET4_SIZES(X) X(32, 8, 4) X(64, 8, 8) X(128, 16, 8)
#define WDD_DET2P4_SIZES(X) X(256, 16, 16) X(512, 32, 16) X(1024, 32, 32)

bool four_step_len(int n) {
#define WDD_FS_CASE(nn, a, b) if (n == nn) return true;
    WDD_FOUR_STEP_SIZES(WDD_FS_CASE)
#undef WDD_FS_CASE
    return false;
}
bool det4_square(int Ny, int Nx) { return Ny == Nx && (Nx == 32 || Nx == 64 || Nx == 128); }
bool det2p4_len(int n) { return n == 256 || n == 512 || n == 1024; }
int scan4_pixels_per_cta(int n) { return std::min(64, std::max(8, kScanLineElems / n)); }
size_t scan4_smem(int n) {
    return sizeof(float2) * ((size_t)n + (size_t)n * scan4_pixels_per_cta(n));
}
size_t det4_smem(int N) { return sizeof(float2) * ((size_t)N + (size_t)N * (N + N / 16 + 1)); }

template <typename F>
cudaError_t for_each_offline_kernel(F f) {
    cudaError_t e = cudaSuccess;
#define WDD_OFF_K(k) \
    if (e == cudaSuccess) e = f(reinterpret_cast<const void*>(k))
#define WDD_OFF_K4(nn, a, b)                                   \
    WDD_OFF_K((scan_axis4_kernel<uint16_t, a, b>));            \
    WDD_OFF_K((scan_axis4_kernel<float, a, b>));               \
    WDD_OFF_K((scan_axis4_kernel<double, a, b>));              \
    WDD_OFF_K((scan_axis4_kernel<float2, a, b>));
    WDD_FOUR_STEP_SIZES(WDD_OFF_K4)
#undef WDD_OFF_K4
#define WDD_OFF_D4(nn, a, b)                                   \
    WDD_OFF_K((det_fused4_kernel<0, a, b>));                   \
    WDD_OFF_K((det_fused4_kernel<1, a, b>));
    WDD_DET4_SIZES(WDD_OFF_D4)
#undef WDD_OFF_D4
#define WDD_OFF_2P4(nn, a, b)                                  \
    WDD_OFF_K((det_rows4_kernel<a, b>));                       \
    WDD_OFF_K((det_cols4_kernel<0, a, b>));                    \
    WDD_OFF_K((det_cols4_kernel<1, a, b>));
    WDD_DET2P4_SIZES(WDD_OFF_2P4)
#undef WDD_OFF_2P4
    WDD_OFF_K((scan_axis_kernel<uint16_t, true>));
    WDD_OFF_K((scan_axis_kernel<uint16_t, false>));
    WDD_OFF_K((scan_axis_kernel<float, true>));
    WDD_OFF_K((scan_axis_kernel<float, false>));
    WDD_OFF_K((scan_axis_kernel<double, true>));
    WDD_OFF_K((scan_axis_kernel<double, false>));
    WDD_OFF_K((scan_axis_kernel<float2, true>));
    WDD_OFF_K((scan_axis_kernel<float2, false>));
    WDD_OFF_K((det_fused_kernel<0, true>));
    WDD_OFF_K((det_fused_kernel<0, false>));
    WDD_OFF_K((det_fused_kernel<1, true>));
    WDD_OFF_K((det_fused_kernel<1, false>));
    WDD_OFF_K((det_rows_kernel<true>));
    WDD_OFF_K((det_rows_kernel<false>));
    WDD_OFF_K((det_cols_kernel<0, true>));
    WDD_OFF_K((det_cols_kernel<0, false>));
    WDD_OFF_K((det_cols_kernel<1, true>));
    WDD_OFF_K((det_cols_kernel<1, false>));
#undef WDD_OFF_K
    return e;
}

cudaError_t prepare_offline_kernels() {
    static cudaError_t status = for_each_offline_kernel(
        [](const void* k) { return allow_max_dynamic_smem(k); });
    return status;
}

// Forward transform along one scan axis: `outer` lines of n elements spaced es apart.
template <typename T>
cudaError_t launch_scan_axis(const T* src, float2* dst, const float2* tw, int n, int npix,
                             int outer, int64_t outer_stride, int64_t es, cudaStream_t st) {
    if (four_step_len(n)) {
        const int P = scan4_pixels_per_cta(n);
        dim3 grid((npix + P - 1) / P, outer);
        const size_t smem = scan4_smem(n);
#define WDD_SCAN4(nn, a, b)                                                                  \
        if (n == nn)                                                                         \
            scan_axis4_kernel<T, a, b><<<grid, kOffThreads, smem, st>>>(src, dst, tw, P, npix, \
                                                                        outer_stride, es);
        WDD_FOUR_STEP_SIZES(WDD_SCAN4)
#undef WDD_SCAN4
        return cudaGetLastError();
    }
    const int P = scan_pixels_per_cta(n);
    const int logn = log2_exact(n);
    dim3 grid((npix + P - 1) / P, outer);
    const size_t smem = scan_smem(n);
    if (logn >= 0)
        scan_axis_kernel<T, true><<<grid, kOffThreads, smem, st>>>(src, dst, tw, n, logn, P, npix,
                                                                   outer_stride, es);
    else
        scan_axis_kernel<T, false><<<grid, kOffThreads, smem, st>>>(src, dst, tw, n, logn, P, npix,
                                                                    outer_stride, es);
    return cudaGetLastError();
}

// Inverse detector transform of every plane of X: MODE 0 reduces against K into d_o, MODE 1
// writes scale * the result back into X and folds its max |.|^2 into d_max.
template <int MODE>
cudaError_t launch_detector(const wdd_offline_plan* P, float2* X, cudaStream_t st) {
    const int Ny = P->Ny, Nx = P->Nx;
    const int ly = log2_exact(Ny), lx = log2_exact(Nx);
    const float scale = (float)(1.0 / ((double)Ny * (double)Nx));
    if (det4_square(Ny, Nx)) {
        const size_t smem = det4_smem(Nx);
#define WDD_DET4(nn, a, b)                                                                     \
        if (Nx == nn)                                                                          \
            det_fused4_kernel<MODE, a, b><<<P->S, kDetThreads, smem, st>>>(                    \
                X, P->d_K, P->d_mask, P->d_o, P->d_max, P->d_tw_dx, scale);
        WDD_DET4_SIZES(WDD_DET4)
#undef WDD_DET4
        return cudaGetLastError();
    }
    if (P->fused) {
        const size_t smem = fused_smem(Ny, Nx);
        if (ly >= 0 && lx >= 0)
            det_fused_kernel<MODE, true><<<P->S, kDetThreads, smem, st>>>(
                X, P->d_K, P->d_mask, P->d_o, P->d_max, P->d_tw_dy, P->d_tw_dx, Ny, Nx, ly, lx, scale);
        else
            det_fused_kernel<MODE, false><<<P->S, kDetThreads, smem, st>>>(
                X, P->d_K, P->d_mask, P->d_o, P->d_max, P->d_tw_dy, P->d_tw_dx, Ny, Nx, ly, lx, scale);
        return cudaGetLastError();
    }
    if (det2p4_len(Nx) && det2p4_len(Ny)) {
        {
            dim3 grid(P->S, (Ny + P->rb - 1) / P->rb);
            const size_t smem = sizeof(float2) * ((size_t)Nx + (size_t)P->rb * (Nx + Nx / 16 + 1));
#define WDD_ROWS4(nn, a, b)                                                                    \
            if (Nx == nn) det_rows4_kernel<a, b><<<grid, kOffThreads, smem, st>>>(X, P->d_tw_dx, Ny, P->rb);
            WDD_DET2P4_SIZES(WDD_ROWS4)
#undef WDD_ROWS4
        }
        {
            dim3 grid(P->S, P->ncb);
            const size_t smem = sizeof(float2) * ((size_t)Ny + (size_t)Ny * P->cp);
#define WDD_COLS4(nn, a, b)                                                                    \
            if (Ny == nn)                                                                      \
                det_cols4_kernel<MODE, a, b><<<grid, kOffThreads, smem, st>>>(                 \
                    X, P->d_K, P->d_mask, P->d_part, P->d_max, P->d_tw_dy, Nx, P->cp, scale);
            WDD_DET2P4_SIZES(WDD_COLS4)
#undef WDD_COLS4
        }
        if (MODE == 0)
            det_reduce_kernel<<<(P->S + kOffThreads - 1) / kOffThreads, kOffThreads, 0, st>>>(
                P->d_part, P->d_mask, P->d_o, P->S, P->ncb, scale);
        return cudaGetLastError();
    }
    {
        dim3 grid(P->S, (Ny + P->rb - 1) / P->rb);
        const size_t smem = sizeof(float2) * ((lx >= 0 ? Nx / 2 : Nx) + (size_t)P->rb * Nx);
        if (lx >= 0)
            det_rows_kernel<true><<<grid, kOffThreads, smem, st>>>(X, P->d_tw_dx, Ny, Nx, lx, P->rb);
        else
            det_rows_kernel<false><<<grid, kOffThreads, smem, st>>>(X, P->d_tw_dx, Ny, Nx, lx, P->rb);
    }
    {
        dim3 grid(P->S, P->ncb);
        const size_t smem = sizeof(float2) * ((ly >= 0 ? Ny / 2 : Ny) + (size_t)Ny * P->cp);
        if (ly >= 0)
            det_cols_kernel<MODE, true><<<grid, kOffThreads, smem, st>>>(
                X, P->d_K, P->d_mask, P->d_part, P->d_max, P->d_tw_dy, Ny, Nx, ly, P->cp, scale);
        else
            det_cols_kernel<MODE, false><<<grid, kOffThreads, smem, st>>>(
                X, P->d_K, P->d_mask, P->d_part, P->d_max, P->d_tw_dy, Ny, Nx, ly, P->cp, scale);
    }
    if (MODE == 0)
        det_reduce_kernel<<<(P->S + kOffThreads - 1) / kOffThreads, kOffThreads, 0, st>>>(
            P->d_part, P->d_mask, P->d_o, P->S, P->ncb, scale);
    return cudaGetLastError();
}

int64_t offline_planned_bytes(const wdd_offline_plan* P) {
    const int64_t big = (int64_t)P->S * P->npix * 8;
    int64_t b = 2 * big;
    b += (int64_t)P->S * (1 + 8 + 8) + 8 * (int64_t)(P->Sy + P->Sx);
    b += 8 * (int64_t)(2 * P->Sy + 2 * P->Sx + P->Ny + P->Nx);
    if (!P->fused) b += (int64_t)P->S * P->ncb * 8;
    if (P->swapped)
        b += 16 * ((int64_t)P->Sy * P->Ny * P->Sy + (int64_t)P->Ny * P->Sy +
                   (int64_t)P->Sx * P->Nx * P->Sx + (int64_t)P->Nx * P->Sx +
                   (int64_t)P->Sx * P->Sy * P->Nx + (int64_t)P->Sy * P->Nx +
                   (int64_t)P->Ny * P->Nx) +
             4 * (int64_t)P->S;
    return b + 4;
}

template <typename T>
wdd_status off_alloc(wdd_offline_plan* P, T** ptr, size_t count) {
    const size_t bytes = sizeof(T) * (count ? count : 1);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return off_fail(WDD_ERR_OUT_OF_MEMORY, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    P->allocs.push_back({p, bytes});
    P->device_bytes += (int64_t)bytes;
    *ptr = static_cast<T*>(p);
    return WDD_OK;
}

void off_release(wdd_offline_plan* P) {
    for (auto& a : P->allocs) cudaFree(a.ptr);
    P->allocs.clear();
}

// obj != NULL builds the plan of the swapped deconvolution (probe reconstruction, Sect. 10)
// from that object estimate: complex64 [Sy][Sx], device or pinned host memory, read during the
// call only.
wdd_status offline_create_impl(const wdd_params* prm, wdd_offline_plan** out, int64_t* footprint,
                               const void* obj) {
    if (!prm || !out) return off_fail(WDD_ERR_INVALID_ARG, "params or out is NULL");
    *out = nullptr;
    const wdd_params& p = *prm;
    if (p.scan_y <= 0 || p.scan_x <= 0 || p.det_y <= 0 || p.det_x <= 0)
        return off_fail(WDD_ERR_INVALID_ARG, "scan and detector sizes must be positive");
    if (p.scan_y > 4096 || p.scan_x > 4096)
        return off_fail(WDD_ERR_UNSUPPORTED, "scan side above 4096");
    if (p.det_y > 1024 || p.det_x > 1024)
        return off_fail(WDD_ERR_UNSUPPORTED, "detector side above 1024");
    if (!(p.scan_step_m > 0) || !(p.det_px_inv_m > 0) || !(p.voltage_v > 0) ||
        !(p.semiconv_rad > 0) || !std::isfinite(p.defocus_m))
        return off_fail(WDD_ERR_INVALID_ARG, "step, sampling, voltage and angle must be positive");
    if (!(p.epsilon >= 0) || !std::isfinite(p.epsilon))
        return off_fail(WDD_ERR_INVALID_ARG, "epsilon must be finite and non-negative");
    if (p.frame_dtype < WDD_FRAME_U16 || p.frame_dtype > WDD_FRAME_F64)
        return off_fail(WDD_ERR_INVALID_ARG, "unknown frame dtype");
    if (!std::isfinite(p.scan_rotation_rad))
        return off_fail(WDD_ERR_INVALID_ARG, "scan_rotation_rad must be finite");
    if (obj && p.scan_rotation_rad != 0.0)
        return off_fail(WDD_ERR_UNSUPPORTED,
                        "probe reconstruction on the GPU takes the object spectrum one scan axis "
                        "at a time: scan_rotation_rad must be 0");
    const bool cy_default = p.det_center_y < 0 || p.det_center_y == (double)(p.det_y / 2);
    const bool cx_default = p.det_center_x < 0 || p.det_center_x == (double)(p.det_x / 2);
    if (!cy_default || !cx_default)
        return off_fail(WDD_ERR_UNSUPPORTED,
                        "classical WDD moves the zero frequency by an integer roll: the detector "
                        "centre must be det / 2");

    wdd_offline_plan* P = new wdd_offline_plan();
    P->p = p;
    P->Sy = p.scan_y;
    P->Sx = p.scan_x;
    P->S = p.scan_y * p.scan_x;
    P->Ny = p.det_y;
    P->Nx = p.det_x;
    P->npix = p.det_y * p.det_x;
    P->fused = (fused_fits(P->Ny, P->Nx) || det4_square(P->Ny, P->Nx)) ? 1 : 0;
    P->rb = rows_per_cta(P->Nx);
    P->cp = cols_per_cta(P->Ny);
    P->ncb = (P->Nx + P->cp - 1) / P->cp;
    P->swapped = obj ? 1 : 0;
    P->lambda = electron_wavelength(p.voltage_v);
    P->R = p.semiconv_rad / (P->lambda * p.det_px_inv_m);
    std::vector<double> qy, qx;
    std::vector<uint8_t> mask;
    P->n_active = scan_geometry(p, P->R, qy, qx, mask);

    const int64_t need = offline_planned_bytes(P);
    if (footprint) {
        *footprint = need;
        delete P;
        return WDD_OK;
    }
    if (p.hbm_budget_bytes > 0 && need > p.hbm_budget_bytes) {
        delete P;
        char buf[160];
        std::snprintf(buf, sizeof buf, "classical plan needs %lld bytes, budget is %lld",
                      (long long)need, (long long)p.hbm_budget_bytes);
        return off_fail(WDD_ERR_OUT_OF_MEMORY, buf);
    }
    const float2* O = nullptr;  // the object estimate as a device address (swapped plan)
    if (obj) {
        cudaPointerAttributes attr{};
        if (cudaPointerGetAttributes(&attr, obj) != cudaSuccess) {
            cudaGetLastError();
            attr.type = cudaMemoryTypeUnregistered;
        }
        if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)
            O = static_cast<const float2*>(obj);
        else if (attr.type == cudaMemoryTypeHost)
            O = static_cast<const float2*>(attr.devicePointer ? attr.devicePointer : obj);
        if (!O) {
            delete P;
            return off_fail(WDD_ERR_INVALID_ARG,
                            "object estimate must be in device or pinned host memory");
        }
    }
    {
        cudaError_t pe = prepare_offline_kernels();
        if (pe == cudaSuccess) pe = prepare_kernels();
        if (pe != cudaSuccess) {
            delete P;
            return off_cuda_fail(pe, "kernel attributes");
        }
    }
    wdd_status sst = WDD_OK;
#define WDD_OFF_ALLOC(ptr, n)                                           \
    do {                                                                \
        sst = off_alloc(P, &(ptr), (n));                                \
        if (sst != WDD_OK) { off_release(P); delete P; return sst; }    \
    } while (0)
    const size_t big = (size_t)P->S * P->npix;
    WDD_OFF_ALLOC(P->d_G, big);
    WDD_OFF_ALLOC(P->d_K, big);
    WDD_OFF_ALLOC(P->d_mask, P->S);
    WDD_OFF_ALLOC(P->d_qy, P->Sy);
    WDD_OFF_ALLOC(P->d_qx, P->Sx);
    WDD_OFF_ALLOC(P->d_tw_sy, P->Sy);
    WDD_OFF_ALLOC(P->d_tw_sx, P->Sx);
    WDD_OFF_ALLOC(P->d_tw_dy, P->Ny);
    WDD_OFF_ALLOC(P->d_tw_dx, P->Nx);
    WDD_OFF_ALLOC(P->d_twy_inv, P->Sy);
    WDD_OFF_ALLOC(P->d_twx_inv, P->Sx);
    WDD_OFF_ALLOC(P->d_o, P->S);
    WDD_OFF_ALLOC(P->d_tmp, P->S);
    WDD_OFF_ALLOC(P->d_max, 1);
    if (!P->fused) WDD_OFF_ALLOC(P->d_part, (size_t)P->S * P->ncb);
    if (P->swapped) {
        WDD_OFF_ALLOC(P->d_Ey, (size_t)P->Sy * P->Ny * P->Sy);
        WDD_OFF_ALLOC(P->d_Ey0, (size_t)P->Ny * P->Sy);
        WDD_OFF_ALLOC(P->d_Ex, (size_t)P->Sx * P->Nx * P->Sx);
        WDD_OFF_ALLOC(P->d_Ex0, (size_t)P->Nx * P->Sx);
        WDD_OFF_ALLOC(P->d_T, (size_t)P->Sx * P->Sy * P->Nx);
        WDD_OFF_ALLOC(P->d_T0, (size_t)P->Sy * P->Nx);
        WDD_OFF_ALLOC(P->d_Psi0, (size_t)P->Ny * P->Nx);
        WDD_OFF_ALLOC(P->d_vmax, P->S);
    }
#undef WDD_OFF_ALLOC

    cudaStream_t s0 = nullptr;
    auto cbail = [&](cudaError_t e, const char* w) {
        off_cuda_fail(e, w);
        off_release(P);
        delete P;
        return WDD_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMemcpy(P->d_qy, qy.data(), 8 * P->Sy, cudaMemcpyHostToDevice))) return cbail(e, "copy shifts");
    if ((e = cudaMemcpy(P->d_qx, qx.data(), 8 * P->Sx, cudaMemcpyHostToDevice))) return cbail(e, "copy shifts");
    if ((e = cudaMemcpy(P->d_mask, mask.data(), P->S, cudaMemcpyHostToDevice))) return cbail(e, "copy mask");
    auto tw = [&](float2* d, int n) {
        twiddle_kernel<<<(n + kOffThreads - 1) / kOffThreads, kOffThreads, 0, s0>>>(d, n);
    };
    tw(P->d_tw_sy, P->Sy);
    tw(P->d_tw_sx, P->Sx);
    tw(P->d_tw_dy, P->Ny);
    tw(P->d_tw_dx, P->Nx);
    if ((e = launch_idft_tables(P->d_twy_inv, P->Sy, P->d_twx_inv, P->Sx, s0))) return cbail(e, "tables");

    const int64_t total = (int64_t)big;
    const int ew_blocks = (int)std::min<int64_t>((total + kOffThreads - 1) / kOffThreads, 152 * 64);
    if (P->swapped) {
        // ---- Wiener kernel of the swapped deconvolution: Omega_v from the object estimate,
        // W_O = IFFT2(ifftshift Omega_v), eps_v = epsilon max_r |W_O(v, r)|^2 per frequency,
        // conj(W_O) / (|W_O|^2 + eps_v) ----
        const double dks = p.det_px_inv_m * p.scan_step_m;
        auto table = [&](double2* E, const double* q, int nv, int n, int ns, double c) {
            const int64_t tot = (int64_t)nv * n * ns;
            const int b = (int)std::min<int64_t>((tot + kOffThreads - 1) / kOffThreads, 152 * 64);
            axis_dtft_table_kernel<<<b, kOffThreads, 0, s0>>>(E, q, nv, n, ns, c, dks);
        };
        auto xsum = [&](const double2* E, double2* T, int nu) {
            const int64_t tot = (int64_t)nu * P->Sy * P->Nx;
            const int b = (int)std::min<int64_t>((tot + kOffThreads - 1) / kOffThreads, 152 * 64);
            obj_xsum_kernel<<<b, kOffThreads, 0, s0>>>(O, E, T, nu, P->Sy, P->Sx, P->Nx);
        };
        table(P->d_Ey, P->d_qy, P->Sy, P->Ny, P->Sy, (double)(P->Ny / 2));
        table(P->d_Ey0, nullptr, 1, P->Ny, P->Sy, (double)(P->Ny / 2));
        table(P->d_Ex, P->d_qx, P->Sx, P->Nx, P->Sx, (double)(P->Nx / 2));
        table(P->d_Ex0, nullptr, 1, P->Nx, P->Sx, (double)(P->Nx / 2));
        xsum(P->d_Ex, P->d_T, P->Sx);
        xsum(P->d_Ex0, P->d_T0, 1);
        psi0_kernel<<<(P->npix + kOffThreads - 1) / kOffThreads, kOffThreads, 0, s0>>>(
            P->d_Ey0, P->d_T0, P->d_Psi0, P->Sy, P->Ny, P->Nx);
        omega_kernel<<<ew_blocks, kOffThreads, 0, s0>>>(P->d_K, P->d_Ey, P->d_T, P->d_Psi0,
                                                        P->Sy, P->Sx, P->Ny, P->Nx, total);
        if ((e = cudaGetLastError())) return cbail(e, "object autocorrelation");
        if ((e = cudaMemset(P->d_max, 0, 4))) return cbail(e, "zero max");
        if ((e = launch_detector<1>(P, P->d_K, s0))) return cbail(e, "object transform");
        plane_max_kernel<<<P->S, kOffThreads, 0, s0>>>(P->d_K, P->d_vmax, P->npix);
        if ((e = cudaGetLastError())) return cbail(e, "plane maxima");
        unsigned maxbits = 0;
        if ((e = cudaMemcpy(&maxbits, P->d_max, 4, cudaMemcpyDeviceToHost))) return cbail(e, "max");
        float maxwo;
        std::memcpy(&maxwo, &maxbits, 4);
        P->eps_eff = p.eps_absolute ? p.epsilon : p.epsilon * (double)maxwo;
        if (!(maxwo > 0)) {
            off_release(P);
            delete P;
            return off_fail(WDD_ERR_INVALID_ARG, "object autocorrelation is zero everywhere");
        }
        wiener_pf_kernel<<<ew_blocks, kOffThreads, 0, s0>>>(P->d_K, P->d_mask, P->d_vmax, P->npix,
                                                            total, (float)p.epsilon,
                                                            p.eps_absolute ? 1 : 0);
        if ((e = cudaGetLastError())) return cbail(e, "Wiener kernel");
        if ((e = cudaDeviceSynchronize())) return cbail(e, "probe plan build");
        *out = P;
        return WDD_OK;
    }

    // ---- Wiener kernel: Y_v, W_P = IFFT2(ifftshift Y_v), eps_eff, conj(W_P) / (|W_P|^2 + eps) ----
    const double R2 = P->R * P->R;
    const double coef = 3.14159265358979323846 * P->lambda * p.defocus_m *
                        (p.det_px_inv_m * p.det_px_inv_m);
    const double rc = std::cos(p.scan_rotation_rad), rs = std::sin(p.scan_rotation_rad);
    probe_autocorr_kernel<<<ew_blocks, kOffThreads, 0, s0>>>(
        P->d_K, P->d_qy, P->d_qx, P->Sx, P->Ny, P->Nx, (double)(P->Ny / 2), (double)(P->Nx / 2),
        R2, coef, rc, rs, total);
    if ((e = cudaGetLastError())) return cbail(e, "probe autocorrelation");
    if ((e = cudaMemset(P->d_max, 0, 4))) return cbail(e, "zero max");
    if ((e = launch_detector<1>(P, P->d_K, s0))) return cbail(e, "probe transform");
    unsigned maxbits = 0;
    if ((e = cudaMemcpy(&maxbits, P->d_max, 4, cudaMemcpyDeviceToHost))) return cbail(e, "max");
    float maxwp;
    std::memcpy(&maxwp, &maxbits, 4);
    P->eps_eff = p.eps_absolute ? p.epsilon : p.epsilon * (double)maxwp;
    if (!(P->eps_eff > 0) && p.epsilon > 0) {
        off_release(P);
        delete P;
        return off_fail(WDD_ERR_INVALID_ARG, "probe autocorrelation is zero everywhere");
    }
    wiener_kernel<<<ew_blocks, kOffThreads, 0, s0>>>(P->d_K, P->d_mask, P->npix, total,
                                                     (float)P->eps_eff);
    if ((e = cudaGetLastError())) return cbail(e, "Wiener kernel");
    if ((e = cudaDeviceSynchronize())) return cbail(e, "classical plan build");
    *out = P;
    return WDD_OK;
}

}  // namespace
}  // namespace wdd

using namespace wdd;

wdd_status wdd_offline_plan_create(const wdd_params* p, wdd_offline_plan** out) {
    return offline_create_impl(p, out, nullptr, nullptr);
}

wdd_status wdd_offline_probe_plan_create(const wdd_params* p, const void* obj,
                                         wdd_offline_plan** out) {
    if (!obj) {
        if (out) *out = nullptr;
        return off_fail(WDD_ERR_INVALID_ARG, "object estimate is NULL");
    }
    return offline_create_impl(p, out, nullptr, obj);
}

wdd_status wdd_offline_footprint(const wdd_params* p, int64_t* bytes) {
    if (!bytes) return off_fail(WDD_ERR_INVALID_ARG, "bytes is NULL");
    wdd_offline_plan* unused = nullptr;
    return offline_create_impl(p, &unused, bytes, nullptr);
}

wdd_status wdd_offline_plan_destroy(wdd_offline_plan* P) {
    if (!P) return off_fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    cudaDeviceSynchronize();
    off_release(P);
    delete P;
    return WDD_OK;
}

wdd_status wdd_offline_reconstruct(wdd_offline_plan* P, const void* frames, wdd_result* out,
                                   wdd_stream_t stream) {
    if (!P || !frames || !out || !out->obj)
        return off_fail(WDD_ERR_INVALID_ARG, "plan, frames, out and out->obj must not be NULL");
    cudaPointerAttributes attr{};
    cudaError_t e = cudaPointerGetAttributes(&attr, frames);
    if (e != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    const void* src = nullptr;
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)
        src = frames;
    else if (attr.type == cudaMemoryTypeHost)
        src = attr.devicePointer ? attr.devicePointer : frames;
    else
        return off_fail(WDD_ERR_INVALID_ARG, "frames must be in device or pinned host memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int npix = P->npix;
    const int64_t sx_stride = (int64_t)P->Sx * npix;
    // Eq. 2: forward transform over s_x (from the frames), then over s_y (in place)
    switch (P->p.frame_dtype) {
        case WDD_FRAME_U16:
            e = launch_scan_axis(static_cast<const uint16_t*>(src), P->d_G, P->d_tw_sx, P->Sx, npix,
                                 P->Sy, sx_stride, npix, st);
            break;
        case WDD_FRAME_F32:
            e = launch_scan_axis(static_cast<const float*>(src), P->d_G, P->d_tw_sx, P->Sx, npix,
                                 P->Sy, sx_stride, npix, st);
            break;
        default:
            e = launch_scan_axis(static_cast<const double*>(src), P->d_G, P->d_tw_sx, P->Sx, npix,
                                 P->Sy, sx_stride, npix, st);
            break;
    }
    if (e == cudaSuccess)
        e = launch_scan_axis(static_cast<const float2*>(P->d_G), P->d_G, P->d_tw_sy, P->Sy, npix,
                             P->Sx, npix, sx_stride, st);
    // Eq. 2-3: detector transform, Wiener product and the sum over r
    if (e == cudaSuccess) e = launch_detector<0>(P, P->d_G, st);
    // Eq. 3: normalisation, conjugated inverse DFT over the scan
    if (e == cudaSuccess)
        e = launch_idft(P->d_o, P->d_twx_inv, P->d_twy_inv, P->d_tmp, P->Sy, P->Sx,
                        static_cast<float2*>(out->obj), out->phase, st);
    // swapped plan: the probe IFFT2(conj(p / sqrt(p_0))) is that result at the negated index
    if (e == cudaSuccess && P->swapped) {
        e = cudaMemcpyAsync(P->d_tmp, out->obj, 8 * (size_t)P->S, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) {
            negate_index_kernel<<<(P->S + kOffThreads - 1) / kOffThreads, kOffThreads, 0, st>>>(
                P->d_tmp, static_cast<float2*>(out->obj), out->phase, P->Sy, P->Sx);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return off_cuda_fail(e, "classical reconstruction");
    out->frames_seen = P->S;
    out->positions_covered = P->S;
    return WDD_OK;
}

wdd_status wdd_offline_copy_array(wdd_offline_plan* P, int32_t which, void* dst, int64_t bytes,
                                  int64_t* written) {
    if (!P || !dst) return off_fail(WDD_ERR_INVALID_ARG, "plan or destination is NULL");
    const void* src = nullptr;
    size_t size = 0;
    switch (which) {
        case WDD_OFFLINE_SPECTRUM: src = P->d_o; size = 8 * (size_t)P->S; break;
        case WDD_OFFLINE_WIENER: src = P->d_K; size = 8 * (size_t)P->S * P->npix; break;
        case WDD_OFFLINE_MASK: src = P->d_mask; size = (size_t)P->S; break;
        default: return off_fail(WDD_ERR_INVALID_ARG, "unknown array");
    }
    if (bytes < (int64_t)size) return off_fail(WDD_ERR_INVALID_ARG, "destination too small");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(dst, src, size, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return off_cuda_fail(e, "copy");
    if (written) *written = (int64_t)size;
    return WDD_OK;
}

wdd_status wdd_offline_get_info(const wdd_offline_plan* P, int64_t* device_bytes,
                                int32_t* n_active, int32_t* fused, double* eps_eff) {
    if (!P) return off_fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    if (device_bytes) *device_bytes = P->device_bytes;
    if (n_active) *n_active = P->n_active;
    if (fused) *fused = P->fused;
    if (eps_eff) *eps_eff = P->eps_eff;
    return WDD_OK;
}
