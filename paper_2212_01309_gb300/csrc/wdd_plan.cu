// Plan-time kernels (FP64): reduced bases, projected probe autocorrelation chi_v and the Wiener
// filter of Algorithm 1, and the scan-phase tables of Algorithm 2's initialisation.
//
// Decisions that turn floating point into a yes/no (is a detector point inside the shifted
// aperture?) are evaluated with explicitly rounded FP64 operations (__dmul_rn / __dadd_rn, no
// fused multiply-add) in the order ky*ky + kx*kx <= R*R, so that the CPU oracle, which evaluates
// the same expression in IEEE double, takes the same decision on every pixel.

#include <cuda_fp16.h>

#include <cmath>

#include "wdd_device.cuh"
#include "wdd_internal.h"

namespace wdd {

namespace {

__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b) {  // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Normalised 1-D oscillator eigenfunctions (Eq. 7) by the three-term recurrence:
//   psi_0 = pi^-1/4 exp(-x^2/2), psi_1 = sqrt(2) x psi_0,
//   psi_{n+1} = sqrt(2/(n+1)) x psi_n - sqrt(n/(n+1)) psi_{n-1},  x = (j - center) / sigma.
// One thread per sample; column norms are fixed by hg_normalise_kernel.
__global__ void hg_basis_kernel(double2* B, int n, int L, double sigma, double center) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double x = ((double)j - center) / sigma;
    double pm1 = 0.0;
    double p0 = 0.75112554446494248286 * exp(-0.5 * x * x);  // pi^(-1/4)
    B[(size_t)j * L] = make_double2(p0, 0.0);
    if (L > 1) {
        double p1 = 1.41421356237309504880 * x * p0;
        B[(size_t)j * L + 1] = make_double2(p1, 0.0);
        pm1 = p0;
        p0 = p1;
        for (int k = 1; k < L - 1; ++k) {
            double nxt = sqrt(2.0 / (k + 1)) * x * p0 - sqrt((double)k / (k + 1.0)) * pm1;
            B[(size_t)j * L + k + 1] = make_double2(nxt, 0.0);
            pm1 = p0;
            p0 = nxt;
        }
    }
}

// Scales every column of B (n x L) to unit discrete L2 norm; one block per column.
__global__ void hg_normalise_kernel(double2* B, int n, int L) {
    __shared__ double red[kThreads];
    int col = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double v = B[(size_t)j * L + col].x;
        s += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    double nrm = sqrt(red[0]);
    if (nrm == 0.0) nrm = 1.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) B[(size_t)j * L + col].x /= nrm;
}

// Fourier family: B[j][r] = exp(+2 pi i (j - center) r / n) / n (inverse-DFT rows).
__global__ void fourier_basis_kernel(double2* B, int n, double center) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * n) return;
    int j = t / n, r = t % n;
    double s, c;
    sincospi(2.0 * (((double)j - center) * (double)r) / (double)n, &s, &c);
    B[t] = make_double2(c / n, s / n);
}

constexpr int kChiRows = 8;

// chi_v = By^T Y_v Bx for one scan frequency v per block, Y_v(q) = p(q) conj p(q + q_v)
// (Algorithm 1), with q_v the scan-axis shift (qy, qx) turned by the scan rotation (rc, rs):
// (rc qy - rs qx, rs qy + rc qx) along the detector axes (exact for rc = 1, rs = 0).  Y is built row block by row block in shared memory; Z accumulates in registers.
// Also folds max |chi_v[m]|^2 over the used indices into *maxbits (as ordered uint64 bits).
template <int ZPT>
__global__ void __launch_bounds__(kThreads)
chi_kernel(const double2* __restrict__ By, const double2* __restrict__ Bx,
           const double* __restrict__ qy, const double* __restrict__ qx,
           const uint8_t* __restrict__ used, double2* __restrict__ chi,
           unsigned long long* maxbits, int Sx, int Ny, int Nx, int Ly, int Lx,
           double cy, double cx, double R, double R2, double coef, double rc, double rs) {
    extern __shared__ double2 sm[];
    double2* sBx = sm;                          // Nx * Lx
    double2* sY = sBx + (size_t)Nx * Lx;        // kChiRows * Nx
    double2* sT = sY + (size_t)kChiRows * Nx;   // kChiRows * Lx
    __shared__ double red[kThreads];

    const int v = blockIdx.x;
    const double sa = qy[v / Sx];
    const double sb = qx[v % Sx];
    const double shy = __dsub_rn(__dmul_rn(rc, sa), __dmul_rn(rs, sb));
    const double shx = __dadd_rn(__dmul_rn(rs, sa), __dmul_rn(rc, sb));
    const int M = Ly * Lx;

    for (int t = threadIdx.x; t < Nx * Lx; t += blockDim.x) sBx[t] = Bx[t];

    double2 z[ZPT];
#pragma unroll
    for (int u = 0; u < ZPT; ++u) z[u] = make_double2(0.0, 0.0);

    for (int i0 = 0; i0 < Ny; i0 += kChiRows) {
        // skip row blocks that lie entirely outside the unshifted aperture
        double dlo = (double)i0 - cy, dhi = (double)(i0 + kChiRows - 1) - cy;
        double dmin = (dlo > 0) ? dlo : ((dhi < 0) ? -dhi : 0.0);
        if (dmin > R + 1.0) continue;
        __syncthreads();
        for (int t = threadIdx.x; t < kChiRows * Nx; t += blockDim.x) {
            int r = t / Nx, j = t % Nx, i = i0 + r;
            double2 y = make_double2(0.0, 0.0);
            if (i < Ny) {
                double ky = (double)i - cy;
                double kx = (double)j - cx;
                double k2 = __dadd_rn(__dmul_rn(ky, ky), __dmul_rn(kx, kx));
                double2 a = probe_at(k2, R2, coef);
                if (a.x != 0.0 || a.y != 0.0) {
                    double ky2 = __dadd_rn(ky, shy);
                    double kx2 = __dadd_rn(kx, shx);
                    double k2s = __dadd_rn(__dmul_rn(ky2, ky2), __dmul_rn(kx2, kx2));
                    double2 b = probe_at(k2s, R2, coef);
                    y = cmul_conj(a, b);
                }
            }
            sY[t] = y;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < kChiRows * Lx; t += blockDim.x) {
            int r = t / Lx, lx = t % Lx;
            double2 acc = make_double2(0.0, 0.0);
            const double2* yr = sY + (size_t)r * Nx;
            for (int j = 0; j < Nx; ++j) {
                double2 y = yr[j];
                double2 b = sBx[(size_t)j * Lx + lx];
                acc.x += y.x * b.x - y.y * b.y;
                acc.y += y.x * b.y + y.y * b.x;
            }
            sT[t] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < ZPT; ++u) {
            int o = threadIdx.x + u * kThreads;
            if (o < M) {
                int ly = o / Lx, lx = o % Lx;
                for (int r = 0; r < kChiRows && i0 + r < Ny; ++r) {
                    double2 b = By[(size_t)(i0 + r) * Ly + ly];
                    double2 tt = sT[r * Lx + lx];
                    z[u].x += b.x * tt.x - b.y * tt.y;
                    z[u].y += b.x * tt.y + b.y * tt.x;
                }
            }
        }
    }
    double mx = 0.0;
#pragma unroll
    for (int u = 0; u < ZPT; ++u) {
        int o = threadIdx.x + u * kThreads;
        if (o < M) {
            chi[(size_t)v * M + o] = z[u];
            if (used[o]) {
                double a2 = z[u].x * z[u].x + z[u].y * z[u].y;
                mx = a2 > mx ? a2 : mx;
            }
        }
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(red[0]));
}

__device__ __forceinline__ double2 wiener(double2 z, double eps) {
    double d = z.x * z.x + z.y * z.y + eps;
    return make_double2(z.x / d, -z.y / d);
}

// W_v[k] from chi_v (Algorithm 1: K_v = conj(chi_v) / (|chi_v|^2 + eps_eff)).  Hermite-Gauss
// rows take K_v[m_k]; Fourier cos/sin rows pair r with -r:
//   W[cos r] = K(r) + K(-r)  (K(r) when r = -r),  W[sin r] = i (K(r) - K(-r)).
__global__ void weights_kernel(const double2* __restrict__ chi, const int2* __restrict__ ktab,
                               const uint8_t* __restrict__ mask, float2* __restrict__ W,
                               int S, int K, int Ly, int Lx, int complex_basis, double eps) {
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)S * K) return;
    int v = (int)(t / K), k = (int)(t % K);
    if (!mask[v]) {
        W[t] = make_float2(0.f, 0.f);
        return;
    }
    int M = Ly * Lx;
    int2 e = ktab[k];
    double2 Kr = wiener(chi[(size_t)v * M + e.x], eps);
    double2 w;
    if (!complex_basis) {
        w = Kr;
    } else {
        int ry = e.x / Lx, rx = e.x % Lx;
        int mn = ((Ly - ry) % Ly) * Lx + (Lx - rx) % Lx;
        double2 Kn = wiener(chi[(size_t)v * M + mn], eps);
        if (e.y == 0) {
            w = (mn == e.x) ? Kr : make_double2(Kr.x + Kn.x, Kr.y + Kn.y);
        } else {
            // i * (Kr - Kn)
            w = make_double2(-(Kr.y - Kn.y), Kr.x - Kn.x);
        }
    }
    W[t] = make_float2((float)w.x, (float)w.y);
}

// exp(-2 pi i m / lcm) (forward scan phase) in FP32 and as an FP16 hi/lo split packed as
// (re_hi | re_lo << 16, im_hi | im_lo << 16), and the inverse
// DFT twiddles exp(+2 pi i m / n) for both scan axes.
__global__ void tables_kernel(float2* tw, uint2* tw16, int lcm, float2* twy, int Sy, float2* twx,
                              int Sx) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < lcm) {
        double s, c;
        sincospi(2.0 * (double)t / (double)lcm, &s, &c);
        double re = c, im = -s;
        tw[t] = make_float2((float)re, (float)im);
        __half rh = __double2half(re);
        __half rl = __double2half(re - (double)__half2float(rh));
        __half ih = __double2half(im);
        __half il = __double2half(im - (double)__half2float(ih));
        tw16[t] = make_uint2((uint32_t)__half_as_ushort(rh) | ((uint32_t)__half_as_ushort(rl) << 16),
                             (uint32_t)__half_as_ushort(ih) | ((uint32_t)__half_as_ushort(il) << 16));
    }
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

// Detector centre of mass, pass 1: per-pixel sums over one contiguous group of frames
// (blockIdx.y), in FP64 in frame order.  part is [groups][npix].
template <typename FT>
__global__ void com_partial_kernel(const FT* __restrict__ f, int64_t n, int npix, int64_t per,
                                   double* __restrict__ part) {
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    const int64_t f0 = (int64_t)blockIdx.y * per;
    const int64_t f1 = f0 + per < n ? f0 + per : n;
    double s = 0.0;
    for (int64_t t = f0; t < f1; ++t) s += (double)f[t * npix + pix];
    part[(size_t)blockIdx.y * npix + pix] = s;
}

// Pass 2 (one block of kComThreads): pixel sums over the groups in group order, then the total
// and the row- and column-weighted totals, reduced over the block in a fixed tree.
constexpr int kComThreads = 1024;
__global__ void __launch_bounds__(kComThreads)
com_final_kernel(const double* __restrict__ part, int groups, int Ny, int Nx,
                 double* __restrict__ out) {
    __shared__ double red[3][kComThreads];
    const int npix = Ny * Nx;
    double s0 = 0.0, sy = 0.0, sx = 0.0;
    for (int pix = threadIdx.x; pix < npix; pix += kComThreads) {
        double v = 0.0;
        for (int g = 0; g < groups; ++g) v += part[(size_t)g * npix + pix];
        s0 += v;
        sy += v * (double)(pix / Nx);
        sx += v * (double)(pix % Nx);
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = sy;
    red[2][threadIdx.x] = sx;
    __syncthreads();
    for (int w = kComThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

cudaError_t launch_detector_center(const void* frames, int64_t n, int Ny, int Nx, int dtype,
                                   double sums[3], cudaStream_t st) {
    const int npix = Ny * Nx;
    const int pix_blocks = (npix + kThreads - 1) / kThreads;
    // about four blocks per SM over the pixel blocks and frame groups
    int64_t groups = (4 * 152 + pix_blocks - 1) / pix_blocks;
    if (groups > n) groups = n;
    if (groups > 65535) groups = 65535;
    if (groups < 1) groups = 1;
    const int64_t per = (n + groups - 1) / groups;
    groups = (n + per - 1) / per;
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * ((size_t)groups * npix + 3));
    if (e != cudaSuccess) return e;
    dim3 grid(pix_blocks, (unsigned)groups);
    switch (dtype) {
        case WDD_FRAME_U16:
            com_partial_kernel<<<grid, kThreads, 0, st>>>(static_cast<const uint16_t*>(frames), n,
                                                          npix, per, d + 3);
            break;
        case WDD_FRAME_F32:
            com_partial_kernel<<<grid, kThreads, 0, st>>>(static_cast<const float*>(frames), n,
                                                          npix, per, d + 3);
            break;
        default:
            com_partial_kernel<<<grid, kThreads, 0, st>>>(static_cast<const double*>(frames), n,
                                                          npix, per, d + 3);
            break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        com_final_kernel<<<1, kComThreads, 0, st>>>(d + 3, (int)groups, Ny, Nx, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sums, d, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(d);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_hg_basis(double2* B, int n, int L, double sigma, double center, cudaStream_t st) {
    hg_basis_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(B, n, L, sigma, center);
    hg_normalise_kernel<<<L, kThreads, 0, st>>>(B, n, L);
    return cudaGetLastError();
}

cudaError_t launch_fourier_basis(double2* B, int n, double center, cudaStream_t st) {
    fourier_basis_kernel<<<(n * n + kThreads - 1) / kThreads, kThreads, 0, st>>>(B, n, center);
    return cudaGetLastError();
}

cudaError_t launch_chi(const wdd_plan* P, unsigned long long* d_maxbits, cudaStream_t st) {
    // used-index flags
    std::vector<uint8_t> used(P->M, 0);
    for (int k = 0; k < P->K; ++k) {
        int m = P->h_ktab[2 * k];
        used[m] = 1;
        if (P->complex_basis) {
            int ry = m / P->Lx, rx = m % P->Lx;
            used[((P->Ly - ry) % P->Ly) * P->Lx + (P->Lx - rx) % P->Lx] = 1;
        }
    }
    uint8_t* d_used = nullptr;
    cudaError_t e = cudaMalloc(&d_used, P->M);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d_used, used.data(), P->M, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { cudaFree(d_used); return e; }
    size_t smem = sizeof(double2) * ((size_t)P->Nx * P->Lx + (size_t)kChiRows * P->Nx +
                                     (size_t)kChiRows * P->Lx);
    int zpt = (P->M + kThreads - 1) / kThreads;
    double R2 = P->R * P->R;
    double coef = 3.14159265358979323846 * P->lambda * P->p.defocus_m *
                  (P->p.det_px_inv_m * P->p.det_px_inv_m);
    const double rc = std::cos(P->p.scan_rotation_rad), rs = std::sin(P->p.scan_rotation_rad);
#define WDD_CHI(Z)                                                                                \
    do {                                                                                          \
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(chi_kernel<Z>));                 \
        if (e == cudaSuccess)                                                                     \
            chi_kernel<Z><<<P->S, kThreads, smem, st>>>(P->d_By, P->d_Bx, P->d_qy, P->d_qx,       \
                                                        d_used, P->d_chi, d_maxbits, P->Sx,       \
                                                        P->Ny, P->Nx, P->Ly, P->Lx, P->cy, P->cx, \
                                                        P->R, R2, coef, rc, rs);                  \
    } while (0)
    if (zpt <= 1) WDD_CHI(1);
    else if (zpt <= 2) WDD_CHI(2);
    else if (zpt <= 4) WDD_CHI(4);
    else if (zpt <= 8) WDD_CHI(8);
    else if (zpt <= 16) WDD_CHI(16);
    else e = cudaErrorInvalidValue;
#undef WDD_CHI
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(d_used);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_weights(const wdd_plan* P, cudaStream_t st) {
    size_t n = (size_t)P->S * P->K;
    weights_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        P->d_chi, P->d_ktab, P->d_mask, P->d_W, P->S, P->K, P->Ly, P->Lx, P->complex_basis,
        P->eps_eff);
    return cudaGetLastError();
}

cudaError_t launch_tables(const wdd_plan* P, cudaStream_t st) {
    int n = P->lcm;
    if (P->Sy > n) n = P->Sy;
    if (P->Sx > n) n = P->Sx;
    tables_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(
        P->d_tw, P->d_tw16, P->lcm, P->d_twy, P->Sy, P->d_twx, P->Sx);
    return cudaGetLastError();
}

}  // namespace wdd
