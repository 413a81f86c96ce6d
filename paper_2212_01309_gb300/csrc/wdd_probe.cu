// Wiener filter update from a recovered probe (Sect. 10): Algorithm 1 rebuilt on a live plan with
//   Y_v(q) = A(q) conj A(q + q_v),   A(k) = [|k|^2 <= R^2] exp(i arg P(k)),
// where P(k) = sum_s probe_s exp(-2 pi i dk k . r_s) is the spectrum of the recovered probe (given
// on the scan grid, e.g. by the swapped classical plan) at detector-pixel frequencies: the known
// condenser aperture keeps its support and amplitude, the recovered probe supplies the phase
// inside it.  chi_v = By^T Y_v Bx, eps_eff and the weights follow exactly as at plan creation; the
// accumulator is untouched, so the next snapshot deconvolves every frame pushed so far with the
// updated filter.
//
// Without a scan rotation the trigonometric sum separates into one sum per scan axis: tables
// E[v][i][s] = exp(-2 pi i frac(((i - c + q[v]) dk Delta) s)) per axis, the x sums of the probe
// T[vx][sy][j] = sum_sx probe[sy][sx] Ex[vx][j][sx], and P at the shifted pixel (i, j) of
// frequency v = sum_sy Ey[vy][i][sy] T[vx][sy][j], all in FP64.  Aperture membership is decided
// with explicitly rounded FP64 operations in the order ky*ky + kx*kx <= R*R, as everywhere else.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "wdd_device.cuh"
#include "wdd_internal.h"

namespace wdd {
namespace {

constexpr int kRows = 8;   // detector rows of Y_v staged per pass

__device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 c) {  // c + a b
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// exp(i arg z); 1 for z == 0
__device__ __forceinline__ double2 unit_phase(double2 z) {
    const double r = hypot(z.x, z.y);
    return r > 0.0 ? make_double2(z.x / r, z.y / r) : make_double2(1.0, 0.0);
}

// E[(v * n + i) * ns + s] = exp(-2 pi i frac(((i - c + q[v]) * dks) * s)) (q == NULL: no shift).
__global__ void probe_table_kernel(double2* __restrict__ E, const double* __restrict__ q, int nv,
                                   int n, int ns, double c, double dks) {
    const int64_t total = (int64_t)nv * n * ns;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(t % ns);
        const int64_t r = t / ns;
        const int i = (int)(r % n);
        const int v = (int)(r / n);
        const double k = (double)i - c + (q ? q[v] : 0.0);
        const double ph = (k * dks) * (double)s;
        const double f = ph - floor(ph);
        double sn, cs;
        sincospi(-2.0 * f, &sn, &cs);
        E[t] = make_double2(cs, sn);
    }
}

// T[(u * Sy + sy) * Nx + j] = sum_sx probe[sy][sx] Ex[(u * Nx + j) * Sx + sx], u < nu.
__global__ void probe_xsum_kernel(const float2* __restrict__ Pr, const double2* __restrict__ Ex,
                                  double2* __restrict__ T, int nu, int Sy, int Sx, int Nx) {
    const int64_t total = (int64_t)nu * Sy * Nx;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % Nx);
        const int64_t r = t / Nx;
        const int sy = (int)(r % Sy);
        const int u = (int)(r / Sy);
        const float2* pr = Pr + (size_t)sy * Sx;
        const double2* e = Ex + ((size_t)u * Nx + j) * Sx;
        double2 acc = make_double2(0.0, 0.0);
        for (int sx = 0; sx < Sx; ++sx) {
            const float2 pv = pr[sx];
            acc = zfma(make_double2(pv.x, pv.y), e[sx], acc);
        }
        T[t] = acc;
    }
}

// A0[i][j] = [inside the aperture] exp(i arg sum_sy Ey0[i][sy] T0[sy][j]) at k = (i - cy, j - cx).
__global__ void probe_a0_kernel(const double2* __restrict__ Ey0, const double2* __restrict__ T0,
                                double2* __restrict__ A0, int Sy, int Ny, int Nx, double cy,
                                double cx, double R2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Ny * Nx) return;
    const int i = t / Nx, j = t - (t / Nx) * Nx;
    const double ky = (double)i - cy, kx = (double)j - cx;
    const double k2 = __dadd_rn(__dmul_rn(ky, ky), __dmul_rn(kx, kx));
    double2 a = make_double2(0.0, 0.0);
    if (k2 <= R2) {
        double2 z = make_double2(0.0, 0.0);
        for (int sy = 0; sy < Sy; ++sy) z = zfma(Ey0[(size_t)i * Sy + sy], T0[(size_t)sy * Nx + j], z);
        a = unit_phase(z);
    }
    A0[t] = a;
}

struct ChiTabArgs {
    const double2* By;    // [Ny][Ly]
    const double2* Bx;    // [Nx][Lx]
    const double2* Ey;    // [Sy][Ny][Sy] at k_y = i - cy + qy[vy]
    const double2* T;     // [Sx][Sy][Nx] x sums at k_x = j - cx + qx[vx]
    const double2* A0;    // [Ny][Nx]
    const double* qy;     // [Sy]
    const double* qx;     // [Sx]
    const uint8_t* used;  // [M]
    double2* chi;         // [S][M]
    unsigned long long* maxbits;
    int Sy, Sx, Ny, Nx, Ly, Lx;
    double cy, cx, R, R2;
};

// chi_v = By^T Y_v Bx for one scan frequency per block, Y_v built kRows detector rows at a time
// in shared memory from A0 and the recovered probe's spectrum at the shifted pixels; folds
// max |chi_v[m]|^2 over the used indices into *maxbits.
template <int ZPT>
__global__ void __launch_bounds__(kThreads) chi_tab_kernel(ChiTabArgs a) {
    extern __shared__ double2 sm[];
    double2* sBx = sm;                            // Nx * Lx
    double2* sY = sBx + (size_t)a.Nx * a.Lx;      // kRows * Nx
    double2* sT = sY + (size_t)kRows * a.Nx;      // kRows * Lx
    __shared__ double red[kThreads];
    const int v = blockIdx.x;
    const int vy = v / a.Sx, vx = v - (v / a.Sx) * a.Sx;
    const double shy = a.qy[vy], shx = a.qx[vx];
    const int M = a.Ly * a.Lx;
    for (int t = threadIdx.x; t < a.Nx * a.Lx; t += blockDim.x) sBx[t] = a.Bx[t];
    double2 z[ZPT];
#pragma unroll
    for (int u = 0; u < ZPT; ++u) z[u] = make_double2(0.0, 0.0);
    for (int i0 = 0; i0 < a.Ny; i0 += kRows) {
        // row blocks entirely outside the unshifted aperture have Y = 0
        const double dlo = (double)i0 - a.cy, dhi = (double)(i0 + kRows - 1) - a.cy;
        const double dmin = (dlo > 0) ? dlo : ((dhi < 0) ? -dhi : 0.0);
        if (dmin > a.R + 1.0) continue;
        __syncthreads();
        for (int t = threadIdx.x; t < kRows * a.Nx; t += blockDim.x) {
            const int r = t / a.Nx, j = t - (t / a.Nx) * a.Nx, i = i0 + r;
            double2 y = make_double2(0.0, 0.0);
            if (i < a.Ny) {
                const double2 p0 = a.A0[(size_t)i * a.Nx + j];
                if (p0.x != 0.0 || p0.y != 0.0) {
                    const double ky2 = __dadd_rn((double)i - a.cy, shy);
                    const double kx2 = __dadd_rn((double)j - a.cx, shx);
                    const double k2s = __dadd_rn(__dmul_rn(ky2, ky2), __dmul_rn(kx2, kx2));
                    if (k2s <= a.R2) {
                        const double2* ey = a.Ey + ((size_t)vy * a.Ny + i) * a.Sy;
                        const double2* tv = a.T + (size_t)vx * a.Sy * a.Nx + j;
                        double2 s = make_double2(0.0, 0.0);
                        for (int sy = 0; sy < a.Sy; ++sy) s = zfma(ey[sy], tv[(size_t)sy * a.Nx], s);
                        const double2 p1 = unit_phase(s);
                        y = make_double2(p0.x * p1.x + p0.y * p1.y, p0.y * p1.x - p0.x * p1.y);
                    }
                }
            }
            sY[t] = y;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < kRows * a.Lx; t += blockDim.x) {
            const int r = t / a.Lx, lx = t - (t / a.Lx) * a.Lx;
            double2 acc = make_double2(0.0, 0.0);
            const double2* yr = sY + (size_t)r * a.Nx;
            for (int j = 0; j < a.Nx; ++j) acc = zfma(yr[j], sBx[(size_t)j * a.Lx + lx], acc);
            sT[t] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < ZPT; ++u) {
            const int o = threadIdx.x + u * kThreads;
            if (o < M) {
                const int ly = o / a.Lx, lx = o - (o / a.Lx) * a.Lx;
                for (int r = 0; r < kRows && i0 + r < a.Ny; ++r)
                    z[u] = zfma(a.By[(size_t)(i0 + r) * a.Ly + ly], sT[r * a.Lx + lx], z[u]);
            }
        }
    }
    double mx = 0.0;
#pragma unroll
    for (int u = 0; u < ZPT; ++u) {
        const int o = threadIdx.x + u * kThreads;
        if (o < M) {
            a.chi[(size_t)v * M + o] = z[u];
            if (a.used[o]) {
                const double a2 = z[u].x * z[u].x + z[u].y * z[u].y;
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
    if (threadIdx.x == 0) atomicMax(a.maxbits, (unsigned long long)__double_as_longlong(red[0]));
}

wdd_status pfail(wdd_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

struct TempBufs {
    std::vector<void*> ptrs;
    ~TempBufs() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t get(T** out, size_t count) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, sizeof(T) * (count ? count : 1));
        if (e != cudaSuccess) return e;
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return cudaSuccess;
    }
};

int blocks_for(int64_t n) {
    return (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 64);
}

}  // namespace
}  // namespace wdd

using namespace wdd;

wdd_status wdd_plan_set_probe(wdd_plan* P, const void* probe) {
    if (!P || !probe) return pfail(WDD_ERR_INVALID_ARG, "plan or probe is NULL");
    if (P->p.scan_rotation_rad != 0.0)
        return pfail(WDD_ERR_UNSUPPORTED,
                     "the probe update takes the probe spectrum one scan axis at a time: "
                     "scan_rotation_rad must be 0");
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, probe) != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    const float2* Pr = nullptr;
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)
        Pr = static_cast<const float2*>(probe);
    else if (attr.type == cudaMemoryTypeHost)
        Pr = static_cast<const float2*>(attr.devicePointer ? attr.devicePointer : probe);
    if (!Pr) return pfail(WDD_ERR_INVALID_ARG, "probe must be in device or pinned host memory");
    const int ZPT = (P->M + kThreads - 1) / kThreads;
    const size_t smem = sizeof(double2) * ((size_t)P->Nx * P->Lx + (size_t)kRows * P->Nx +
                                           (size_t)kRows * P->Lx);
    if (ZPT > 16 || smem > 200 * 1024)
        return pfail(WDD_ERR_UNSUPPORTED, "basis too large for the probe update");

    // the filter is read by every queued snapshot: finish them first
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return pfail(WDD_ERR_CUDA, std::string("synchronise: ") + cudaGetErrorString(e));
    const int Sy = P->Sy, Sx = P->Sx, Ny = P->Ny, Nx = P->Nx;
    TempBufs tmp;
    double2 *Ey = nullptr, *Ey0 = nullptr, *Ex = nullptr, *Ex0 = nullptr, *T = nullptr, *T0 = nullptr,
            *A0 = nullptr, *chi = nullptr;
    uint8_t* d_used = nullptr;
    unsigned long long* d_max = nullptr;
    if (!e) e = tmp.get(&Ey, (size_t)Sy * Ny * Sy);
    if (!e) e = tmp.get(&Ey0, (size_t)Ny * Sy);
    if (!e) e = tmp.get(&Ex, (size_t)Sx * Nx * Sx);
    if (!e) e = tmp.get(&Ex0, (size_t)Nx * Sx);
    if (!e) e = tmp.get(&T, (size_t)Sx * Sy * Nx);
    if (!e) e = tmp.get(&T0, (size_t)Sy * Nx);
    if (!e) e = tmp.get(&A0, (size_t)Ny * Nx);
    if (!e) e = tmp.get(&d_used, (size_t)P->M);
    if (!e) e = tmp.get(&d_max, 1);
    // chi is built in a buffer of its own and replaces the plan's copy only once the update
    // has succeeded, so a refused update leaves WDD_ARRAY_CHI as it was
    if (!e) e = tmp.get(&chi, (size_t)P->S * P->M);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pfail(WDD_ERR_OUT_OF_MEMORY, std::string("probe update buffers: ") + cudaGetErrorString(e));
    }
    std::vector<uint8_t> used(P->M, 0);
    for (int k = 0; k < P->K; ++k) {
        const int m = P->h_ktab[2 * k];
        used[m] = 1;
        if (P->complex_basis) {
            const int ry = m / P->Lx, rx = m % P->Lx;
            used[((P->Ly - ry) % P->Ly) * P->Lx + (P->Lx - rx) % P->Lx] = 1;
        }
    }
    cudaStream_t st = nullptr;
    e = cudaMemcpy(d_used, used.data(), P->M, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(d_max, 0, sizeof(unsigned long long));
    const double dks = P->p.det_px_inv_m * P->p.scan_step_m;
    if (!e) {
        probe_table_kernel<<<blocks_for((int64_t)Sy * Ny * Sy), kThreads, 0, st>>>(Ey, P->d_qy, Sy, Ny, Sy, P->cy, dks);
        probe_table_kernel<<<blocks_for((int64_t)Ny * Sy), kThreads, 0, st>>>(Ey0, nullptr, 1, Ny, Sy, P->cy, dks);
        probe_table_kernel<<<blocks_for((int64_t)Sx * Nx * Sx), kThreads, 0, st>>>(Ex, P->d_qx, Sx, Nx, Sx, P->cx, dks);
        probe_table_kernel<<<blocks_for((int64_t)Nx * Sx), kThreads, 0, st>>>(Ex0, nullptr, 1, Nx, Sx, P->cx, dks);
        probe_xsum_kernel<<<blocks_for((int64_t)Sx * Sy * Nx), kThreads, 0, st>>>(Pr, Ex, T, Sx, Sy, Sx, Nx);
        probe_xsum_kernel<<<blocks_for((int64_t)Sy * Nx), kThreads, 0, st>>>(Pr, Ex0, T0, 1, Sy, Sx, Nx);
        probe_a0_kernel<<<(Ny * Nx + kThreads - 1) / kThreads, kThreads, 0, st>>>(
            Ey0, T0, A0, Sy, Ny, Nx, P->cy, P->cx, P->R * P->R);
        e = cudaGetLastError();
    }
    if (!e) {
        ChiTabArgs a{P->d_By, P->d_Bx, Ey, T, A0, P->d_qy, P->d_qx, d_used, chi, d_max,
                     Sy, Sx, Ny, Nx, P->Ly, P->Lx, P->cy, P->cx, P->R, P->R * P->R};
#define WDD_CHI_TAB(Z)                                                                     \
        do {                                                                               \
            e = allow_max_dynamic_smem(reinterpret_cast<const void*>(chi_tab_kernel<Z>));  \
            if (!e) chi_tab_kernel<Z><<<P->S, kThreads, smem, st>>>(a);                    \
        } while (0)
        if (ZPT <= 1) WDD_CHI_TAB(1);
        else if (ZPT <= 2) WDD_CHI_TAB(2);
        else if (ZPT <= 4) WDD_CHI_TAB(4);
        else if (ZPT <= 8) WDD_CHI_TAB(8);
        else WDD_CHI_TAB(16);
#undef WDD_CHI_TAB
        if (!e) e = cudaGetLastError();
    }
    unsigned long long maxbits = 0;
    if (!e) e = cudaMemcpy(&maxbits, d_max, sizeof maxbits, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return pfail(WDD_ERR_CUDA, std::string("probe update: ") + cudaGetErrorString(e));
    double maxchi;
    std::memcpy(&maxchi, &maxbits, 8);
    const double eps_eff = P->p.eps_absolute ? P->p.epsilon : P->p.epsilon * maxchi;
    if (!(eps_eff > 0) && P->p.epsilon > 0)
        return pfail(WDD_ERR_INVALID_ARG, "recovered probe autocorrelation is zero everywhere");
    // Wiener weights from the new chi (the plan's own kernel reads P->d_chi and P->eps_eff)
    double2* keep_chi = P->d_chi;
    const double keep_eps = P->eps_eff;
    P->d_chi = chi;
    P->eps_eff = eps_eff;
    e = launch_weights(P, st);
    if (!e && keep_chi)
        e = cudaMemcpyAsync(keep_chi, chi, sizeof(double2) * (size_t)P->S * P->M,
                            cudaMemcpyDeviceToDevice, st);
    if (!e) e = cudaDeviceSynchronize();
    P->d_chi = keep_chi;
    if (e != cudaSuccess) {
        P->eps_eff = keep_eps;
        return pfail(WDD_ERR_CUDA, std::string("probe update weights: ") + cudaGetErrorString(e));
    }
    return WDD_OK;
}
