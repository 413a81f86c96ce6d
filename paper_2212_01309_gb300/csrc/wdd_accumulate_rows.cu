// Phase accumulation factorised by scan rows (accumulation mode SEPARABLE; not in the paper).
//
// The phase factor of Eq. 14 separates, exp(-2 pi i (v_y s_y / S_y + v_x s_x / S_x)) =
// Ey[v_y, s_y] Ex[v_x, s_x], so the frames of one scan row s_y contribute
//   H[(v_y, v_x), k] += Ey[v_y, s_y] G_{s_y}[v_x, k],   G_{s_y}[v_x, k] = sum_{s_x} Ex[v_x, s_x] c_s[k]
// (a 1-D DFT along the row, then one rank-R complex update of H for the R rows touched).  For
// frames in raster order this needs 4 S_x K flops per frame plus 8 S K per touched row, instead
// of the 4 S K per frame of the direct form; the result is the same H up to rounding.  All three
// steps run in FP32 on the SIMT cores:
//   rows_plan_kernel   finds the rows the staged frames touch, gives each a slot (in row order)
//                      and records each slot's first and last staged frame;
//   rowdft_kernel      G[slot][v_x][k] for every slot, frames taken in staging order;
//   outer_kernel       H[v_y][(v_x, k)] += sum over slots of Ey[v_y, row(slot)] G[slot][(v_x, k)],
//                      slots in row order, one read-modify-write of H.
// Every sum is taken in a fixed order, so results are bit-reproducible.  Phase factors come
// from the plan's FP32 table exp(-2 pi i m / lcm) with the exact integer index
// m = (v s mod S) (lcm / S) for each axis.

#include <climits>

#include "wdd_internal.h"

namespace wdd {

namespace {

constexpr int kPlanThreads = 1024;
constexpr int kT = 64;     // tile edge of rowdft / outer kernels
constexpr int kB = 16;     // frames (rowdft) or slots (outer) per shared-memory chunk

// Block-wide exclusive scan of one int per thread (1024 threads); returns the prefix, and the
// total in *total.
__device__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;   // inclusive
    }
    __syncthreads();
    const int before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    *total = warp_sums[31];
    return before;
}

// One CTA of 1024 threads.  Shared memory: mark[Sy] (row -> slot), first[Rmax], last[Rmax].
__global__ void __launch_bounds__(kPlanThreads)
rows_plan_kernel(const int32_t* __restrict__ idx, int n, int Sx, int Sy, int Rmax,
                 int32_t* __restrict__ slotrow, int32_t* __restrict__ slot_first,
                 int32_t* __restrict__ slot_last, int32_t* __restrict__ frame_slot,
                 int32_t* __restrict__ R_out) {
    extern __shared__ int sm_plan[];
    int* mark = sm_plan;            // Sy
    int* sfirst = mark + Sy;        // Rmax
    int* slast = sfirst + Rmax;     // Rmax
    __shared__ int warp_sums[32];
    __shared__ int s_total;
    for (int t = threadIdx.x; t < Sy; t += blockDim.x) mark[t] = 0;
    for (int t = threadIdx.x; t < Rmax; t += blockDim.x) {
        sfirst[t] = INT_MAX;
        slast[t] = -1;
    }
    __syncthreads();
    for (int f = threadIdx.x; f < n; f += blockDim.x) mark[idx[f] / Sx] = 1;
    __syncthreads();
    // slots in row order: exclusive scan of the marks, each thread owning a run of rows
    const int per = (Sy + kPlanThreads - 1) / kPlanThreads;
    const int r0 = threadIdx.x * per;
    int cnt = 0;
    for (int r = r0; r < r0 + per && r < Sy; ++r) cnt += mark[r];
    int total = 0;
    int pos = block_exclusive_scan(cnt, warp_sums, &total);
    for (int r = r0; r < r0 + per && r < Sy; ++r) {
        if (mark[r]) {
            slotrow[pos] = r;
            mark[r] = pos++;
        } else {
            mark[r] = -1;
        }
    }
    if (threadIdx.x == 0) s_total = total;
    __syncthreads();
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
        const int s = mark[idx[f] / Sx];
        frame_slot[f] = s;
        atomicMin(&sfirst[s], f);
        atomicMax(&slast[s], f);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < s_total; t += blockDim.x) {
        slot_first[t] = sfirst[t];
        slot_last[t] = slast[t];
    }
    if (threadIdx.x == 0) *R_out = s_total;
}

// G[slot][v_x][k] = sum over the slot's staged frames (in staging order) of Ex[v_x, s_x] c[k].
// Grid (Rmax, tiles of 64 v_x, tiles of 64 k); each thread keeps a 4 x 4 block of complex sums.
__global__ void __launch_bounds__(kThreads)
rowdft_kernel(const float* __restrict__ c, const int32_t* __restrict__ idx,
              const int32_t* __restrict__ frame_slot, const int32_t* __restrict__ slot_first,
              const int32_t* __restrict__ slot_last, const int32_t* __restrict__ R_ptr, int Sx,
              int K, int mx, const float2* __restrict__ tw, float2* __restrict__ G) {
    const int slot = blockIdx.x;
    if (slot >= *R_ptr) return;
    __shared__ __align__(16) float2 sE[kB][kT];
    __shared__ __align__(16) float sC[kB][kT];
    const int x0 = blockIdx.y * kT, k0 = blockIdx.z * kT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int first = slot_first[slot], last = slot_last[slot];
    float ar[4][4], ai[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0.f;
    for (int f0 = first; f0 <= last; f0 += kB) {
        for (int t = threadIdx.x; t < kB * kT; t += blockDim.x) {
            const int bb = t / kT, q = t % kT;
            const int f = f0 + bb;
            const bool in = f <= last && frame_slot[f] == slot;
            const int k = k0 + q, vx = x0 + q;
            sC[bb][q] = (in && k < K) ? c[(size_t)f * K + k] : 0.f;
            float2 e = make_float2(0.f, 0.f);
            if (in && vx < Sx) {
                const int sx = idx[f] % Sx;
                e = tw[(size_t)((vx * sx) % Sx) * mx];
            }
            sE[bb][q] = e;
        }
        __syncthreads();
#pragma unroll 4
        for (int bb = 0; bb < kB; ++bb) {
            const float4 e01 = *reinterpret_cast<const float4*>(&sE[bb][ty * 4]);
            const float4 e23 = *reinterpret_cast<const float4*>(&sE[bb][ty * 4 + 2]);
            const float4 cc = *reinterpret_cast<const float4*>(&sC[bb][tx * 4]);
            const float er[4] = {e01.x, e01.z, e23.x, e23.z};
            const float ei[4] = {e01.y, e01.w, e23.y, e23.w};
            const float cv[4] = {cc.x, cc.y, cc.z, cc.w};
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
        const int vx = x0 + ty * 4 + i;
        if (vx >= Sx) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + tx * 4 + j;
            if (k < K) G[((size_t)slot * Sx + vx) * K + k] = make_float2(ar[i][j], ai[i][j]);
        }
    }
}

// H[v_y][q] += sum_{slot < R} Ey[v_y, row(slot)] G[slot][q], q = v_x K + k (so that H row
// v = v_y S_x + v_x is H[v_y][q] with stride S_x K).  Grid (tiles of 64 q, tiles of 64 v_y).
__global__ void __launch_bounds__(kThreads)
outer_kernel(const float2* __restrict__ G, const int32_t* __restrict__ slotrow,
             const int32_t* __restrict__ R_ptr, int Sy, int Q, int my,
             const float2* __restrict__ tw, float2* __restrict__ H) {
    __shared__ __align__(16) float2 sY[kB][kT];
    __shared__ __align__(16) float2 sG[kB][kT];
    const int R = *R_ptr;
    const int q0 = blockIdx.x * kT;
    const int y0 = blockIdx.y * kT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float ar[4][4], ai[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0.f;
    for (int s0 = 0; s0 < R; s0 += kB) {
        for (int t = threadIdx.x; t < kB * kT; t += blockDim.x) {
            const int ss = t / kT, p = t % kT;
            const int s = s0 + ss;
            float2 ey = make_float2(0.f, 0.f), g = make_float2(0.f, 0.f);
            if (s < R) {
                const int vy = y0 + p;
                if (vy < Sy) ey = tw[(size_t)((vy * slotrow[s]) % Sy) * my];
                const int q = q0 + p;
                if (q < Q) g = G[(size_t)s * Q + q];
            }
            sY[ss][p] = ey;
            sG[ss][p] = g;
        }
        __syncthreads();
#pragma unroll 4
        for (int ss = 0; ss < kB; ++ss) {
            const float4 y01 = *reinterpret_cast<const float4*>(&sY[ss][ty * 4]);
            const float4 y23 = *reinterpret_cast<const float4*>(&sY[ss][ty * 4 + 2]);
            const float4 g01 = *reinterpret_cast<const float4*>(&sG[ss][tx * 4]);
            const float4 g23 = *reinterpret_cast<const float4*>(&sG[ss][tx * 4 + 2]);
            const float yr[4] = {y01.x, y01.z, y23.x, y23.z};
            const float yi[4] = {y01.y, y01.w, y23.y, y23.w};
            const float gr[4] = {g01.x, g01.z, g23.x, g23.z};
            const float gi[4] = {g01.y, g01.w, g23.y, g23.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    ar[i][j] = fmaf(yr[i], gr[j], fmaf(-yi[i], gi[j], ar[i][j]));
                    ai[i][j] = fmaf(yr[i], gi[j], fmaf(yi[i], gr[j], ai[i][j]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int vy = y0 + ty * 4 + i;
        if (vy >= Sy) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = q0 + tx * 4 + j;
            if (q < Q) {
                float2* h = H + (size_t)vy * Q + q;
                float2 hv = *h;
                hv.x += ar[i][j];
                hv.y += ai[i][j];
                *h = hv;
            }
        }
    }
}

size_t plan_smem_bytes(int Sy, int Rmax) { return 4 * ((size_t)Sy + 2 * (size_t)Rmax); }

}  // namespace

int rows_slots(int Sy, int depth_pad) { return Sy < depth_pad ? Sy : depth_pad; }

cudaError_t prepare_rows_kernels() {
    return allow_max_dynamic_smem(reinterpret_cast<const void*>(rows_plan_kernel));
}

cudaError_t launch_accumulate_rows(const wdd_plan* P, const float* c, const int32_t* idx, int n,
                                   cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int Rmax = rows_slots(P->Sy, n);
    rows_plan_kernel<<<1, kPlanThreads, plan_smem_bytes(P->Sy, Rmax), st>>>(
        idx, n, P->Sx, P->Sy, Rmax, P->d_slotrow, P->d_slotfirst, P->d_slotlast, P->d_frameslot,
        P->d_nslots);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int mx = P->lcm / P->Sx, my = P->lcm / P->Sy;
    dim3 g1(Rmax, (P->Sx + kT - 1) / kT, (P->K + kT - 1) / kT);
    rowdft_kernel<<<g1, kThreads, 0, st>>>(c, idx, P->d_frameslot, P->d_slotfirst, P->d_slotlast,
                                           P->d_nslots, P->Sx, P->K, mx, P->d_tw, P->d_G);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int Q = P->Sx * P->K;
    dim3 g2((Q + kT - 1) / kT, (P->Sy + kT - 1) / kT);
    outer_kernel<<<g2, kThreads, 0, st>>>(P->d_G, P->d_slotrow, P->d_nslots, P->Sy, Q, my,
                                          P->d_tw, P->d_H);
    return cudaGetLastError();
}

}  // namespace wdd
