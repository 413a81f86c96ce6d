// Frame ingest and projection onto the reduced basis (Sect. 5, operator H of Eq. 12; Algorithm 2, step 1):
//   c_b[k] = component_k( sum_{i,j} By[i, ly_k] I_b[i, j] Bx[j, lx_k] )
// computed separably: U = By^T I (contraction over detector rows), then Z = U Bx.
//
// Each frame is handled by a thread-block cluster of CS CTAs (CS = 1..8, chosen so that a launch
// covers the SMs); CTA q of the cluster reduces a contiguous slice of detector rows.  The slice
// streams through shared memory in row blocks of up to 32 KB, double buffered.  Device-resident
// frames arrive by 1-D TMA bulk copies (cp.async.bulk) issued ahead by one thread; frames in
// pinned host memory are read straight over the host link with coalesced 16-byte loads.  Frames stay in their stored type (uint16, float32, float64) in
// shared memory and are converted to FP32 in registers.
//
// First contraction: a work item is (detector column j, group of 8 basis rows, row part p); it
// accumulates over its rows with the basis values read as broadcasts; the row parts are then
// added in part order.  Second contraction: each coefficient's dot product over the columns is
// split across threads and added in a fixed order; the CTAs of a cluster then add their partial coefficients into the leader CTA's shared
// memory (distributed shared memory) and the leader sums them in rank order.  No step depends
// on scheduling, so results are bit-reproducible.
//
// Consecutive projection launches overlap through programmatic dependent launch: a launch starts
// its loads and contractions while the previous kernel in the stream finishes, and waits for it
// (griddepcontrol.wait) only before writing its outputs.
//
// The scan indices of the launch arrive as a by-value parameter block and are stored next to the
// staged coefficients for the phase accumulation, so a push needs no host-to-device copy.  For the
// split-precision path the kernel also keeps a running maximum of |c| per coefficient (float bits
// compared as unsigned integers), from which the accumulation picks its scales.

#include <cooperative_groups.h>

#include "wdd_device.cuh"
#include "wdd_internal.h"

namespace cg = cooperative_groups;

namespace wdd {

namespace {

constexpr int kGroup = 8;

template <typename FT>
__device__ __forceinline__ float to_f(FT v) { return (float)v; }

// Copies `count` frame elements from global (device or host-mapped) memory into shared memory,
// with 16-byte vector loads when both ends allow it.
template <typename FT>
__device__ __forceinline__ void copy_rows(const FT* __restrict__ src, FT* dst, int count) {
    constexpr int V = 16 / sizeof(FT);
    const bool aligned = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && (count % V == 0);
    if (aligned) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        const int nv = count / V;
        const int bd = blockDim.x;
        int t = threadIdx.x;
        // four independent loads in flight per thread before the first store
        for (; t + 3 * bd < nv; t += 4 * bd) {
            uint4 a0 = __ldg(s4 + t), a1 = __ldg(s4 + t + bd);
            uint4 a2 = __ldg(s4 + t + 2 * bd), a3 = __ldg(s4 + t + 3 * bd);
            d4[t] = a0;
            d4[t + bd] = a1;
            d4[t + 2 * bd] = a2;
            d4[t + 3 * bd] = a3;
        }
        for (; t < nv; t += bd) d4[t] = __ldg(s4 + t);
    } else {
        for (int t = threadIdx.x; t < count; t += blockDim.x) dst[t] = src[t];
    }
}

// COLS consecutive frame values from shared memory as FP32 (vector load when COLS == 4).
template <typename FT, int COLS>
__device__ __forceinline__ void load_cols(const FT* p, float* x) {
    if constexpr (COLS == 4 && sizeof(FT) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else if constexpr (COLS == 4 && sizeof(FT) == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        x[0] = (float)(v.x & 0xFFFFu); x[1] = (float)(v.x >> 16);
        x[2] = (float)(v.y & 0xFFFFu); x[3] = (float)(v.y >> 16);
    } else {
#pragma unroll
        for (int c = 0; c < COLS; ++c) x[c] = to_f(p[c]);
    }
}

template <typename FT, bool CPLX, int COLS>
__global__ void __launch_bounds__(kThreads)
project_kernel(const FT* __restrict__ frames, const ProjGeom g, const float2* __restrict__ By,
               const float2* __restrict__ Bx, const int2* __restrict__ ktab,
               float* __restrict__ c_out, const IndexBlock ids, int32_t* __restrict__ idx_out,
               unsigned* __restrict__ colmax, unsigned* __restrict__ status, uint64_t wait_ns) {
    extern __shared__ __align__(128) uint8_t sm[];
    constexpr int CW = CPLX ? 2 : 1;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int b = blockIdx.x / g.CS;                 // frame of this cluster
    const int r0 = rank * g.rows_cta;                // first detector row of this CTA
    const int nrows = max(0, min(g.rows_cta, g.Ny - r0));
    const int LyW = g.Ly * CW;            // real rows of U (re/im interleaved for CPLX)
    const int LyWp = g.G * kGroup;        // padded to whole groups
    uint8_t* raw = sm;                    // [2][buf_bytes]
    float* sBy = reinterpret_cast<float*>(sm + 2 * g.buf_bytes);      // [rows_cta][LyWp]
    float* sBx = sBy + (size_t)g.rows_cta * LyWp;                     // [Nx][Lx*CW]
    float* Up = sBx + (size_t)g.Nx * g.Lx * CW;                       // [P][LyWp][Nx]
    float* red = Up + (size_t)g.P * LyWp * g.Nx;                      // [SP][K]  (second contraction)
    float* part = reinterpret_cast<float*>(                            // [CS][K]  (leader only)
        (reinterpret_cast<uintptr_t>(red + (size_t)g.SP * g.K) + 15) & ~uintptr_t(15));
    uint64_t* bar = reinterpret_cast<uint64_t*>(
        reinterpret_cast<uint8_t*>(part) + ((4 * (size_t)g.CS * g.K + 15) & ~size_t(15)));
    __shared__ int s_fail;

    // let the next launch in the stream start its loads while this one runs
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const FT* src = frames + (size_t)b * g.Ny * g.Nx + (size_t)r0 * g.Nx;
    const int rowElems = g.RB * g.Nx;
    const int nblk = (nrows + g.RB - 1) / g.RB;
    if (threadIdx.x == 0) {
        s_fail = 0;
        if (g.use_tma) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            for (int q = 0; q < 2 && q < nblk; ++q) {
                const int rows = min(g.RB, nrows - q * g.RB);
                const unsigned bytes = (unsigned)(rows * g.Nx * sizeof(FT));
                mbar_arrive_tx(&bar[q], bytes);
                tma_load_1d(raw + q * g.buf_bytes, src + (size_t)q * rowElems, bytes, &bar[q]);
            }
        }
    }
    // bases into shared memory while the first row blocks are in flight
    for (int t = threadIdx.x; t < nrows * LyWp; t += blockDim.x) {
        const int i = t / LyWp, w = t % LyWp;
        float v = 0.f;
        if (w < LyW) {
            const float2 e = By[(size_t)(r0 + i) * g.Ly + w / CW];
            v = (CPLX && (w & 1)) ? e.y : e.x;
        }
        sBy[t] = v;
    }
    for (int t = threadIdx.x; t < g.Nx * g.Lx; t += blockDim.x) {
        const float2 e = Bx[t];
        if (CPLX) {
            sBx[2 * t] = e.x;
            sBx[2 * t + 1] = e.y;
        } else {
            sBx[t] = e.x;
        }
    }
    const int ncq = g.Nx / COLS;                 // column quads (or single columns)
    const int items = ncq * g.G * g.P;
    for (int t = threadIdx.x; t < g.P * LyWp * g.Nx; t += blockDim.x) Up[t] = 0.f;   // U = 0
    __syncthreads();

    for (int blk = 0; blk < nblk; ++blk) {
        const int buf = blk & 1;
        const int rows = min(g.RB, nrows - blk * g.RB);
        FT* rb = reinterpret_cast<FT*>(raw + buf * g.buf_bytes);
        if (g.use_tma) {
            if (threadIdx.x == 0 && !mbar_wait(&bar[buf], (blk >> 1) & 1, wait_ns)) s_fail = 1;
        } else {
            copy_rows<FT>(src + (size_t)blk * rowElems, rb, rows * g.Nx);
        }
        __syncthreads();
        if (s_fail) break;
        for (int w = threadIdx.x; w < items; w += blockDim.x) {
            const int jq = w % ncq;
            const int rest = w / ncq;
            const int gi = rest % g.G;
            const int p = rest / g.G;
            const int j0 = jq * COLS;
            float* u = Up + ((size_t)p * LyWp + gi * kGroup) * g.Nx + j0;
            float acc[kGroup][COLS];
#pragma unroll
            for (int q = 0; q < kGroup; ++q)
#pragma unroll
                for (int c = 0; c < COLS; ++c) acc[q][c] = u[(size_t)q * g.Nx + c];
            const float* byb = sBy + (size_t)(blk * g.RB) * LyWp + gi * kGroup;
            for (int r = p; r < rows; r += g.P) {
                float x[COLS];
                load_cols<FT, COLS>(rb + r * g.Nx + j0, x);
                const float4 b0 = *reinterpret_cast<const float4*>(byb + (size_t)r * LyWp);
                const float4 b1 = *reinterpret_cast<const float4*>(byb + (size_t)r * LyWp + 4);
                const float bv[kGroup] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int q = 0; q < kGroup; ++q)
#pragma unroll
                    for (int c = 0; c < COLS; ++c) acc[q][c] = fmaf(x[c], bv[q], acc[q][c]);
            }
#pragma unroll
            for (int q = 0; q < kGroup; ++q)
#pragma unroll
                for (int c = 0; c < COLS; ++c) u[(size_t)q * g.Nx + c] = acc[q][c];
        }
        __syncthreads();   // row block consumed: its buffer can be refilled
        if (g.use_tma && threadIdx.x == 0 && blk + 2 < nblk) {
            const int rows2 = min(g.RB, nrows - (blk + 2) * g.RB);
            const unsigned bytes = (unsigned)(rows2 * g.Nx * sizeof(FT));
            mbar_arrive_tx(&bar[buf], bytes);
            tma_load_1d(raw + buf * g.buf_bytes, src + (size_t)(blk + 2) * rowElems, bytes,
                        &bar[buf]);
        }
    }
    const bool failed = s_fail != 0;
    if (failed && threadIdx.x == 0) atomicExch(status, 5u);

    // fold the row parts: U = sum_p U_p, added in part order
    if (!failed && g.P > 1) {
        const size_t plane = (size_t)LyWp * g.Nx;
        for (size_t t = threadIdx.x; t < plane; t += blockDim.x) {
            float s = Up[t];
            for (int p = 1; p < g.P; ++p) s += Up[p * plane + t];
            Up[t] = s;
        }
        __syncthreads();
    }
    // second contraction: Z[ly][lx] = sum_j U[ly][j] Bx[j][lx], the j range of every
    // coefficient split into SP interleaved slices summed in slice order
    if (!failed) {
        const int slots = g.K * g.SP;
        for (int t = threadIdx.x; t < slots; t += blockDim.x) {
            const int k = t % g.K, sl = t / g.K;
            const int2 e = ktab[k];
            const int ly = e.x / g.Lx, lx = e.x % g.Lx;
            float acc = 0.f;
            {
                if (CPLX) {
                    const float* ur = Up + (size_t)(2 * ly) * g.Nx;
                    const float* ui = ur + g.Nx;
                    for (int j = sl; j < g.Nx; j += g.SP) {
                        const float bxr = sBx[2 * (j * g.Lx + lx)], bxi = sBx[2 * (j * g.Lx + lx) + 1];
                        acc = (e.y == 0) ? fmaf(ur[j], bxr, fmaf(-ui[j], bxi, acc))
                                         : fmaf(ur[j], bxi, fmaf(ui[j], bxr, acc));
                    }
                } else {
                    const float* ur = Up + (size_t)ly * g.Nx;
                    for (int j = sl; j < g.Nx; j += g.SP) acc = fmaf(ur[j], sBx[j * g.Lx + lx], acc);
                }
            }
            red[(size_t)sl * g.K + k] = acc;
        }
    }
    __syncthreads();
    // Outputs may alias staging slots that the previous kernel in the stream still reads (the
    // accumulation of the last flush): wait for it to complete before writing anything.  This
    // also keeps completion in stream order.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (rank == 0 && threadIdx.x == 0) idx_out[b] = ids.s[b];   // scan index for the accumulation
    // partial coefficients of this CTA -> the leader's shared memory
    float* lead = cluster.map_shared_rank(part, 0);
    for (int k = threadIdx.x; k < g.K; k += blockDim.x) {
        float acc = 0.f;
        if (!failed)
            for (int sl = 0; sl < g.SP; ++sl) acc += red[(size_t)sl * g.K + k];
        lead[(size_t)rank * g.K + k] = acc;
    }
    cluster.sync();
    if (rank == 0 && !failed) {
        for (int k = threadIdx.x; k < g.K; k += blockDim.x) {
            float acc = 0.f;
            for (int q = 0; q < g.CS; ++q) acc += part[(size_t)q * g.K + k];
            c_out[(size_t)b * g.K + k] = acc;
            if (colmax) atomicMax(colmax + k, __float_as_uint(fabsf(acc)));
        }
    }
}

template <typename FT>
cudaError_t launch_typed(const wdd_plan* P, const FT* frames, int n, bool device_src, bool overlap,
                         const IndexBlock& ids, float* c_out, int32_t* idx_out, cudaStream_t st) {
    ProjGeom g = P->proj;
    g.use_tma = (device_src && ((reinterpret_cast<uintptr_t>(frames) & 15u) == 0) &&
                 ((g.Nx * sizeof(FT)) % 16 == 0)) ? 1 : 0;
    proj_set_frame_bytes(g, (int)sizeof(FT));
    const size_t smem = proj_smem_bytes(g);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n * g.CS), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)g.CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 2 : 1;
    const float2* by = P->d_By32;
    const float2* bx = P->d_Bx32;
    const int2* kt = P->d_ktab;
    const bool quad = (g.Nx % 4) == 0;
    if (P->complex_basis)
        return quad ? cudaLaunchKernelEx(&cfg, project_kernel<FT, true, 4>, frames, g, by, bx, kt,
                                         c_out, ids, idx_out, P->d_colmax, P->d_status, kDeviceWaitNs)
                    : cudaLaunchKernelEx(&cfg, project_kernel<FT, true, 1>, frames, g, by, bx, kt,
                                         c_out, ids, idx_out, P->d_colmax, P->d_status, kDeviceWaitNs);
    return quad ? cudaLaunchKernelEx(&cfg, project_kernel<FT, false, 4>, frames, g, by, bx, kt,
                                     c_out, ids, idx_out, P->d_colmax, P->d_status, kDeviceWaitNs)
                : cudaLaunchKernelEx(&cfg, project_kernel<FT, false, 1>, frames, g, by, bx, kt,
                                     c_out, ids, idx_out, P->d_colmax, P->d_status, kDeviceWaitNs);
}

template <typename FT>
cudaError_t prepare_typed() {
    const void* k[4] = {reinterpret_cast<const void*>(project_kernel<FT, true, 4>),
                        reinterpret_cast<const void*>(project_kernel<FT, true, 1>),
                        reinterpret_cast<const void*>(project_kernel<FT, false, 4>),
                        reinterpret_cast<const void*>(project_kernel<FT, false, 1>)};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = allow_max_dynamic_smem(k[i]);
    return e;
}

}  // namespace

void proj_set_frame_bytes(ProjGeom& g, int elem_bytes) {
    int rb = kRowBlockBytes / (g.Nx * elem_bytes);
    if (rb < 1) rb = 1;
    g.RB = rb < g.rows_cta ? rb : g.rows_cta;
    g.buf_bytes = (g.RB * g.Nx * elem_bytes + 127) & ~127;
}

size_t proj_smem_bytes(const ProjGeom& g) {
    const size_t floats = (size_t)g.rows_cta * g.G * kGroup + (size_t)g.Nx * g.Lx * g.CW +
                          (size_t)g.P * g.G * kGroup * g.Nx + (size_t)g.SP * g.K;
    const size_t part = ((size_t)g.CS * g.K * 4 + 15) & ~size_t(15);
    return ((2 * (size_t)g.buf_bytes + 4 * floats + 15) & ~size_t(15)) + part + 16;
}

// Cluster size, row slices and work split for a plan's projection.  `frames_per_launch` is the
// typical launch size; the cluster is widened until a launch has about two CTAs per SM.
ProjGeom make_proj_geom(int Ny, int Nx, int Ly, int Lx, int K, int complex_basis,
                        int frames_per_launch, int cluster) {
    ProjGeom g{};
    g.Ny = Ny;
    g.Nx = Nx;
    g.Ly = Ly;
    g.Lx = Lx;
    g.K = K;
    g.CW = complex_basis ? 2 : 1;
    g.G = (Ly * g.CW + kGroup - 1) / kGroup;
    int cs = 1;
    if (cluster > 0) {
        while (cs < cluster && cs < 8 && (size_t)(2 * cs) * K * 4 <= 32768 && Ny >= 2 * cs) cs *= 2;
    } else {
        // consecutive launches overlap (programmatic dependent launch), so a frame is split
        // over a cluster only when a launch alone would leave most SMs idle
        while (cs < 8 && frames_per_launch * cs < 64 && Ny / (2 * cs) >= 8 &&
               (size_t)(2 * cs) * K * 4 <= 32768)
            cs *= 2;
    }
    g.CS = cs;
    g.rows_cta = (Ny + cs - 1) / cs;
    const int per = (Nx % 4 == 0 ? Nx / 4 : Nx) * g.G;
    g.P = per >= kThreads ? 1 : kThreads / per;
    if (g.P > g.rows_cta) g.P = g.rows_cta;
    g.SP = K >= kThreads ? 1 : kThreads / K;
    if (g.SP > Nx) g.SP = Nx;
    proj_set_frame_bytes(g, 8);   // largest frame type: the shared-memory bound of the plan
    return g;
}

cudaError_t prepare_project_kernels() {
    cudaError_t e = prepare_typed<uint16_t>();
    if (e == cudaSuccess) e = prepare_typed<float>();
    if (e == cudaSuccess) e = prepare_typed<double>();
    return e;
}

cudaError_t launch_project(const wdd_plan* P, const void* frames, int dtype, int n,
                           bool device_src, bool overlap, const IndexBlock& ids, float* c_out,
                           int32_t* idx_out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > kLaunchFrames) return cudaErrorInvalidValue;
    switch (dtype) {
        case WDD_FRAME_U16:
            return launch_typed(P, static_cast<const uint16_t*>(frames), n, device_src, overlap, ids,
                                c_out, idx_out, st);
        case WDD_FRAME_F32:
            return launch_typed(P, static_cast<const float*>(frames), n, device_src, overlap, ids,
                                c_out, idx_out, st);
        case WDD_FRAME_F64:
            return launch_typed(P, static_cast<const double*>(frames), n, device_src, overlap, ids,
                                c_out, idx_out, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace wdd
