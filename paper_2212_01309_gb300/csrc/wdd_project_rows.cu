// Frame ingest and projection in FP32 on the SIMT cores, streamed by detector rows:
//   c_b[k] = sum_{i,j} By[i, ly_k] I_b[i, j] Bx[j, lx_k]      (Sect. 5, operator H of Eq. 12)
// for real (Hermite-Gauss) bases with at most 16 functions along the detector rows.
//
// The projection reads every frame byte once and does 2 (N_y N_x L_y + L_y N_x L_x) flops per
// frame: about 2 L_y flops per pixel, far below the tensor cores' ridge, so its bound is the
// frame read (HBM, or the host link for frames in pinned host memory).  This kernel is written
// for that bound: one CTA of 128 threads per frame; thread t owns four adjacent detector columns
// 4 (t % G) .. + 3 (G = N_x / 4 column groups) and every (128 / G)-th row, reads its four values
// of a row with one 8- or 16-byte load (a warp reads whole contiguous row segments; two batches
// of eight rows in flight per thread), and accumulates
//   U[ly][col] = sum_i By[i, ly] I[i, col]
// in registers, By[i, .] being a shared-memory broadcast (every lane of a warp reads the same row
// when G >= 32).  The row phases' partial sums are then added in a fixed order in shared memory
// and contracted with Bx for the selected coefficients:
//   c_k = sum_col U[ly_k][col] Bx[col, lx_k].
// All arithmetic is FP32 with FP32 operands (the bases rounded once from FP64), so the
// coefficients carry FP32 rounding only.  Frames in pinned host memory are read by the same loads
// over the host link.
//
// Launch ordering is that of the other projection kernels: the kernel lets the next launch start
// at once (it holds no tensor memory) and writes its outputs after griddepcontrol.wait.

#include <type_traits>

#include "wdd_device.cuh"
#include "wdd_internal.h"

namespace wdd {

namespace {

constexpr int kRowThreads = 128;
constexpr int kRowsLdMax = 512;    // widest detector (G = N_x / 4 <= 128 column groups)

struct PrArgs {
    int Ny, Nx, Ly, Lx, K;
    const float* By;          // [Ny][Ly] real parts of the row basis (FP32)
    const float* Bx;          // [Nx][Lx] real parts of the column basis (FP32)
    const int2* ktab;         // [K] (ly * Lx + lx, 0)
    float* c_out;             // [n][K]
    int32_t* idx_out;         // [n]
    unsigned* colmax;         // [K] running max |c| (float bits) or NULL
};

// Shared-memory layout in floats: By padded to LYP columns, Bx, the row phases' partial sums
// (R * LYP * Nx = 512 LYP floats), and the coefficient slices.
__host__ __device__ inline size_t pr_by_off() { return 0; }
__host__ __device__ inline size_t pr_bx_off(int Ny, int LYP) { return (size_t)Ny * LYP; }
__host__ __device__ inline size_t pr_u_off(int Ny, int Nx, int Lx, int LYP) {
    return ((size_t)Ny * LYP + (size_t)Nx * Lx + 3) / 4 * 4;
}
__host__ __device__ inline size_t pr_red_off(int Ny, int Nx, int Lx, int LYP) {
    return pr_u_off(Ny, Nx, Lx, LYP) + (size_t)4 * kRowThreads * LYP;
}
__host__ __device__ inline size_t pr_floats(int Ny, int Nx, int Lx, int K, int LYP) {
    const int red = K >= kRowThreads ? K : kRowThreads;
    return pr_red_off(Ny, Nx, Lx, LYP) + (size_t)red;
}

__host__ __device__ inline int pr_lyp(int Ly) { return (Ly + 3) / 4 * 4; }

// Four consecutive frame values as FP32 (16-byte aligned for float, 8-byte for uint16).
__device__ __forceinline__ void load4(const float* p, float (&x)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void load4(const uint16_t* p, float (&x)[4]) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    x[0] = (float)(v.x & 0xFFFFu); x[1] = (float)(v.x >> 16);
    x[2] = (float)(v.y & 0xFFFFu); x[3] = (float)(v.y >> 16);
}

// Rows per batch: two batches (2 kNB rows x 16 bytes) are in flight per thread, enough bytes in
// flight per SM to cover the memory latency at the HBM rate.
constexpr int kNB = 8;

// Loads rows r0, r0 + R, ... (kNB of them, those below Ny) of this thread's four columns.
template <typename FT>
__device__ __forceinline__ void load_batch(const FT* col, int Nx, int Ny, int r0, int R,
                                           float (&x)[kNB][4]) {
#pragma unroll
    for (int u = 0; u < kNB; ++u)
        if (r0 + u * R < Ny) load4(col + (size_t)(r0 + u * R) * Nx, x[u]);
}

// acc[ly][v] += By[row][ly] x[u][v] for the batch's rows below Ny (By a shared-memory broadcast).
template <int LYP>
__device__ __forceinline__ void use_batch(const float* sBy, int Ny, int r0, int R,
                                          const float (&x)[kNB][4], float (&acc)[LYP][4]) {
#pragma unroll
    for (int u = 0; u < kNB; ++u) {
        const int row = r0 + u * R;
        if (row < Ny) {
            const float4* byr = reinterpret_cast<const float4*>(sBy + (size_t)row * LYP);
#pragma unroll
            for (int l4 = 0; l4 < LYP / 4; ++l4) {
                const float4 bb = byr[l4];
                const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        acc[4 * l4 + q][v] = fmaf(bv[q], x[u][v], acc[4 * l4 + q][v]);
            }
        }
    }
}

// Projects one frame (this CTA's) and writes its coefficients and scan position as staged frame
// b of a.c_out / a.idx_out.
template <typename FT, int LYP>
__device__ __forceinline__ void project_rows(const PrArgs& a, const FT* frame, int b, int32_t pos) {
    extern __shared__ __align__(16) float smr[];
    float* sBy = smr + pr_by_off();
    float* sBx = smr + pr_bx_off(a.Ny, LYP);
    float* sU = smr + pr_u_off(a.Ny, a.Nx, a.Lx, LYP);
    float* red = smr + pr_red_off(a.Ny, a.Nx, a.Lx, LYP);
    const int t = threadIdx.x;
    const int G = a.Nx >> 2;            // column groups
    const int R = kRowThreads / G;      // row phases
    const int cg = t % G, rp = t / G;

    float acc[LYP][4];
#pragma unroll
    for (int l = 0; l < LYP; ++l)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[l][v] = 0.f;
    const bool active = rp < R;
    const FT* col = frame + 4 * cg;
    // rows of this thread: rp + R n, n = 0, 1, ...; two batches of kNB rows are in flight, the
    // first of them issued before the bases are staged
    float xa[kNB][4], xb[kNB][4];
    if (active) load_batch<FT>(col, a.Nx, a.Ny, rp, R, xa);

    // bases into shared memory (By padded to LYP columns with zeros)
    for (int e = t; e < a.Ny * LYP; e += kRowThreads) {
        const int r = e / LYP, l = e - r * LYP;
        sBy[e] = l < a.Ly ? a.By[(size_t)r * a.Ly + l] : 0.f;
    }
    for (int e = t; e < a.Nx * a.Lx; e += kRowThreads) sBx[e] = a.Bx[e];
    __syncthreads();

    if (active) {
        // U[ly][4 cg + v] += By[i][ly] I[i][4 cg + v]; while one batch of rows is used the next
        // one is in flight
        for (int i = rp; i < a.Ny; i += 2 * kNB * R) {
            load_batch<FT>(col, a.Nx, a.Ny, i + kNB * R, R, xb);
            use_batch<LYP>(sBy, a.Ny, i, R, xa, acc);
            load_batch<FT>(col, a.Nx, a.Ny, i + 2 * kNB * R, R, xa);
            use_batch<LYP>(sBy, a.Ny, i + kNB * R, R, xb, acc);
        }
        // partial sums of this row phase: sU[rp][ly][col]
#pragma unroll
        for (int l = 0; l < LYP; ++l)
            *reinterpret_cast<float4*>(sU + ((size_t)rp * LYP + l) * a.Nx + 4 * cg) =
                make_float4(acc[l][0], acc[l][1], acc[l][2], acc[l][3]);
    }
    __syncthreads();
    // U[ly][col] = sum over the row phases in order, into phase 0's slot
    for (int e = t; e < LYP * a.Nx; e += kRowThreads) {
        float s = sU[e];
        for (int r = 1; r < R; ++r) s += sU[(size_t)r * LYP * a.Nx + e];
        sU[e] = s;
    }
    __syncthreads();
    // c_k = sum_col U[ly_k][col] Bx[col][lx_k], SP interleaved column slices per coefficient
    const int SP = a.K >= kRowThreads ? 1 : kRowThreads / a.K;
    for (int w = t; w < a.K * SP; w += kRowThreads) {
        const int k = w % a.K, sl = w / a.K;
        const int m = __ldg(&a.ktab[k].x);
        const int ly = m / a.Lx, lx = m - (m / a.Lx) * a.Lx;
        const float* ur = sU + (size_t)ly * a.Nx;
        float s = 0.f;
        for (int c = sl; c < a.Nx; c += SP) s = fmaf(ur[c], sBx[(size_t)c * a.Lx + lx], s);
        red[w] = s;
    }
    __syncthreads();
    // outputs may alias staging slots the previous kernel still reads: wait for it first
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (t == 0) a.idx_out[b] = pos;
    for (int k = t; k < a.K; k += kRowThreads) {
        float s = 0.f;
        for (int sl = 0; sl < SP; ++sl) s += red[(size_t)sl * a.K + k];
        a.c_out[(size_t)b * a.K + k] = s;
        if (a.colmax) atomicMax(a.colmax + k, __float_as_uint(fabsf(s)));
    }
}

// Segment of CTA b: segs.first[sg] <= b < segs.first[sg + 1].
__device__ __forceinline__ int frame_segment(const FrameSegs& segs, int b) {
    int sg = 0;
    while (sg + 1 < segs.nseg && b >= segs.first[sg + 1]) ++sg;
    return sg;
}

template <typename FT, int LYP>
__global__ void __launch_bounds__(kRowThreads) project_rows_kernel(const PrArgs a,
                                                                   const FrameSegs segs,
                                                                   const IndexBlock ids) {
    // the next launch may start now; outputs are written after griddepcontrol.wait
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int b = blockIdx.x;
    const int sg = frame_segment(segs, b);
    const FT* frame = static_cast<const FT*>(segs.ptr[sg]) + (size_t)(b - segs.first[sg]) * a.Ny * a.Nx;
    project_rows<FT, LYP>(a, frame, b, ids.s[b]);
}

// Several plans' gathered pushes in one launch: CTAs first[j] .. first[j + 1] - 1 project the
// frames of member j (its own detector size, bases, K and staging slots in args[j]); the frame
// segments and scan positions of all members follow one another in segs and ids.
struct PrGroup {
    PrArgs args[kProjGroupMax];
    int32_t first[kProjGroupMax + 1];
    int32_t n;
};

template <typename FT, int LYP>
__global__ void __launch_bounds__(kRowThreads) project_rows_group_kernel(const PrGroup g,
                                                                         const FrameSegs segs,
                                                                         const IndexBlock ids) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int b = blockIdx.x;
    int j = 0;
    while (j + 1 < g.n && b >= g.first[j + 1]) ++j;
    const PrArgs& a = g.args[j];
    const int sg = frame_segment(segs, b);
    const FT* frame = static_cast<const FT*>(segs.ptr[sg]) + (size_t)(b - segs.first[sg]) * a.Ny * a.Nx;
    project_rows<FT, LYP>(a, frame, b - g.first[j], ids.s[b]);
}

template <typename FT, int LYP>
cudaError_t prepare_rows_typed() {
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(project_rows_kernel<FT, LYP>));
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(project_rows_group_kernel<FT, LYP>));
    return e;
}

template <typename FT>
cudaError_t launch_rows_group_typed(const PrGroup& g, int LYP, const cudaLaunchConfig_t& cfg,
                                    const FrameSegs& segs, const IndexBlock& ids) {
    switch (LYP) {
        case 4: return cudaLaunchKernelEx(&cfg, project_rows_group_kernel<FT, 4>, g, segs, ids);
        case 8: return cudaLaunchKernelEx(&cfg, project_rows_group_kernel<FT, 8>, g, segs, ids);
        case 12: return cudaLaunchKernelEx(&cfg, project_rows_group_kernel<FT, 12>, g, segs, ids);
        default: return cudaLaunchKernelEx(&cfg, project_rows_group_kernel<FT, 16>, g, segs, ids);
    }
}

template <typename FT>
cudaError_t launch_rows_typed(const PrArgs& a, int LYP, const cudaLaunchConfig_t& cfg,
                              const FrameSegs& segs, const IndexBlock& ids) {
    switch (LYP) {
        case 4: return cudaLaunchKernelEx(&cfg, project_rows_kernel<FT, 4>, a, segs, ids);
        case 8: return cudaLaunchKernelEx(&cfg, project_rows_kernel<FT, 8>, a, segs, ids);
        case 12: return cudaLaunchKernelEx(&cfg, project_rows_kernel<FT, 12>, a, segs, ids);
        default: return cudaLaunchKernelEx(&cfg, project_rows_kernel<FT, 16>, a, segs, ids);
    }
}

}  // namespace

bool proj_rows_supported(int Ny, int Nx, int Ly, int Lx, int K, int complex_basis,
                         int frame_dtype) {
    if (complex_basis || Ly > 16 || Nx % 4 != 0 || Nx > kRowsLdMax || Nx < 16) return false;
    if (frame_dtype != WDD_FRAME_U16 && frame_dtype != WDD_FRAME_F32) return false;
    return proj_rows_smem_bytes(Ny, Nx, Ly, Lx, K) <= 200u * 1024u;
}

size_t proj_rows_smem_bytes(int Ny, int Nx, int Ly, int Lx, int K) {
    return 4 * pr_floats(Ny, Nx, Lx, K, pr_lyp(Ly));
}

cudaError_t prepare_project_rows_kernels() {
    cudaError_t e = cudaSuccess;
    if (!e) e = prepare_rows_typed<float, 4>();
    if (!e) e = prepare_rows_typed<float, 8>();
    if (!e) e = prepare_rows_typed<float, 12>();
    if (!e) e = prepare_rows_typed<float, 16>();
    if (!e) e = prepare_rows_typed<uint16_t, 4>();
    if (!e) e = prepare_rows_typed<uint16_t, 8>();
    if (!e) e = prepare_rows_typed<uint16_t, 12>();
    if (!e) e = prepare_rows_typed<uint16_t, 16>();
    return e;
}

cudaError_t launch_project_rows(const wdd_plan* P, const FrameSegs& segs, int dtype, int n,
                                bool overlap, const IndexBlock& ids, float* c_out,
                                int32_t* idx_out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > kLaunchFrames) return cudaErrorInvalidValue;
    PrArgs a;
    a.Ny = P->Ny;
    a.Nx = P->Nx;
    a.Ly = P->Ly;
    a.Lx = P->Lx;
    a.K = P->K;
    a.By = P->d_Byre;
    a.Bx = P->d_Bxre;
    a.ktab = P->d_ktab;
    a.c_out = c_out;
    a.idx_out = idx_out;
    a.colmax = P->d_colmax;
    const int LYP = pr_lyp(P->Ly);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n, 1, 1);
    cfg.blockDim = dim3(kRowThreads, 1, 1);
    cfg.dynamicSmemBytes = proj_rows_smem_bytes(P->Ny, P->Nx, P->Ly, P->Lx, P->K);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1 : 0;
    if (dtype == WDD_FRAME_U16) return launch_rows_typed<uint16_t>(a, LYP, cfg, segs, ids);
    if (dtype == WDD_FRAME_F32) return launch_rows_typed<float>(a, LYP, cfg, segs, ids);
    return cudaErrorInvalidValue;
}

int proj_rows_class(const wdd_plan* P) { return P->p.frame_dtype * 64 + pr_lyp(P->Ly); }

cudaError_t launch_project_rows_group(wdd_plan* const* plans, int count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (count > kProjGroupMax) return cudaErrorInvalidValue;
    const int cls = proj_rows_class(plans[0]);
    // the merged segment list and scan positions (kernel parameters, 17 KB: kept off the stack)
    thread_local FrameSegs segs;
    thread_local IndexBlock ids;
    PrGroup g{};
    int frames = 0, nseg = 0;
    size_t smem = 0;
    for (int j = 0; j < count; ++j) {
        const wdd_plan* P = plans[j];
        const PendingLaunch& q = P->pend;
        if (!P->proj_rows || proj_rows_class(P) != cls || q.n <= 0) return cudaErrorInvalidValue;
        if (frames + q.n > kLaunchFrames || nseg + q.segs.nseg > kMaxSegs) return cudaErrorInvalidValue;
        PrArgs& a = g.args[j];
        a.Ny = P->Ny;
        a.Nx = P->Nx;
        a.Ly = P->Ly;
        a.Lx = P->Lx;
        a.K = P->K;
        a.By = P->d_Byre;
        a.Bx = P->d_Bxre;
        a.ktab = P->d_ktab;
        a.c_out = P->d_cstage + (size_t)q.slot0 * P->K;
        a.idx_out = P->d_idxstage + q.slot0;
        a.colmax = P->d_colmax;
        g.first[j] = frames;
        for (int k = 0; k < q.segs.nseg; ++k) {
            segs.ptr[nseg + k] = q.segs.ptr[k];
            segs.first[nseg + k] = frames + q.segs.first[k];
        }
        for (int b = 0; b < q.n; ++b) ids.s[frames + b] = q.ids.s[b];
        nseg += q.segs.nseg;
        frames += q.n;
        const size_t m = proj_rows_smem_bytes(P->Ny, P->Nx, P->Ly, P->Lx, P->K);
        if (m > smem) smem = m;
    }
    g.first[count] = frames;
    g.n = count;
    segs.first[nseg] = frames;
    segs.nseg = nseg;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)frames, 1, 1);
    cfg.blockDim = dim3(kRowThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    const int LYP = pr_lyp(plans[0]->Ly);
    const int dtype = plans[0]->p.frame_dtype;
    if (dtype == WDD_FRAME_U16) return launch_rows_group_typed<uint16_t>(g, LYP, cfg, segs, ids);
    if (dtype == WDD_FRAME_F32) return launch_rows_group_typed<float>(g, LYP, cfg, segs, ids);
    return cudaErrorInvalidValue;
}

}  // namespace wdd
