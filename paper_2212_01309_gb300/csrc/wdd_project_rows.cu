// Frame ingest and projection in FP32 on the SIMT cores, one warp per frame:
//   c_b[k] = sum_{i,j} By[i, ly_k] I_b[i, j] Bx[j, lx_k]      (Sect. 5, operator H of Eq. 12)
// for real (Hermite-Gauss) bases with at most 16 functions along each detector axis.
//
// The projection reads every frame byte once and does about 2 L_y flops per pixel, far below the
// tensor cores' ridge, so its bound is the frame read (HBM, or the host link for frames in pinned
// host memory), provided the arithmetic around the reads stays small.  This kernel is written for
// that bound:
//
//  * A team of TW = ceil(N_x / 128) warps owns a frame; lane l of warp w owns the four adjacent
//    detector columns 4 (32 w + l) .. + 3 and reads its four values of each row with one 16-byte
//    (float32) or 8-byte (uint16) load, so a warp reads whole contiguous rows.  Detectors of
//    16, 32 or 64 columns fold 32 / (N_x / 4) row phases into the warp instead.  Each lane keeps
//    two batches of rows in flight (8 float32 or 16 uint16 rows, 32 registers each) and
//    accumulates U[ly][col] = sum_i By[i, ly] I[i, col] for its columns in registers.
//  * Nothing is reduced across warps for the first contraction: a frame's U for a column lives in
//    one lane.  The second contraction c_k = sum_col U[ly_k][col] Bx[col, lx_k] is formed per
//    lane over its four columns for blocks of (32 / LXP) basis rows x LXP basis columns, and the
//    32 lanes' partial sums are combined by a butterfly reduce-scatter (five xor shuffles),
//    after which lane l holds one finished (ly, lx) sum of the block.  Row phases within a warp
//    are first added by xor shuffles.  Teams of several warps add their partial results in
//    shared memory, in warp order.
//  * The CTAs are persistent: a launch runs as many CTAs as fit on the SMs, shared among the
//    launch's plans in proportion to their frames; each CTA serves one plan, whose row basis
//    (zero-padded to LYP columns) it stages in shared memory once, and team t of a plan's T teams
//    projects the contiguous frames [t n / T, (t + 1) n / T) of its n.  The first batch of rows
//    of a team's next frame is loaded before the current frame's contraction, so loads stay in
//    flight across it.  Frame loads skip L1 allocation (each byte is read once); the column
//    basis, zero-padded to LXP columns, is read through L1.
//  * The running maximum |c| per coefficient (float bits compared as unsigned integers, read by
//    the split pre-pass for its scales) is kept per lane and added into colmax once per team
//    and plan, not once per frame.
//
// Every sum has a fixed order (rows in order per lane, butterfly pairs by lane index, warps in
// order), so results are bit-reproducible and independent of where the frames are stored and of
// how a launch's frames are shared among CTAs.
//
// One kernel serves single-plan and grouped launches: the launch describes 1 .. 8 plans
// ("members", each with its own detector size, bases, K and staging slots, one team size) whose
// frames follow one another in the launch's frame list.
//
// Launch ordering is that of the other projection kernels: the kernel lets the next launch start
// at once (it holds no tensor memory) and writes its outputs after griddepcontrol.wait.

#include <algorithm>
#include <type_traits>

#include "wdd_device.cuh"
#include "wdd_internal.h"

namespace wdd {

namespace {

constexpr int kWarpsPerCta = 4;
constexpr int kColsMax = 512;      // widest detector: teams of up to four warps

struct PrArgs {
    int Ny, Nx, K;
    const float* By;          // [Ny][LYP] real parts of the row basis, zero-padded (FP32)
    const float* Bx;          // [Nx][LXP] real parts of the column basis, zero-padded (FP32)
    const int32_t* kpad;      // [K] ly * LXP + lx of coefficient k
    float* c_out;             // [n][K]
    int32_t* idx_out;         // [n]
    unsigned* colmax;         // [K] running max |c| (float bits) or NULL
};

// Members of a launch: member j's frames are launch frames first[j] .. first[j + 1] - 1 (every
// member has at least one frame) and its CTAs are cfirst[j] .. cfirst[j + 1] - 1; the frame
// segments and scan positions of all members follow one another in the launch's FrameSegs and
// IndexBlock.  All members have the same team size tw.
struct PrGroup {
    PrArgs args[kProjGroupMax];
    int32_t first[kProjGroupMax + 1];
    int32_t cfirst[kProjGroupMax + 1];   // CTAs cfirst[j] .. cfirst[j + 1] - 1 serve member j
    int32_t n;
    int32_t tw;
};

__host__ __device__ inline int pr_team(int Nx) { return (Nx / 4 + 31) / 32; }

// Rows of one batch per lane: 32 registers of raw frame values either way.
template <typename FT> struct RowBatch;
template <> struct RowBatch<float> {
    static constexpr int kRows = 8;
    float4 v[kRows];
};
template <> struct RowBatch<uint16_t> {
    static constexpr int kRows = 16;
    uint2 v[kRows];
};

// Exact uint16 -> float: the 16-bit value in the mantissa of 2^23, minus 2^23.
__device__ __forceinline__ float u16_lo(unsigned w) {
    return __uint_as_float(0x4B000000u | (w & 0xFFFFu)) - 8388608.0f;
}
__device__ __forceinline__ float u16_hi(unsigned w) {
    return __uint_as_float(0x4B000000u | (w >> 16)) - 8388608.0f;
}
__device__ __forceinline__ void unpack(const float4& r, float (&x)[4]) {
    x[0] = r.x; x[1] = r.y; x[2] = r.z; x[3] = r.w;
}
__device__ __forceinline__ void unpack(const uint2& r, float (&x)[4]) {
    x[0] = u16_lo(r.x); x[1] = u16_hi(r.x); x[2] = u16_lo(r.y); x[3] = u16_hi(r.y);
}

// This lane's place in its team for a member's detector width.
struct Lane {
    int cg;      // column group: columns 4 cg .. 4 cg + 3
    int rp;      // row phase
    int rw;      // row phases in the warp
    bool on;     // owns columns
};

__device__ __forceinline__ Lane lane_of(int Nx, int tw, int wt, int lane) {
    Lane q;
    const int G = Nx >> 2;
    if (tw == 1 && (G & (G - 1)) == 0 && G < 32) {
        q.rw = 32 / G;
        q.cg = lane & (G - 1);
        q.rp = lane / G;
        q.on = true;
    } else {
        q.rw = 1;
        q.cg = wt * 32 + lane;
        q.rp = 0;
        q.on = q.cg < G;
    }
    return q;
}

__device__ __forceinline__ int member_of(const PrGroup& g, int b) {
    int j = 0;
    while (j + 1 < g.n && b >= g.first[j + 1]) ++j;
    return j;
}

// Segment holding launch frame b, searching onward from segment sg.
__device__ __forceinline__ int segment_from(const FrameSegs& segs, int sg, int b) {
    while (sg + 1 < segs.nseg && b >= segs.first[sg + 1]) ++sg;
    return sg;
}

template <typename FT>
__device__ __forceinline__ const FT* frame_ptr(const FrameSegs& segs, int sg, int b, const PrArgs& a) {
    return static_cast<const FT*>(segs.ptr[sg]) + (size_t)(b - segs.first[sg]) * a.Ny * a.Nx;
}

// Frame rows are read once: the loads skip L1 allocation so they do not evict the bases.
__device__ __forceinline__ void ldg_row(const float* p, float4& r) {
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
}
__device__ __forceinline__ void ldg_row(const uint16_t* p, uint2& r) {
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
}

// Loads rows r0, r0 + R, ... (one batch, those below Ny) of this lane's four columns.
template <typename FT>
__device__ __forceinline__ void load_batch(const FT* col, int Nx, int Ny, int r0, int R,
                                           RowBatch<FT>& x) {
#pragma unroll
    for (int u = 0; u < RowBatch<FT>::kRows; ++u)
        if (r0 + u * R < Ny) ldg_row(col + (size_t)(r0 + u * R) * Nx, x.v[u]);
}

// acc[ly][v] += By[row][ly] I[row][col v] for the batch's rows below Ny (By in shared memory, the
// same row for every lane of a warp).
template <typename FT, int LYP>
__device__ __forceinline__ void use_batch(const float* sBy, int Ny, int r0, int R,
                                          const RowBatch<FT>& x, float (&acc)[LYP][4]) {
#pragma unroll
    for (int u = 0; u < RowBatch<FT>::kRows; ++u) {
        const int row = r0 + u * R;
        if (row < Ny) {
            float xv[4];
            unpack(x.v[u], xv);
            const float4* byr = reinterpret_cast<const float4*>(sBy + (size_t)row * LYP);
#pragma unroll
            for (int l4 = 0; l4 < LYP / 4; ++l4) {
                const float4 bb = byr[l4];
                const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        acc[4 * l4 + q][v] = fmaf(bv[q], xv[v], acc[4 * l4 + q][v]);
            }
        }
    }
}

// One butterfly step of the reduce-scatter: of the LEN values in P, a lane whose `mask` bit is
// set keeps the upper half and the other lane of the pair the lower half, each adding its
// partner's copy of the half it keeps; the kept half moves to P[0 .. LEN/2).
template <int LEN>
__device__ __forceinline__ void rs_step(float (&P)[32], int mask, int lane) {
    const bool up = (lane & mask) != 0;
#pragma unroll
    for (int i = 0; i < LEN / 2; ++i) {
        const float send = up ? P[i] : P[LEN / 2 + i];
        const float keep = up ? P[LEN / 2 + i] : P[i];
        P[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, mask);
    }
}

// Adds this lane's running max |c| of coefficients lane + 32 m into the member's colmax.
__device__ __forceinline__ void flush_colmax(const PrArgs& a, unsigned (&cm)[8], int lane) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int k = lane + 32 * m;
        if (a.colmax && k < a.K && cm[m]) atomicMax(a.colmax + k, cm[m]);
        cm[m] = 0u;
    }
}

__device__ __forceinline__ void team_sync(int team, int tw) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(32 * tw) : "memory");
}

// CTAs per SM the register budget is sized for: three for up to eight basis rows, two above.
template <int LYP> struct MinCtas { static constexpr int value = LYP <= 8 ? 3 : 2; };

template <typename FT, int LYP, int LXP>
__global__ void __launch_bounds__(kWarpsPerCta * 32, MinCtas<LYP>::value)
project_rows_kernel(const PrGroup g, const FrameSegs segs, const IndexBlock ids) {
    extern __shared__ __align__(16) float smf[];
    // the next launch may start now; outputs are written after griddepcontrol.wait
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int QB = 32 / LXP;                   // basis rows per contraction block
    constexpr int NB = RowBatch<FT>::kRows;
    static_assert(LYP % QB == 0, "contraction blocks must tile the padded basis rows");
    const int tw = g.tw;
    const int warps = (int)(blockDim.x >> 5);
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int tpc = warps / tw;                    // teams per CTA
    const int team = warp / tw, wt = warp - team * tw;
    // this CTA's plan; its row basis into shared memory after each warp's block sums
    int j = 0;
    while (j + 1 < g.n && (int)blockIdx.x >= g.cfirst[j + 1]) ++j;
    const PrArgs& a = g.args[j];
    float* zw = smf + (size_t)warp * LYP * LXP;
    const float* zt = smf + (size_t)team * tw * LYP * LXP;
    float* sBy = smf + (size_t)warps * LYP * LXP;
    for (int e = (int)threadIdx.x; e < a.Ny * LYP; e += (int)blockDim.x) sBy[e] = a.By[e];
    __syncthreads();
    if (team >= tpc) return;
    const long long T = (long long)(g.cfirst[j + 1] - g.cfirst[j]) * tpc;
    const long long gt = (long long)((int)blockIdx.x - g.cfirst[j]) * tpc + team;
    const int nj = g.first[j + 1] - g.first[j];
    const int b0 = g.first[j] + (int)(gt * nj / T), b1 = g.first[j] + (int)((gt + 1) * nj / T);
    if (b0 >= b1) return;                          // the same for every warp of the team

    const Lane q = lane_of(a.Nx, tw, wt, lane);
    int sg = segment_from(segs, 0, b0);
    RowBatch<FT> xa, xb;
    if (q.on) load_batch<FT>(frame_ptr<FT>(segs, sg, b0, a) + 4 * q.cg, a.Nx, a.Ny, q.rp, q.rw, xa);
    bool waited = false;
    unsigned cm[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};   // running max |c| of k = lane + 32 m
    for (int b = b0; b < b1; ++b) {
        float acc[LYP][4];
#pragma unroll
        for (int l = 0; l < LYP; ++l)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[l][v] = 0.f;
        if (q.on) {
            // U[ly][4 cg + v] += By[i][ly] I[i][4 cg + v]; one batch of rows in flight while the
            // other is used
            const FT* col = frame_ptr<FT>(segs, sg, b, a) + 4 * q.cg;
            for (int i = q.rp; i < a.Ny; i += 2 * NB * q.rw) {
                load_batch<FT>(col, a.Nx, a.Ny, i + NB * q.rw, q.rw, xb);
                use_batch<FT, LYP>(sBy, a.Ny, i, q.rw, xa, acc);
                load_batch<FT>(col, a.Nx, a.Ny, i + 2 * NB * q.rw, q.rw, xa);
                use_batch<FT, LYP>(sBy, a.Ny, i + NB * q.rw, q.rw, xb, acc);
            }
        }
        // the next frame's first rows go in flight now, across this frame's contraction
        const int sgn = b + 1 < b1 ? segment_from(segs, sg, b + 1) : sg;
        if (b + 1 < b1 && q.on)
            load_batch<FT>(frame_ptr<FT>(segs, sgn, b + 1, a) + 4 * q.cg, a.Nx, a.Ny, q.rp, q.rw, xa);
        // row phases folded into the warp: add them (lanes cg + G r), in xor order
        if (q.rw > 1) {
            for (int m = a.Nx >> 2; m < 32; m <<= 1) {
#pragma unroll
                for (int l = 0; l < LYP; ++l)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        acc[l][v] += __shfl_xor_sync(0xFFFFFFFFu, acc[l][v], m);
            }
        }
        const bool contrib = q.on && q.rp == 0;
        // c = U Bx in blocks of QB basis rows x LXP basis columns: per-lane partial sums over the
        // lane's four columns, then the butterfly reduce-scatter over the warp's 32 lanes
#pragma unroll
        for (int l0 = 0; l0 < LYP; l0 += QB) {
            float P[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) P[i] = 0.f;
            if (contrib) {
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float4* bxr = reinterpret_cast<const float4*>(a.Bx + (size_t)(4 * q.cg + v) * LXP);
#pragma unroll
                    for (int x4 = 0; x4 < LXP / 4; ++x4) {
                        const float4 t = __ldg(bxr + x4);
                        const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                        for (int qq = 0; qq < QB; ++qq)
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                P[qq * LXP + 4 * x4 + e] =
                                    fmaf(acc[l0 + qq][v], tv[e], P[qq * LXP + 4 * x4 + e]);
                    }
                }
            }
            rs_step<32>(P, 16, lane);
            rs_step<16>(P, 8, lane);
            rs_step<8>(P, 4, lane);
            rs_step<4>(P, 2, lane);
            rs_step<2>(P, 1, lane);
            // lane holds entry `lane` of the block: basis row l0 + lane / LXP, column lane % LXP
            zw[l0 * LXP + lane] = P[0];
        }
        // outputs may alias staging slots the previous kernel still reads: wait for it first
        if (!waited) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            waited = true;
        }
        const int bl = b - g.first[j];
        if (tw == 1) {
            __syncwarp();
            if (lane == 0) a.idx_out[bl] = ids.s[b];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int k = lane + 32 * m;
                if (k < a.K) {
                    const float c = zw[__ldg(&a.kpad[k])];
                    a.c_out[(size_t)bl * a.K + k] = c;
                    cm[m] = max(cm[m], __float_as_uint(fabsf(c)));
                }
            }
            __syncwarp();
        } else {
            // the team's warps cover different columns: add their block sums in warp order
            team_sync(team, tw);
            if (wt == 0) {
                if (lane == 0) a.idx_out[bl] = ids.s[b];
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int k = lane + 32 * m;
                    if (k < a.K) {
                        const int e = __ldg(&a.kpad[k]);
                        float c = zt[e];
                        for (int w = 1; w < tw; ++w) c += zt[(size_t)w * LYP * LXP + e];
                        a.c_out[(size_t)bl * a.K + k] = c;
                        cm[m] = max(cm[m], __float_as_uint(fabsf(c)));
                    }
                }
            }
            team_sync(team, tw);
        }
        sg = sgn;
    }
    flush_colmax(a, cm, lane);
}

template <typename FT, int LYP, int LXP>
cudaError_t launch_typed(const cudaLaunchConfig_t& cfg, const PrGroup& g, const FrameSegs& segs,
                         const IndexBlock& ids) {
    return cudaLaunchKernelEx(&cfg, project_rows_kernel<FT, LYP, LXP>, g, segs, ids);
}

template <typename FT, int LXP>
const void* kernel_for_lyp(int LYP) {
    switch (LYP) {
        case 4: return reinterpret_cast<const void*>(project_rows_kernel<FT, 4, LXP>);
        case 8: return reinterpret_cast<const void*>(project_rows_kernel<FT, 8, LXP>);
        case 12: return reinterpret_cast<const void*>(project_rows_kernel<FT, 12, LXP>);
        default: return reinterpret_cast<const void*>(project_rows_kernel<FT, 16, LXP>);
    }
}

const void* kernel_for(int dtype, int LYP, int LXP) {
    if (dtype == WDD_FRAME_U16)
        return LXP == 8 ? kernel_for_lyp<uint16_t, 8>(LYP) : kernel_for_lyp<uint16_t, 16>(LYP);
    return LXP == 8 ? kernel_for_lyp<float, 8>(LYP) : kernel_for_lyp<float, 16>(LYP);
}

template <typename FT, int LXP>
cudaError_t launch_lyp(int LYP, const cudaLaunchConfig_t& cfg, const PrGroup& g,
                       const FrameSegs& segs, const IndexBlock& ids) {
    switch (LYP) {
        case 4: return launch_typed<FT, 4, LXP>(cfg, g, segs, ids);
        case 8: return launch_typed<FT, 8, LXP>(cfg, g, segs, ids);
        case 12: return launch_typed<FT, 12, LXP>(cfg, g, segs, ids);
        default: return launch_typed<FT, 16, LXP>(cfg, g, segs, ids);
    }
}

// Dynamic shared memory of a CTA of `warps` warps: block sums and the row basis of Ny rows.
size_t rows_smem(int warps, int Ny, int LYP, int LXP) {
    return sizeof(float) * ((size_t)warps * LYP * LXP + (size_t)Ny * LYP);
}

// Persistent grid: as many CTAs as fit on the device at once (no more than the frames need),
// shared among the members in proportion to their frames, at least one each.
cudaError_t launch_rows(PrGroup& g, int dtype, int LYP, int LXP, int ny_max, bool overlap,
                        const FrameSegs& segs, const IndexBlock& ids, cudaStream_t st) {
    if (dtype != WDD_FRAME_U16 && dtype != WDD_FRAME_F32) return cudaErrorInvalidValue;
    if (g.tw < 1 || g.tw > kWarpsPerCta || g.n < 1) return cudaErrorInvalidValue;
    const int tpc = kWarpsPerCta / g.tw;
    const int threads = 32 * tpc * g.tw;
    const size_t smem = rows_smem(threads / 32, ny_max, LYP, LXP);
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(dtype, LYP, LXP),
                                                                  threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long n = g.first[g.n];
    const long long cap = (long long)std::max(1, per_sm) * sms;
    int ctas = 0;
    for (int j = 0; j < g.n; ++j) {
        const long long nj = g.first[j + 1] - g.first[j];
        const long long need = (nj + tpc - 1) / tpc;
        const long long share = std::max(1LL, cap * nj / n);
        g.cfirst[j] = ctas;
        ctas += (int)std::min(need, share);
    }
    g.cfirst[g.n] = ctas;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1 : 0;
    if (dtype == WDD_FRAME_U16)
        return LXP == 8 ? launch_lyp<uint16_t, 8>(LYP, cfg, g, segs, ids)
                        : launch_lyp<uint16_t, 16>(LYP, cfg, g, segs, ids);
    return LXP == 8 ? launch_lyp<float, 8>(LYP, cfg, g, segs, ids)
                    : launch_lyp<float, 16>(LYP, cfg, g, segs, ids);
}

// Member arguments of one plan whose launch writes staging slots c_out / idx_out.
PrArgs member_args(const wdd_plan* P, float* c_out, int32_t* idx_out) {
    PrArgs a;
    a.Ny = P->Ny;
    a.Nx = P->Nx;
    a.K = P->K;
    a.By = P->d_Byp;
    a.Bx = P->d_Bxp;
    a.kpad = P->d_kpad;
    a.c_out = c_out;
    a.idx_out = idx_out;
    a.colmax = P->d_colmax;
    return a;
}

}  // namespace

int proj_rows_lyp(int Ly) { return (Ly + 3) / 4 * 4; }
int proj_rows_lxp(int Lx) { return Lx <= 8 ? 8 : 16; }

bool proj_rows_supported(int Ny, int Nx, int Ly, int Lx, int K, int complex_basis,
                         int frame_dtype) {
    if (complex_basis || Ly > 16 || Lx > 16 || K > 256 || K < 1 || Ny < 1 || Ny > 2048) return false;
    if (Nx % 4 != 0 || Nx < 16 || Nx > kColsMax) return false;
    return frame_dtype == WDD_FRAME_U16 || frame_dtype == WDD_FRAME_F32;
}

cudaError_t prepare_project_rows_kernels() {
    cudaError_t e = cudaSuccess;
    for (int dt : {WDD_FRAME_U16, WDD_FRAME_F32})
        for (int lyp : {4, 8, 12, 16})
            for (int lxp : {8, 16})
                if (e == cudaSuccess) e = allow_max_dynamic_smem(kernel_for(dt, lyp, lxp));
    return e;
}

cudaError_t launch_project_rows(const wdd_plan* P, const FrameSegs& segs, int dtype, int n,
                                bool overlap, const IndexBlock& ids, float* c_out,
                                int32_t* idx_out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > kLaunchFrames || segs.nseg < 1 || segs.first[0] != 0 || segs.first[segs.nseg] != n)
        return cudaErrorInvalidValue;
    PrGroup g{};
    g.args[0] = member_args(P, c_out, idx_out);
    g.first[0] = 0;
    g.first[1] = n;
    g.n = 1;
    g.tw = pr_team(P->Nx);
    return launch_rows(g, dtype, proj_rows_lyp(P->Ly), proj_rows_lxp(P->Lx), P->Ny, overlap, segs,
                       ids, st);
}

int proj_rows_class(const wdd_plan* P) {
    return ((P->p.frame_dtype * 32 + proj_rows_lyp(P->Ly)) * 32 + proj_rows_lxp(P->Lx)) * 8 +
           pr_team(P->Nx);
}

cudaError_t launch_project_rows_group(wdd_plan* const* plans, int count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (count > kProjGroupMax) return cudaErrorInvalidValue;
    const int cls = proj_rows_class(plans[0]);
    // the merged segment list and scan positions (kernel parameters, 17 KB: kept off the stack)
    thread_local FrameSegs segs;
    thread_local IndexBlock ids;
    PrGroup g{};
    int frames = 0, nseg = 0, ny_max = 0;
    for (int j = 0; j < count; ++j) {
        const wdd_plan* P = plans[j];
        const PendingLaunch& q = P->pend;
        if (!P->proj_rows || proj_rows_class(P) != cls || q.n <= 0) return cudaErrorInvalidValue;
        if (frames + q.n > kLaunchFrames || nseg + q.segs.nseg > kMaxSegs) return cudaErrorInvalidValue;
        g.args[j] = member_args(P, P->d_cstage + (size_t)q.slot0 * P->K, P->d_idxstage + q.slot0);
        g.first[j] = frames;
        for (int k = 0; k < q.segs.nseg; ++k) {
            segs.ptr[nseg + k] = q.segs.ptr[k];
            segs.first[nseg + k] = frames + q.segs.first[k];
        }
        for (int b = 0; b < q.n; ++b) ids.s[frames + b] = q.ids.s[b];
        nseg += q.segs.nseg;
        frames += q.n;
        ny_max = std::max(ny_max, P->Ny);
    }
    g.first[count] = frames;
    g.n = count;
    g.tw = pr_team(plans[0]->Nx);
    segs.first[nseg] = frames;
    segs.nseg = nseg;
    return launch_rows(g, plans[0]->p.frame_dtype, proj_rows_lyp(plans[0]->Ly),
                       proj_rows_lxp(plans[0]->Lx), ny_max, false, segs, ids, st);
}

}  // namespace wdd
