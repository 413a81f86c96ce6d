// Frame ingest and projection on the 5th-generation tensor cores (split-precision path):
//   c_b[k] = sum_{i,j} By[i, ly_k] I_b[i, j] Bx[j, lx_k]      (Sect. 5, operator H of Eq. 12)
// as T = I Bx on the tensor cores (tcgen05.mma, kind::f16, FP32 accumulator in TMEM), then
// Z = By^T T on the SIMT cores and the K selected entries of Z.
//
// Precision: the frame and the basis are both split into FP16 hi and lo parts,
//   I s = I_hi + I_lo,   Bx = Bx_hi + Bx_lo,
// with s = 1/2 for uint16 counts (so that every value up to 65535 has a finite FP16 hi part and an
// exact lo part) and s = 1 for float32 frames, whose values must stay below the FP16 overflow
// threshold (|I| < 65520) and be finite; a value whose hi part overflows to infinity, or a NaN,
// is reported through the plan's device status word (code 9).  The B operand
// holds Bx_hi in rows 0..Lx-1 and Bx_lo in rows Lx..2Lx-1, so two MMAs per 16 columns (A = I_hi,
// then A = I_lo) accumulate all four products; the epilogue adds the hi and lo column groups and
// divides s out.  The representation error of each split is about 2^-22 relative, below FP32
// accumulation error, and uint16 counts are represented exactly.
//
// One CTA per frame.  The frame is read in (128-row tile, 32-column chunk) items with 16-byte
// loads, coalesced along rows (frames in pinned host memory are read over the host link by the
// same loads); the next item's loads are in flight while one item is converted.  The threads
// split an item into its FP16 parts and store them in one of two A buffers in the UMMA
// no-swizzle K-major layout, and one thread issues the MMAs, so converting an item overlaps the
// MMAs of the previous one.  The basis image and By arrive by TMA bulk copies while the first
// item is converted.  After each tile the accumulator rows (one TMEM lane per detector row) are
// read back, the hi and lo column groups added in registers, into a shared-memory T tile.
// Several CTAs share an SM, so one CTA's loads overlap another's conversion.
//
// Launch ordering is the same as the SIMT projection's (programmatic dependent launch, outputs
// written after griddepcontrol.wait).  The CTA allocates its tensor memory before it lets the
// next launch start, so a dependent CTA that waits for this grid never holds memory this grid
// still needs.  Every mbarrier wait is bounded; a wait that gives up records code 8 in the
// status word, skips the remaining MMAs and frees the tensor memory.

#include <cuda_fp16.h>

#include <type_traits>

#include "wdd_device.cuh"
#include "wdd_internal.h"

namespace wdd {

namespace {

constexpr int kTM = 128;          // detector rows per tile (UMMA M, one TMEM lane per row)
constexpr int kTK = 32;           // detector columns per chunk (two UMMA K-steps)
constexpr int kKC = kTK / 8;      // 8-column K-chunks (core matrices) per chunk
constexpr int kU = kTK / 16;      // (8-row group, 32-column quarter) units per thread
constexpr int kAHalfBytes = kTM * kTK * 2;   // one FP16 part of a chunk

struct PtcArgs {
    int Ny, Nx, Ly, Lx, K, Np, SP, tmem_cols;
    float scale, inv_scale;
    const uint16_t* bimg;     // B operand image (see build_bimg_kernel)
    const float* By;          // [Ny * Ly rounded up to 4] real parts of the row basis
    const int2* ktab;         // [K] (ly * Lx + lx, 0)
    float* c_out;             // [n][K]
    int32_t* idx_out;         // [n]
    unsigned* colmax;         // [K] running max |c| (float bits)
    unsigned* status;
    uint64_t wait_ns;
};

struct PtcLayout {
    size_t b, a, by, t, red, bar, slot, total;
};

__host__ __device__ inline size_t by_floats(int Ny, int Ly) { return ((size_t)Ny * Ly + 3) / 4 * 4; }

__host__ __device__ inline PtcLayout ptc_layout(int Ny, int Nx, int Ly, int Lx, int K, int Np,
                                                int SP) {
    PtcLayout L;
    L.b = 0;
    L.a = (L.b + (size_t)Np * Nx * 2 + 127) & ~size_t(127);
    // two A buffers (hi, lo), also holding the padded accumulator rows of a finished tile
    const size_t a_bytes = 4 * (size_t)kAHalfBytes > (size_t)kTM * (Np + 1) * 4
                               ? 4 * (size_t)kAHalfBytes : (size_t)kTM * (Np + 1) * 4;
    L.by = L.a + ((a_bytes + 15) & ~size_t(15));
    L.t = (L.by + 4 * by_floats(Ny, Ly) + 15) & ~size_t(15);
    L.red = (L.t + 4 * (size_t)Ny * Lx + 15) & ~size_t(15);
    L.bar = (L.red + 4 * (size_t)SP * K + 15) & ~size_t(15);   // MMA buffer 0, 1; basis copy
    L.slot = L.bar + 24;
    L.total = L.slot + 8;
    return L;
}

__device__ __forceinline__ uint64_t desc_nosw(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // tcgen05 descriptor version; no swizzle, base offset 0
    return d;
}

__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, float* out) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(r[i]);
}

// Eight consecutive frame values as FP32.
__device__ __forceinline__ void load8(const float* p, float* x) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
__device__ __forceinline__ void load8(const uint16_t* p, float* x) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        x[2 * i] = (float)(w[i] & 0xFFFFu);
        x[2 * i + 1] = (float)(w[i] >> 16);
    }
}

// FP16 hi and lo parts of eight values (already scaled), packed in pairs.
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __half2 hh = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
        const float2 hf = __half22float2(hh);
        const __half2 ll = __floats2half2_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
        h[i] = *reinterpret_cast<const uint32_t*>(&hh);
        l[i] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Loads this thread's part of item `it` = (tile it / chunks, chunk it % chunks); zeros outside
// the frame.  uint16 frames: for unit v = warp + 8 u, row 8 (v % 16) + r of the tile and columns
// 32 (v / 16) + 8 q .. + 7 of the chunk (one 16-byte load; a warp reads 64 contiguous bytes of
// each of 8 rows).  float32 frames: row 8 (v % 16) + (lane >> 2) and columns 4 (lane & 3) .. + 3
// and 16 + 4 (lane & 3) .. + 3 (two 16-byte loads, each reading 64 contiguous bytes of 8 rows:
// whole 32-byte sectors per instruction).
template <typename FT>
__device__ __forceinline__ void load_item(const FT* frame, int it, int n_items, int chunks, int Ny,
                                          int Nx, int warp, int r, int q, float (&dst)[kU][8]) {
    const int mt = it / chunks, kc = it % chunks;
    const int w = min(kTK, Nx - kc * kTK);   // a multiple of 16
    if constexpr (std::is_same<FT, float>::value) {
        const int lane = r + 8 * q;
        const int rr = lane >> 2, c4 = 4 * (lane & 3);
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int v = warp + 8 * u;
            const int row = mt * kTM + 8 * (v & 15) + rr;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = 16 * h + c4;
                if (it < n_items && col < w && row < Ny) {
                    const float4 a = __ldg(reinterpret_cast<const float4*>(
                        frame + (size_t)row * Nx + kc * kTK + col));
                    dst[u][4 * h] = a.x;
                    dst[u][4 * h + 1] = a.y;
                    dst[u][4 * h + 2] = a.z;
                    dst[u][4 * h + 3] = a.w;
                } else {
                    dst[u][4 * h] = dst[u][4 * h + 1] = dst[u][4 * h + 2] = dst[u][4 * h + 3] = 0.f;
                }
            }
        }
        return;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        const int v = warp + 8 * u;
        const int row = mt * kTM + 8 * (v & 15) + r;
        const int col = 32 * (v >> 4) + 8 * q;
        if (it < n_items && col < w && row < Ny) {
            load8(frame + (size_t)row * Nx + kc * kTK + col, dst[u]);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) dst[u][e] = 0.f;
        }
    }
}

// T[row][0 .. LX) = (D[row][n] + D[row][LX + n]) * inv for n < LX from the thread's TMEM lane
// (columns 0 .. LX - 1 hold the Bx_hi products, LX .. 2 LX - 1 the Bx_lo ones).
template <int LX>
__device__ __forceinline__ void tile_rows_direct(uint32_t taddr, float inv, float* trow, bool ok) {
    float d[2 * LX > 16 ? 2 * LX : 16];
#pragma unroll
    for (int c0 = 0; c0 < 2 * LX; c0 += 16) tmem_ld_x16(taddr + (uint32_t)c0, d + c0);
    if (ok) {
#pragma unroll
        for (int n = 0; n < LX; n += 4)
            *reinterpret_cast<float4*>(trow + n) =
                make_float4((d[n] + d[LX + n]) * inv, (d[n + 1] + d[LX + n + 1]) * inv,
                            (d[n + 2] + d[LX + n + 2]) * inv, (d[n + 3] + d[LX + n + 3]) * inv);
    }
}

// Four CTAs per SM (64 registers): more CTAs in flight hide the per-item load latency better
// than staging whole frames in shared memory, which leaves room for only two.
template <typename FT>
__global__ void __launch_bounds__(kThreads, 4)
project_tc_kernel(const PtcArgs a, const FrameSegs segs, const IndexBlock ids) {
    extern __shared__ __align__(128) uint8_t sm[];
    const int tiles = (a.Ny + kTM - 1) / kTM;
    const PtcLayout L = ptc_layout(a.Ny, a.Nx, a.Ly, a.Lx, a.K, a.Np, a.SP);
    uint8_t* sB = sm + L.b;
    uint8_t* sA = sm + L.a;                 // 2 x [hi | lo], each [16 row groups][4 K-chunks][8][8]
    float* sBy = reinterpret_cast<float*>(sm + L.by);
    float* sT = reinterpret_cast<float*>(sm + L.t);
    float* red = reinterpret_cast<float*>(sm + L.red);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + L.bar);   // [2] MMAs of A buffer 0 / 1
    uint64_t* bload = mbar + 2;                                 // basis image and By copies
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + L.slot);
    __shared__ int s_fail;

    const int b = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int sg = 0;
    while (sg + 1 < segs.nseg && b >= segs.first[sg + 1]) ++sg;
    const FT* frame = static_cast<const FT*>(segs.ptr[sg]) + (size_t)(b - segs.first[sg]) * a.Ny * a.Nx;
    // lane -> (row r of an 8-row group, 8-column K-chunk q of a 32-column quarter); warp w
    // converts the units w, w + 8, ... (unit v: row group v % 16, quarter v / 16)
    const int r = lane & 7, q = lane >> 3;
    const int chunks = a.Nx / kTK + (a.Nx % kTK ? 1 : 0);
    const int n_items = tiles * chunks;     // (tile, chunk) items in order
    float x[kU][8];                         // raw values of the item in flight
    // the first item's loads go out before anything else
    load_item(frame, 0, n_items, chunks, a.Ny, a.Nx, warp, r, q, x);

    const unsigned b_bytes = (unsigned)(a.Np * a.Nx * 2);
    const unsigned by_bytes = (unsigned)(4 * by_floats(a.Ny, a.Ly));
    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init(bload, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(slot)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    // the next launch may start now: this CTA already holds its tensor memory
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // basis image (B operand) and By: bulk copies, complete before the first MMA / contraction
    if (threadIdx.x == 0) {
        mbar_arrive_tx(bload, b_bytes + by_bytes);
        tma_load_1d(sB, a.bimg, b_bytes, bload);
        tma_load_1d(sBy, a.By, by_bytes, bload);
    }
    // this thread's first coefficient of the second contraction, fetched early
    const int m_first = threadIdx.x < a.K * a.SP ? __ldg(&a.ktab[threadIdx.x % a.K].x) : 0;

    const uint32_t idesc = idesc_f16(kTM, a.Np);
    const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);
    const uint32_t sboB = (uint32_t)(a.Nx / 8) * 128u;
    uint32_t range_bad = 0;   // float32 frames: nonzero once a hi part is infinite or NaN
    bool basis_ready = false;
    int issued = 0, done = 0;   // items whose MMAs were issued / are known complete

    for (int it = 0; it < n_items; ++it) {
        const int mt = it / chunks, kc = it % chunks;
        const int w = min(kTK, a.Nx - kc * kTK);
        const int ab = it & 1;
        uint8_t* sAb = sA + (size_t)ab * 2 * kAHalfBytes;
        // buffer ab is free once the MMAs of item it - 2 have completed (they complete in order)
        if (it >= 2 && done < it - 1) {
            if (threadIdx.x == 0 &&
                !mbar_wait(&mbar[ab], (unsigned)((it - 2) >> 1) & 1u, a.wait_ns)) {
                atomicExch(a.status, 8u);
                s_fail = 1;
            }
            done = it - 1;
        }
        __syncthreads();
        if (s_fail) break;
        // split and store in the UMMA layout: offset (g * kKC + K-chunk) * 128 + row * 16
        if constexpr (std::is_same<FT, float>::value) {
            // four values per 16-byte load: 8-byte halves of core-matrix rows (two lanes share
            // each bank pair: conflict-free)
            const int rr = lane >> 2, c4 = 4 * (lane & 3);
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int v = warp + 8 * u;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int col = 16 * h + c4;
                    if (col < w) {
                        const float* y = x[u] + 4 * h;   // scale 1 for float32 frames
                        const __half2 h0 = __floats2half2_rn(y[0], y[1]);
                        const __half2 h1 = __floats2half2_rn(y[2], y[3]);
                        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&h0);
                        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&h1);
                        range_bad |= __vcmpeq2(b0 & 0x7C007C00u, 0x7C007C00u) |
                                     __vcmpeq2(b1 & 0x7C007C00u, 0x7C007C00u);
                        const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
                        const __half2 l0 = __floats2half2_rn(y[0] - f0.x, y[1] - f0.y);
                        const __half2 l1 = __floats2half2_rn(y[2] - f1.x, y[3] - f1.y);
                        const int off = ((v & 15) * kKC + (col >> 3)) * 128 + rr * 16 + ((col & 7) >> 2) * 8;
                        *reinterpret_cast<uint2*>(sAb + off) = make_uint2(b0, b1);
                        *reinterpret_cast<uint2*>(sAb + kAHalfBytes + off) =
                            make_uint2(*reinterpret_cast<const uint32_t*>(&l0),
                                       *reinterpret_cast<const uint32_t*>(&l1));
                    }
                }
            }
        } else {
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int v = warp + 8 * u;
            const int kcl = 4 * (v >> 4) + q;     // K-chunk within the chunk
            if (8 * kcl < w) {
                float y[8];   // uint16 counts times 1/2: always within the FP16 range
#pragma unroll
                for (int e = 0; e < 8; ++e) y[e] = x[u][e] * a.scale;
                uint4 hi, lo;
                split8(y, hi, lo);
                const int off = ((v & 15) * kKC + kcl) * 128 + r * 16;
                *reinterpret_cast<uint4*>(sAb + off) = hi;
                *reinterpret_cast<uint4*>(sAb + kAHalfBytes + off) = lo;
            }
        }
        }
        // the next item's loads
        load_item(frame, it + 1, n_items, chunks, a.Ny, a.Nx, warp, r, q, x);
        fence_async_smem();
        __syncthreads();
        // one thread issues the MMAs of this chunk: D[row][n] += A_hi B^T + A_lo B^T
        if (threadIdx.x == 0) {
            if (!basis_ready) {
                if (!mbar_wait(bload, 0, a.wait_ns)) {
                    atomicExch(a.status, 8u);
                    s_fail = 1;
                }
                basis_ready = true;
            }
            if (!s_fail) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sAb_u = sA_u + (uint32_t)(ab * 2 * kAHalfBytes);
                for (int ks = 0; ks < w / 16; ++ks) {
                    const uint64_t ah = desc_nosw(sAb_u + (uint32_t)ks * 256u, 128, kKC * 128);
                    const uint64_t al =
                        desc_nosw(sAb_u + kAHalfBytes + (uint32_t)ks * 256u, 128, kKC * 128);
                    const uint64_t bd =
                        desc_nosw(sB_u + (uint32_t)(kc * kKC + 2 * ks) * 128u, 128, sboB);
                    umma_f16(tmem, ah, bd, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                    umma_f16(tmem, al, bd, idesc, 1u);
                }
                umma_commit(&mbar[ab]);
            }
        }
        issued = it + 1;
        if (kc + 1 < chunks) continue;
        // tile epilogue: wait for this tile's MMAs; TMEM lane = detector row
        if (threadIdx.x == 0 && !s_fail && !mbar_wait(&mbar[ab], (unsigned)(it >> 1) & 1u, a.wait_ns)) {
            atomicExch(a.status, 8u);
            s_fail = 1;
        }
        __syncthreads();
        if (s_fail) break;
        done = it + 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (a.Lx == 8 || a.Lx == 16) {
            // T[row][lx] = (D[lx] + D[Lx + lx]) / s straight from the thread's TMEM lane
            if (warp < 4) {
                const int row = mt * kTM + 32 * warp + lane;
                const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
                float* trow = sT + (size_t)row * a.Lx;
                if (a.Lx == 8)
                    tile_rows_direct<8>(taddr, a.inv_scale, trow, row < a.Ny);
                else
                    tile_rows_direct<16>(taddr, a.inv_scale, trow, row < a.Ny);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();   // TMEM is read: the next tile's first MMA may overwrite it
        } else {
            // raw accumulator rows -> the idle A buffers (row stride Np + 1: conflict-free)
            float* sD = reinterpret_cast<float*>(sA);
            const int ldD = a.Np + 1;
            if (warp < 4) {
                const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
                const int rl = 32 * warp + lane;
                for (int c0 = 0; c0 < a.Np; c0 += 16) {
                    float d[16];
                    tmem_ld_x16(taddr + (uint32_t)c0, d);
#pragma unroll
                    for (int e = 0; e < 16; ++e) sD[(size_t)rl * ldD + c0 + e] = d[e];
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();   // TMEM is read: the next tile's first MMA may overwrite it
            // column n holds basis row n: Bx_hi for n < Lx, Bx_lo for Lx <= n < 2 Lx
            for (int t = threadIdx.x; t < kTM * a.Lx; t += blockDim.x) {
                const int rl = t / a.Lx, lx = t % a.Lx;
                const int row = mt * kTM + rl;
                if (row < a.Ny)
                    sT[(size_t)row * a.Lx + lx] =
                        (sD[(size_t)rl * ldD + lx] + sD[(size_t)rl * ldD + a.Lx + lx]) * a.inv_scale;
            }
            __syncthreads();   // the A buffers are free again
        }
    }
    if (range_bad != 0u) atomicExch(a.status, 9u);
    const bool failed = s_fail != 0;

    // second contraction: Z[ly][lx] = sum_i By[i][ly] T[i][lx], the rows of each selected
    // coefficient split into SP interleaved slices summed in slice order
    if (!failed) {
        for (int t = threadIdx.x; t < a.K * a.SP; t += blockDim.x) {
            const int k = t % a.K, sl = t / a.K;
            const int m = (t == threadIdx.x) ? m_first : __ldg(&a.ktab[k].x);
            const int ly = m / a.Lx, lx = m % a.Lx;
            float acc = 0.f;
            for (int i = sl; i < a.Ny; i += a.SP)
                acc = fmaf(sBy[(size_t)i * a.Ly + ly], sT[(size_t)i * a.Lx + lx], acc);
            red[(size_t)sl * a.K + k] = acc;
        }
    }
    __syncthreads();
    // outputs may alias staging slots the previous kernel still reads: wait for it first
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) a.idx_out[b] = ids.s[b];
    if (!failed) {
        for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
            float acc = 0.f;
            for (int sl = 0; sl < a.SP; ++sl) acc += red[(size_t)sl * a.K + k];
            a.c_out[(size_t)b * a.K + k] = acc;
            if (a.colmax) atomicMax(a.colmax + k, __float_as_uint(fabsf(acc)));
        }
    }
    if (failed && threadIdx.x == 0) {
        // before the tensor and shared memory go: bounded waits for MMAs and copies in flight
        for (int j = done; j < issued; ++j) mbar_wait(&mbar[j & 1], (unsigned)(j >> 1) & 1u, a.wait_ns);
        if (!basis_ready) mbar_wait(bload, 0, a.wait_ns);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(a.tmem_cols));
    }
}

// B operand image for the projection: row n < Lx holds the FP16 hi part of Bx[:, n], row
// Lx + n its lo part (both from the FP64 basis), rows up to Np are zero; layout
//   [n / 8][j / 8][n % 8][j % 8]   (core matrices of 8 rows x 16 bytes, K-major).
__global__ void build_bimg_kernel(const double2* __restrict__ Bx, int Nx, int Lx, int Np,
                                  uint16_t* __restrict__ img) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Np * Nx) return;
    const int n = t / Nx, j = t % Nx;
    __half h = __float2half_rn(0.f);
    if (n < 2 * Lx) {
        const int l = n < Lx ? n : n - Lx;
        const double v = Bx[(size_t)j * Lx + l].x;
        const __half hi = __double2half(v);
        h = n < Lx ? hi : __double2half(v - (double)__half2float(hi));
    }
    const size_t off = ((size_t)(n >> 3) * (Nx >> 3) + (j >> 3)) * 64 + (size_t)(n & 7) * 8 + (j & 7);
    img[off] = __half_as_ushort(h);
}

template <typename FT>
cudaError_t prepare_tc_typed() {
    return allow_max_dynamic_smem(reinterpret_cast<const void*>(project_tc_kernel<FT>));
}

}  // namespace

int proj_tc_np(int Lx) { return (2 * Lx + 15) / 16 * 16; }

size_t proj_tc_smem_bytes(int Ny, int Nx, int Ly, int Lx, int K) {
    const int SP = K >= kThreads ? 1 : kThreads / K;
    return ptc_layout(Ny, Nx, Ly, Lx, K, proj_tc_np(Lx), SP).total + 128;
}

bool proj_tc_supported(int Nx, int Lx, int complex_basis, int frame_dtype) {
    return !complex_basis && (frame_dtype == WDD_FRAME_U16 || frame_dtype == WDD_FRAME_F32) &&
           Nx >= 16 && Nx % 16 == 0 && proj_tc_np(Lx) <= 64;
}

size_t proj_tc_bimg_halves(int Nx, int Lx) { return (size_t)proj_tc_np(Lx) * Nx; }

cudaError_t launch_build_bimg(const wdd_plan* P, uint16_t* img, cudaStream_t st) {
    const int Np = proj_tc_np(P->Lx);
    const int total = Np * P->Nx;
    build_bimg_kernel<<<(total + 255) / 256, 256, 0, st>>>(P->d_Bx, P->Nx, P->Lx, Np, img);
    return cudaGetLastError();
}

cudaError_t prepare_project_tc_kernels() {
    cudaError_t e = prepare_tc_typed<uint16_t>();
    if (e == cudaSuccess) e = prepare_tc_typed<float>();
    return e;
}

cudaError_t launch_project_tc(const wdd_plan* P, const FrameSegs& segs, int dtype, int n,
                              bool overlap, const IndexBlock& ids, float* c_out, int32_t* idx_out,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > kLaunchFrames) return cudaErrorInvalidValue;
    PtcArgs a;
    a.Ny = P->Ny;
    a.Nx = P->Nx;
    a.Ly = P->Ly;
    a.Lx = P->Lx;
    a.K = P->K;
    a.Np = proj_tc_np(P->Lx);
    a.SP = P->K >= kThreads ? 1 : kThreads / P->K;
    a.tmem_cols = a.Np <= 32 ? 32 : 64;
    a.scale = dtype == WDD_FRAME_U16 ? 0.5f : 1.0f;
    a.inv_scale = dtype == WDD_FRAME_U16 ? 2.0f : 1.0f;
    a.bimg = P->d_bimg;
    a.By = P->d_Byre;
    a.ktab = P->d_ktab;
    a.c_out = c_out;
    a.idx_out = idx_out;
    a.colmax = P->d_colmax;
    a.status = P->d_status;
    a.wait_ns = kDeviceWaitNs;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = proj_tc_smem_bytes(P->Ny, P->Nx, P->Ly, P->Lx, P->K);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1 : 0;
    if (dtype == WDD_FRAME_U16)
        return cudaLaunchKernelEx(&cfg, project_tc_kernel<uint16_t>, a, segs, ids);
    if (dtype == WDD_FRAME_F32) return cudaLaunchKernelEx(&cfg, project_tc_kernel<float>, a, segs, ids);
    return cudaErrorInvalidValue;
}

}  // namespace wdd
