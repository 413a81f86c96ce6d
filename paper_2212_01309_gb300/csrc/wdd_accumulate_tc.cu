// Phase accumulation on the 5th-generation tensor cores (tcgen05, TMEM), split FP16 precision:
//   H[v, k] += sum_b E[v, s_b] c_b[k],  E = exp(-2 pi i m / lcm)  (Eq. 14, Algorithm 2)
//
// Computed transposed, D^T = C^T E^T, so that every UMMA is as wide as the hardware allows:
//   A operand (M = 128 rows): 64 coefficients, rows 0-63 their FP16 hi parts and rows 64-127 their
//             lo parts, each column scaled by a power of two first (split_coeff_kernel);
//   B operand (N = 256 rows): Re and Im of E for 128 scan frequencies, in FP16 hi and lo parts.
// Two MMAs per 16-frame K-step (B = E_hi, then B = E_lo) accumulate in FP32 TMEM all four products
// (c_hi + c_lo)(E_hi + E_lo) = c E up to FP16-split rounding (~2^-22 relative); the epilogue adds
// the hi and lo rows and divides the scale out.
//
// Kernel structure (one CTA per 128 scan frequencies x 64 or 128 coefficients):
//   warps 0-7  build the B operand (Re/Im, hi/lo of E) for their rows in shared memory, in the
//              no-swizzle K-major core-matrix layout, from the exact integer phase index and an
//              FP64-built table; they then run the epilogue (tcgen05.ld -> shared-memory tiles ->
//              coalesced H += (hi + lo) / scale).
//   warp 8     streams the A operand (split coefficients, pre-arranged in the same layout) into
//              shared memory with 1-D TMA bulk copies, in a pipeline of its own that runs up to
//              8 stages ahead, hiding the copy latency.
//   warp 9     allocates TMEM and one elected lane issues tcgen05.mma; tcgen05.commit frees
//              each pipeline stage and finally signals the epilogue.
// Every mbarrier wait is bounded; a wait that runs out records an error code in *status and the
// CTA leaves the pipeline (after a bounded wait for its issued MMAs) and frees its TMEM.

#include <cuda_fp16.h>

#include "wdd_device.cuh"
#include "wdd_internal.h"

namespace wdd {

namespace {

constexpr int kTileV = 128;        // scan frequencies per CTA (Re and Im rows: UMMA N = 256)
constexpr int kChunk = 32;         // frames per pipeline stage (two UMMA K-steps of 16)
constexpr int kProducers = 256;    // warps 0-7
constexpr int kThreadsTC = 320;    // + TMA warp + MMA warp
constexpr int kEKStepBytes = 2 * kTileV * 16 * 2;   // one K-step of an E operand: 256 rows x 16 frames
constexpr int kEStageBytes = 2 * 2 * kEKStepBytes;  // hi and lo, two K-steps: 32 KB
constexpr int kCMTileKStep = 128 * 16 * 2;          // one K-step of a 128-row coefficient tile: 4 KB

// Shared-memory matrix descriptor, no swizzle, K-major core matrices of 8 rows x 16 bytes:
// LBO = byte distance between the two core matrices along K, SBO = between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor for kind::f16: FP16 A and B, FP32 accumulator, K-major A and B.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4)                          // D format F32
           | (0u << 7) | (0u << 10)           // A, B format F16
           | ((uint32_t)(N >> 3) << 17)       // N / 8
           | ((uint32_t)(M >> 4) << 24);      // M / 16
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* out) {
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

// x mod d for x < 2^32 with a precomputed 64-bit reciprocal (Lemire's fast modulo).
struct FastMod {
    uint64_t M;
    uint32_t d;
};
__host__ FastMod make_fastmod(uint32_t d) { return {~0ull / d + 1ull, d}; }
__device__ __forceinline__ uint32_t fastmod(uint32_t x, FastMod f) {
    uint64_t low = f.M * (uint64_t)x;
    return (uint32_t)__umul64hi(low, (uint64_t)f.d);
}
__device__ __forceinline__ uint32_t fastdiv(uint32_t x, FastMod f) {
    return (f.d == 1u) ? x : (uint32_t)__umul64hi(f.M, (uint64_t)x);
}

struct TcArgs {
    const uint16_t* csplit;   // pre-arranged A operand (see split_coeff_kernel)
    const float* scale_inv;   // [Kp] 1 / column scale
    unsigned* colmax;         // [K] per-column max |c| (reset here for the next flush)
    const int32_t* idx;       // [n] scan index of each staged frame
    const uint2* tw16;        // [lcm] (re_hi | re_lo << 16, im_hi | im_lo << 16)
    float2* H;                // [S][K]
    unsigned* status;         // error word (0 = ok)
    int n_pad, S, K, NT, Sy, Sx, lcm, my, mx, stages_total, tmem_cols, tab_mode;
    int stagesE, stagesC;     // pipeline depths (E: generated phase factors, C: coefficients)
    int rotate;               // 1: each CTA starts at its own stage (see below)
    int ktile_stages;         // stages per coefficient k-tile in the split operand
    int last;                 // 1: the last launch of a flush (resets the column maxima)
    uint64_t wait_ns;
    FastMod mod_y, mod_x;
};

// Shared-memory layout of accumulate_tc_kernel (offsets from a 1024-byte aligned base).
struct TcLayout {
    size_t e, c, bar, tmem, scale, tab, total;
};
__host__ __device__ inline TcLayout tc_layout(int NT, int stagesE, int stagesC, int lcm, int tab) {
    TcLayout L;
    const size_t cStage = (size_t)(NT / 64) * 2 * kCMTileKStep;
    L.e = 0;
    L.c = L.e + (size_t)stagesE * kEStageBytes;
    L.bar = L.c + (size_t)stagesC * cStage;
    L.tmem = L.bar + 8 * (size_t)(2 * stagesE + 2 * stagesC + 1);
    L.scale = (L.tmem + 16 + 15) & ~size_t(15);
    L.tab = (L.scale + 4 * (size_t)NT + 15) & ~size_t(15);
    // tab: 0 none (global), 1 the table twice over (index m + d < 2 lcm), 2 that doubled table
    // in 16 interleaved copies, one per bank pair
    L.total = L.tab + (tab == 1 ? 16 * (size_t)lcm : tab == 2 ? 256 * (size_t)lcm : 0);
    return L;
}

// Named barrier among the 256 threads of warps 0-7 (the epilogue phases).
__device__ __forceinline__ void epilogue_barrier() {
    asm volatile("bar.sync 1, 256;" ::: "memory");
}

// 64-bit load from a shared-memory byte address.
__device__ __forceinline__ uint2 lds_u2(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

// kTab > 0: the phase table sits in shared memory twice over (entries m and m + lcm equal), so
// the fast path adds a frame's phase step to a byte address with no reduction mod lcm; with
// kTab == 2 the doubled table is stored in 16 interleaved copies (entry e, copy c at 8 (16 e + c)
// bytes) and lane l reads copy l % 16, so the 16 lanes of a half-warp always hit 16 different
// bank pairs, whatever entries they look up.  kTab == 0: the table is read from global memory
// with reduced indices.
template <int kTab>
__global__ void __launch_bounds__(kThreadsTC, 1) accumulate_tc_kernel(const TcArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NT = a.NT;                 // coefficients per CTA (64 or 128)
    const int MT = NT / 64;              // 128-row coefficient tiles (hi rows 0-63, lo rows 64-127)
    const int SE = a.stagesE, SC = a.stagesC;
    constexpr bool kTabSmem = kTab > 0;
    constexpr uint32_t kEntryBytes = kTab == 2 ? 128u : 8u;   // stride of the table index
    const TcLayout L = tc_layout(NT, SE, SC, a.lcm, kTab);
    const int cStageBytes = MT * 2 * kCMTileKStep;
    uint8_t* e_base = base + L.e;
    uint8_t* c_base = base + L.c;
    uint64_t* fullE = reinterpret_cast<uint64_t*>(base + L.bar);
    uint64_t* emptyE = fullE + SE;
    uint64_t* fullC = emptyE + SE;
    uint64_t* emptyC = fullC + SC;
    uint64_t* done = emptyC + SC;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.tmem);
    float* s_scale = reinterpret_cast<float*>(base + L.scale);
    uint2* s_tab = reinterpret_cast<uint2*>(base + L.tab);
    const uint2* gtab = a.tw16;
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int v0 = blockIdx.x * kTileV;
    const int k0 = blockIdx.y * NT;
    // The CTAs of a launch walk the staged frames from evenly spread starting stages, so that at
    // any moment they read different parts of the coefficient operand instead of all fetching the
    // same lines from L2.  Only the order of the frames' FP32 additions changes.
    const int T = a.stages_total;
    const int rot = a.rotate ? (int)(((long long)blockIdx.x * T) / gridDim.x) : 0;
    auto stage_of = [T, rot](int it) { const int x = it + rot; return x >= T ? x - T : x; };

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < SE; ++s) {
            mbar_init(&fullE[s], kProducers / 32);   // one arrival per producer warp
            mbar_init(&emptyE[s], 1);
        }
        for (int s = 0; s < SC; ++s) {
            mbar_init(&fullC[s], 1);
            mbar_init(&emptyC[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (kTab == 1)
        for (int t = threadIdx.x; t < 2 * a.lcm; t += blockDim.x)
            s_tab[t] = a.tw16[t < a.lcm ? t : t - a.lcm];
    if (kTab == 2)
        for (int t = threadIdx.x; t < 32 * a.lcm; t += blockDim.x) {
            const int e = t >> 4;
            s_tab[t] = a.tw16[e < a.lcm ? e : e - a.lcm];
        }
    if (warp == 9) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // The next launch may start now (it holds tensor memory only where this grid does not): a
    // following segment runs its main loop, and a following projection its loads and MMAs,
    // on SMs this grid leaves free; both wait (griddepcontrol.wait) before touching anything
    // this grid writes.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (warp < 8) {
        // ---------------- E producers: phase factors as the B operand (N rows = Re, Im) ----
        const int row = threadIdx.x & (kTileV - 1);    // 0..127
        const int kstep = threadIdx.x >> 7;            // 0..1: which 16-frame K-step of a stage
        // Rows of scan frequencies beyond S (last tile) are generated for v = 0; the epilogue
        // never writes their results.
        const int v = (v0 + row < a.S) ? v0 + row : 0;
        const uint32_t vy = (uint32_t)(v / a.Sx);
        const uint32_t vx = (uint32_t)(v % a.Sx);
        const int g_re = row >> 3, g_im = 16 + (row >> 3), r = row & 7;
        // phase steps j * vx * mx mod lcm between a frame and its j-th successor in a scan row
        // (as byte offsets into the shared table when it is there)
        uint32_t dxj[16];
        {
            const uint32_t dx = vx * (uint32_t)a.mx;   // < lcm
            uint32_t acc = 0;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                dxj[j] = kTabSmem ? acc * kEntryBytes : acc;
                acc += dx;
                if (acc >= (uint32_t)a.lcm) acc -= (uint32_t)a.lcm;
            }
        }
        const uint32_t tab_s = smem_u32(s_tab) + (kTab == 2 ? (uint32_t)(lane & 15) * 8u : 0u);
        // first and last frame index of this thread's K-step, prefetched one stage ahead
        const int32_t* ip0 = a.idx + (size_t)stage_of(0) * kChunk + kstep * 16;
        int32_t nf = __ldg(ip0), nl = __ldg(ip0 + 15);
        for (int it = 0; it < a.stages_total; ++it) {
            const int st = it % SE;
            const int32_t s_first = nf, s_last = nl;
            if (it + 1 < a.stages_total) {
                const int32_t* ipn = a.idx + (size_t)stage_of(it + 1) * kChunk + kstep * 16;
                nf = __ldg(ipn);
                nl = __ldg(ipn + 15);
            }
            // one lane per warp waits for the stage to be free and tells its warp
            int ok = 1;
            if (lane == 0) {
                if (it >= SE && !mbar_wait(&emptyE[st], ((it / SE) - 1) & 1, a.wait_ns)) {
                    atomicExch(a.status, 1u);
                    s_abort = 1;
                }
                ok = !s_abort;
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            // Phase index of this thread's 16 frames, m = (vy sy mod Sy) my + (vx sx mod Sx) mx
            // (mod lcm).  Fast path, decided per K-step (warp-uniform): the 16 frames are
            // consecutive positions of one scan row, so m advances by dx = vx mx per frame.
            // Otherwise each frame's index is decoded on its own.
            const int32_t* ip = a.idx + (size_t)stage_of(it) * kChunk + kstep * 16;
            uint32_t mm[16];   // table byte addresses (shared table) or reduced indices (global)
            {
                const uint32_t s0 = (uint32_t)s_first;
                const uint32_t sy0 = fastdiv(s0, a.mod_x);
                const uint32_t sx0 = s0 - sy0 * (uint32_t)a.Sx;
                if (s_last == s_first + 15 && sx0 + 15u < (uint32_t)a.Sx) {
                    uint32_t m = fastmod(vy * sy0, a.mod_y) * (uint32_t)a.my +
                                 fastmod(vx * sx0, a.mod_x) * (uint32_t)a.mx;
                    if (m >= (uint32_t)a.lcm) m -= (uint32_t)a.lcm;
                    if (kTabSmem) {
                        const uint32_t b = tab_s + m * kEntryBytes;
#pragma unroll
                        for (int j = 0; j < 16; ++j) mm[j] = b + dxj[j];   // entry m + d < 2 lcm
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const uint32_t mj = m + dxj[j];
                            mm[j] = (mj >= (uint32_t)a.lcm) ? mj - (uint32_t)a.lcm : mj;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const uint32_t s = (uint32_t)__ldg(ip + j);
                        const uint32_t sy = fastdiv(s, a.mod_x);
                        const uint32_t sx = s - sy * (uint32_t)a.Sx;
                        uint32_t m = fastmod(vy * sy, a.mod_y) * (uint32_t)a.my +
                                     fastmod(vx * sx, a.mod_x) * (uint32_t)a.mx;
                        m = (m >= (uint32_t)a.lcm) ? m - (uint32_t)a.lcm : m;
                        mm[j] = kTabSmem ? tab_s + m * kEntryBytes : m;
                    }
                }
            }
            uint8_t* ehi = e_base + (size_t)st * kEStageBytes + kstep * kEKStepBytes;
            uint8_t* elo = ehi + 2 * kEKStepBytes;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uint2 q[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) q[e] = kTabSmem ? lds_u2(mm[c * 8 + e]) : gtab[mm[c * 8 + e]];
                uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    rh[e] = __byte_perm(q[2 * e].x, q[2 * e + 1].x, 0x5410);
                    rl[e] = __byte_perm(q[2 * e].x, q[2 * e + 1].x, 0x7632);
                    ih[e] = __byte_perm(q[2 * e].y, q[2 * e + 1].y, 0x5410);
                    il[e] = __byte_perm(q[2 * e].y, q[2 * e + 1].y, 0x7632);
                }
                const int o_re = g_re * 256 + c * 128 + r * 16;
                const int o_im = g_im * 256 + c * 128 + r * 16;
                *reinterpret_cast<uint4*>(ehi + o_re) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                *reinterpret_cast<uint4*>(ehi + o_im) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                *reinterpret_cast<uint4*>(elo + o_re) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                *reinterpret_cast<uint4*>(elo + o_im) = make_uint4(il[0], il[1], il[2], il[3]);
            }
            fence_async_smem();    // this thread's stores -> visible to the tensor core
            __syncwarp();
            if (lane == 0) mbar_arrive(&fullE[st]);
        }
    } else if (warp == 8) {
        // ---------------- C loader (TMA), running up to SC stages ahead ----------------
        if (lane == 0) {
            // the split coefficients come from the launch before (the split pre-pass)
            asm volatile("griddepcontrol.wait;" ::: "memory");
            const uint8_t* src = reinterpret_cast<const uint8_t*>(a.csplit) +
                                 (size_t)blockIdx.y * a.ktile_stages * cStageBytes;
            for (int it = 0; it < a.stages_total; ++it) {
                const int sc = it % SC;
                if (it >= SC && !mbar_wait(&emptyC[sc], ((it / SC) - 1) & 1, a.wait_ns)) {
                    atomicExch(a.status, 2u);
                    s_abort = 1;
                    break;
                }
                if (s_abort) break;
                mbar_arrive_tx(&fullC[sc], cStageBytes);
                tma_load_1d(c_base + (size_t)sc * cStageBytes, src + (size_t)stage_of(it) * cStageBytes,
                            cStageBytes, &fullC[sc]);
            }
        }
    } else {
        // ---------------- MMA issuer: D_j[coefficient row][Re v | Im v] --------------------
        // With one coefficient tile the E_hi and E_lo products go to two accumulators (added in
        // the epilogue), so consecutive MMAs do not wait on each other's accumulation.
        // Descriptors are formed once and advanced by the byte offsets of stages and K-steps.
        if (lane == 0) {
            const uint32_t idesc = instr_desc(128, 2 * kTileV);
            const uint64_t de0 = smem_desc(smem_u32(e_base), 128, 256);
            const uint64_t dc0 = smem_desc(smem_u32(c_base), 128, 256);
            const int nacc = MT == 1 ? 2 : 1;
            uint32_t acc = 0;
            int st = 0, sc = 0;
            uint32_t pe = 0, pc = 0;
            for (int it = 0; it < a.stages_total; ++it) {
                if (!mbar_wait(&fullC[sc], pc, a.wait_ns) || !mbar_wait(&fullE[st], pe, a.wait_ns)) {
                    atomicExch(a.status, 3u);
                    s_abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t de = de0 + (uint64_t)((st * kEStageBytes) >> 4);
                const uint64_t dc = dc0 + (uint64_t)((sc * cStageBytes) >> 4);
#pragma unroll
                for (int ks = 0; ks < kChunk / 16; ++ks) {
                    const uint64_t e_h = de + (uint64_t)((ks * kEKStepBytes) >> 4);
                    const uint64_t e_l = e_h + (uint64_t)((2 * kEKStepBytes) >> 4);
                    for (int j = 0; j < MT; ++j) {
                        const uint64_t cd = dc + (uint64_t)(((j * 2 + ks) * kCMTileKStep) >> 4);
                        const uint32_t d = tmem + (uint32_t)(j * nacc * 2 * kTileV);
                        mma_f16(d, cd, e_h, idesc, acc);
                        mma_f16(d + (uint32_t)((nacc - 1) * 2 * kTileV), cd, e_l, idesc,
                                nacc == 2 ? acc : 1u);
                    }
                    acc = 1u;
                }
                mma_commit(&emptyE[st]);   // free both stages once these MMAs have read them
                mma_commit(&emptyC[sc]);
                if (++st == SE) { st = 0; pe ^= 1u; }
                if (++sc == SC) { sc = 0; pc ^= 1u; }
            }
            mma_commit(done);              // all issued MMAs complete -> epilogue
        }
    }

    // H (and the column maxima) may still be written by the previous launch: wait for it to
    // complete before the epilogue reads them.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // ---------------- epilogue: warps 0-7 ----------------
    // TMEM lane = coefficient row (0-63: hi part, 64-127: lo part); column = Re v | Im v.
    // Warps whose lane quarter holds hi rows write tile T_hi[v][k], the others T_lo[v][k]
    // (both in the freed E stage buffers), then all eight warps add T_hi + T_lo, scale and
    // update H with whole 128-byte row segments.
    if (warp < 8) {
        int ok = 1;
        if (lane == 0) {
            ok = mbar_wait(done, 0, a.wait_ns) ? 1 : 0;
            if (!ok) atomicExch(a.status, 4u);
            ok = ok && !s_abort;
        }
        const bool go = __shfl_sync(0xffffffffu, ok, 0) != 0;   // tcgen05.ld needs the whole warp
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // column scales (from the split pre-pass; read after the wait above, ordered before
        // their use by the epilogue barrier below)
        for (int t = threadIdx.x; t < NT; t += kProducers) {
            const int k = k0 + t;
            s_scale[t] = (k < a.K) ? a.scale_inv[k] : 0.f;
        }
        const int quarter = warp & 3;                 // TMEM lanes 32 q .. 32 q + 31
        const int half = warp >> 2;                   // which half of the v columns
        const int krow = (quarter & 1) * 32 + lane;   // coefficient within the m-tile
        float2* T = reinterpret_cast<float2*>(e_base) + (size_t)(quarter >> 1) * kTileV * 64;
        const int nacc = MT == 1 ? 2 : 1;
        for (int j = 0; j < MT; ++j) {
            if (go) {
                const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) +
                                           (uint32_t)(j * nacc * 2 * kTileV);
                for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 16) {
                    float re[16], im[16];
                    tmem_ld16(lane_addr + (uint32_t)c0, re);
                    tmem_ld16(lane_addr + (uint32_t)(kTileV + c0), im);
                    if (nacc == 2) {   // E_lo products in the second accumulator
                        float re2[16], im2[16];
                        tmem_ld16(lane_addr + (uint32_t)(2 * kTileV + c0), re2);
                        tmem_ld16(lane_addr + (uint32_t)(3 * kTileV + c0), im2);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            re[i] += re2[i];
                            im[i] += im2[i];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) T[(size_t)(c0 + i) * 64 + krow] = make_float2(re[i], im[i]);
                }
            }
            epilogue_barrier();
            if (go) {
                // Each warp updates rows vr = warp + 8 i of the tile, a lane two coefficients
                // per row; the H values of 8 rows are loaded before any is stored, so the loads
                // overlap instead of waiting on each other's stores.
                const float2* Thi = reinterpret_cast<const float2*>(e_base);
                const float2* Tlo = Thi + (size_t)kTileV * 64;
                for (int vb = 0; vb < kTileV / 8; vb += 8) {
                    float2 hv[8][2];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int vv = v0 + warp + 8 * (vb + i);
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const int k = k0 + j * 64 + hh * 32 + lane;
                            hv[i][hh] = (vv < a.S && k < a.K) ? a.H[(size_t)vv * a.K + k]
                                                              : make_float2(0.f, 0.f);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int vr = warp + 8 * (vb + i);
                        const int vv = v0 + vr;
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const int kl = hh * 32 + lane;
                            const int k = k0 + j * 64 + kl;
                            if (vv < a.S && k < a.K) {
                                const float2 x = Thi[(size_t)vr * 64 + kl], y = Tlo[(size_t)vr * 64 + kl];
                                const float sc = s_scale[j * 64 + kl];
                                float2 h = hv[i][hh];
                                h.x = fmaf(x.x + y.x, sc, h.x);
                                h.y = fmaf(x.y + y.y, sc, h.y);
                                a.H[(size_t)vv * a.K + k] = h;
                            }
                        }
                    }
                }
            }
            epilogue_barrier();
        }
    }
    if (blockIdx.x == 0 && blockIdx.y == 0)
        if (a.last)
            for (int t = threadIdx.x; t < a.K; t += blockDim.x) a.colmax[t] = 0u;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 9) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(a.tmem_cols));
    }
}

// Splits the staged FP32 coefficients into FP16 hi/lo parts with a power-of-two scale per column
// and writes them as the A operand of accumulate_tc_kernel:
//   [k-tile][stage][m-tile][K-step][row group][core matrix b/8 % 2][row % 8][b % 8]
// where an m-tile holds 64 coefficients, rows 0-63 their hi parts and rows 64-127 their lo
// parts.  Frames beyond n and coefficients beyond K are zero.  One thread per (frame, column).
__global__ void split_coeff_kernel(const float* __restrict__ c, const unsigned* __restrict__ colmax,
                                   uint16_t* __restrict__ out, float* __restrict__ scale_inv,
                                   int n, int n_pad, int K, int Kp, int NT) {
    // the accumulation launched next sets up and generates phase factors meanwhile; it reads
    // this kernel's output only after griddepcontrol.wait.  Its producers read the staged scan
    // indices at once: that is safe because this kernel is launched without programmatic
    // serialization, so the projection that wrote them has completed before it started.  (A
    // programmatic launch of this kernel would have to wait before releasing its dependents.)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int kk = t % Kp;
    const int b = t / Kp;
    if (b >= n_pad) return;
    float cm = (kk < K) ? __uint_as_float(colmax[kk]) : 0.f;
    int e = 0;
    if (cm > 0.f) frexpf(cm, &e);
    const float sc = (cm > 0.f) ? ldexpf(1.f, 14 - e) : 1.f;
    if (b == 0) scale_inv[kk] = (kk < K && cm > 0.f) ? ldexpf(1.f, e - 14) : 0.f;
    const float x = (b < n && kk < K) ? c[(size_t)b * K + kk] * sc : 0.f;
    const __half hi = __float2half_rn(x);
    const __half lo = __float2half_rn(x - __half2float(hi));
    const int ktile = kk / NT, kl = kk % NT;
    const int mtile = kl / 64, km = kl % 64;
    const int MT = NT / 64;
    const int stage = b / kChunk, bs = b % kChunk;
    const int ks = bs / 16, bk = bs % 16;
    const int stages_total = n_pad / kChunk;
    const size_t stage_halves = (size_t)MT * 2 * (kCMTileKStep / 2);
    const size_t base = ((size_t)ktile * stages_total + stage) * stage_halves +
                        (size_t)(mtile * 2 + ks) * (kCMTileKStep / 2);
    const int rh = km, rl = 64 + km;
    const size_t in_hi = (size_t)(rh >> 3) * 128 + (size_t)(bk >> 3) * 64 + (size_t)(rh & 7) * 8 + (bk & 7);
    const size_t in_lo = (size_t)(rl >> 3) * 128 + (size_t)(bk >> 3) * 64 + (size_t)(rl & 7) * 8 + (bk & 7);
    out[base + in_hi] = __half_as_ushort(hi);
    out[base + in_lo] = __half_as_ushort(lo);
}

// Exercises the bounded mbarrier wait on a barrier that nothing arrives on: the wait must give
// up after wait_ns and record code 7 in *status, leaving the context usable.
__global__ void bounded_wait_selftest_kernel(unsigned* status, uint64_t wait_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait(&bar, 0, wait_ns)) atomicExch(status, 7u);
        mbar_arrive(&bar);   // complete the phase so no wait is left pending
    }
}

}  // namespace

cudaError_t launch_bounded_wait_selftest(unsigned* status, uint64_t wait_ns, cudaStream_t st) {
    bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(status, wait_ns);
    return cudaGetLastError();
}

bool split_path_available() { return true; }

cudaError_t prepare_split_kernels() {
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(accumulate_tc_kernel<0>));
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(accumulate_tc_kernel<1>));
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(accumulate_tc_kernel<2>));
    return e;
}

// Coefficients per CTA: 64 (one hi/lo m-tile) or 128 (two).
int split_tile_n(int K) { return K <= 64 ? 64 : 128; }

// Pipeline depths for a tile width NT within the shared-memory budget.  The E region must hold
// the two epilogue tiles (128 KB), so it keeps 4 stages; C takes what is left, up to 8, after
// the phase table.  The table goes to shared memory in the best form that leaves 3 or more C
// stages: the bank-interleaved copies, else the doubled table; otherwise it stays in global.
static void split_stages(int NT, int lcm, int* se, int* sc, int* tab) {
    const size_t limit = 226 * 1024 - 1024;   // dynamic bytes after the alignment slack
    const int E = 4;
    for (int mode = 2; mode >= 1; --mode)
        for (int C = 8; C >= 3; --C)
            if (tc_layout(NT, E, C, lcm, mode).total <= limit) {
                *se = E;
                *sc = C;
                *tab = mode;
                return;
            }
    int C = 8;
    while (C > 2 && tc_layout(NT, E, C, lcm, 0).total > limit) --C;
    *se = E;
    *sc = C;
    *tab = 0;
}

size_t split_smem_bytes(int NT) {
    int E, C, T;
    split_stages(NT, 1, &E, &C, &T);
    return 1024 + tc_layout(NT, E, C, 1, 0).total;
}

// Kernel launches of one flush of n staged frames: the split pre-pass and one per segment.
int split_launch_count(int n, int segment) {
    const int n_pad = (n + kChunk - 1) / kChunk * kChunk;
    return 1 + (n_pad + segment - 1) / segment;
}

size_t split_coeff_bytes(int K, int depth_pad) {
    const int NT = split_tile_n(K);
    const int Kp = (K + NT - 1) / NT * NT;
    return (size_t)Kp * depth_pad * 2 * 2;   // hi and lo halves
}

cudaError_t launch_accumulate_split(const wdd_plan* P, const float* c, const int32_t* idx, int n,
                                    cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int NT = split_tile_n(P->K);
    const int Kp = (P->K + NT - 1) / NT * NT;
    const int n_pad = (n + kChunk - 1) / kChunk * kChunk;
    if (n_pad > P->depth_pad) return cudaErrorInvalidValue;
    // 1. split the coefficients (per-column scale from the projection's running max)
    {
        const size_t total = (size_t)n_pad * Kp;
        split_coeff_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            c, P->d_colmax, reinterpret_cast<uint16_t*>(P->d_bsplit), P->d_scale_inv, n, n_pad,
            P->K, Kp, NT);
    }
    // 2. tensor-core accumulation
    TcArgs a;
    a.csplit = reinterpret_cast<const uint16_t*>(P->d_bsplit);
    a.scale_inv = P->d_scale_inv;
    a.colmax = P->d_colmax;
    a.idx = idx;
    a.tw16 = reinterpret_cast<const uint2*>(P->d_tw16);
    a.H = P->d_H;
    a.status = P->d_status;
    a.n_pad = n_pad;
    a.S = P->S;
    a.K = P->K;
    a.NT = NT;
    a.Sx = P->Sx;
    a.Sy = P->Sy;
    a.lcm = P->lcm;
    a.my = P->lcm / P->Sy;
    a.mx = P->lcm / P->Sx;
    a.stages_total = n_pad / kChunk;
    a.tmem_cols = 4 * kTileV;   // two 256-column accumulators (E_hi / E_lo parts, or two tiles)
    a.wait_ns = kDeviceWaitNs;
    a.rotate = 1;
    a.mod_y = make_fastmod((uint32_t)P->Sy);
    a.mod_x = make_fastmod((uint32_t)P->Sx);
    split_stages(NT, P->lcm, &a.stagesE, &a.stagesC, &a.tab_mode);
    const size_t smem = 1024 + tc_layout(NT, a.stagesE, a.stagesC, P->lcm, a.tab_mode).total;
    dim3 grid((P->S + kTileV - 1) / kTileV, Kp / NT);
    // One launch per segment of at most P->segment staged frames: the tensor cores' FP32
    // accumulation loses a little precision with every MMA added into an accumulator (error
    // linear in the number added), so long flushes run as several launches whose sums are added
    // into H in FP32 in between.
    const int stages_all = n_pad / kChunk;
    const int seg = P->segment / kChunk;
    const size_t c_stage_halves = (size_t)(NT / 64) * kCMTileKStep;   // one stage of one k-tile
    a.ktile_stages = stages_all;
    for (int s0 = 0; s0 < stages_all; s0 += seg) {
        TcArgs b = a;
        b.stages_total = stages_all - s0 < seg ? stages_all - s0 : seg;
        b.csplit = a.csplit + (size_t)s0 * c_stage_halves;
        b.idx = idx + (size_t)s0 * kChunk;
        b.last = s0 + seg >= stages_all ? 1 : 0;
        // every segment overlaps the launch before it (programmatic dependent launch): the first
        // sets up and generates phase factors while the split pre-pass runs and loads the split
        // coefficients after griddepcontrol.wait; later ones overlap the previous segment's
        // tail and read H only after griddepcontrol.wait
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(kThreadsTC, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e;
        if (b.tab_mode == 2)
            e = cudaLaunchKernelEx(&cfg, accumulate_tc_kernel<2>, b);
        else if (b.tab_mode == 1)
            e = cudaLaunchKernelEx(&cfg, accumulate_tc_kernel<1>, b);
        else
            e = cudaLaunchKernelEx(&cfg, accumulate_tc_kernel<0>, b);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace wdd
