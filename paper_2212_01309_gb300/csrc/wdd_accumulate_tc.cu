// Phase accumulation on the 5th-generation tensor cores (tcgen05, TMEM), split FP16 precision:
//   H[v, k] += sum_b E[v, s_b] c_b[k],  E = exp(-2 pi i m / lcm)  (Eq. 14, Algorithm 2)
//
// For K > 64 one CTA owns 64 scan frequencies and NT = 128 coefficients and runs every staged
// frame of a flush through them (K <= 64: accumulate_narrow_kernel below).  The 128 rows of the MMA (TMEM lanes) hold the real parts of the 64
// frequencies' phase factors (rows 0-63) and their imaginary parts (rows 64-127):
//   A operand (TMEM, M = 128 x K = 16 frames): Re or Im of E, generated in the kernel and written
//             straight into tensor memory (tcgen05.st) as an FP16 hi part and an FP16 lo part, so
//             it never passes through shared memory;
//   B operand (SMEM, N = 2 NT rows): the NT coefficients' FP16 hi parts (rows 0 .. NT-1) and lo
//             parts (rows NT .. 2NT-1), each column scaled by a power of two first
//             (split_coeff_kernel), streamed in by 1-D TMA bulk copies.
// Per 16-frame K-step two MMAs accumulate in FP32 TMEM
//   D[row, 0:2NT] += A_hi [c_hi | c_lo],   D[row, 0:NT] += A_lo c_hi,
// i.e. (E_hi + E_lo)(c_hi + c_lo) without the lo*lo product, which lies below FP32 rounding
// (~2^-24 relative): the split carries about 22 significant bits.  The epilogue adds columns k
// and NT + k, divides the scale out and adds row r (Re) and row 64 + r (Im) into H.
// Stacking Re and Im in M halves each thread's arithmetic per phase factor, and with NT = 128
// every generated value feeds an N = 256 MMA.
//
// Phase factors: E[v, s] = exp(-2 pi i (v_y s_y / S_y + v_x s_x / S_x)) (the 2-D scan DFT of
// Eq. 14, separable in the scan axes).  For 16 frames at consecutive positions of one scan row
// (raster order), E[v, s0 + j] = E[v, s0] w_v^j with w_v = exp(-2 pi i v_x / S_x): one FP32 table
// entry (exact integer index m = (v_y s_y mod S_y)(lcm / S_y) + (v_x s_x mod S_x)(lcm / S_x)
// mod lcm into a table built in FP64) times powers w_v^j read once from the same table.  The
// split pre-pass marks each 16-frame group that is such a run; other groups take one table entry
// per frame.  Both are products of correctly rounded FP32 values, within a few 2^-24 of the FP64
// phase factor before the FP16 split.
//
// Accuracy bookkeeping: TMEM accumulates `seg_stages` stages (accum_segment frames); then the
// epilogue adds the segment into H in FP32 and the next segment starts a fresh accumulator (the
// tensor cores' FP32 accumulation error grows with the number of products added into one
// accumulator).  All segments of a flush run in one launch.
//
// Warp roles (576 threads, one CTA per SM: all 512 TMEM columns):
//   warps 0-15  producers: warp w fills TMEM lanes 32 (w % 4) .. + 31 for K-step w / 4 of every
//               64-frame stage; they also run the epilogue (tcgen05.ld -> FP32 running sums
//               in shared-memory tiles -> coalesced H += sum / scale);
//   warp 16     TMA loader of the B operand;
//   warp 17     TMEM allocation; one elected lane issues tcgen05.mma and the commits.
// A stage (64 frames, eight MMAs) is filled by the sixteen producer warps and one TMA copy, all
// arriving on one `full` barrier, and released by one tcgen05.commit on its `empty` barrier.
// The issue loop has no integer division (a single thread's scalar latency bounded an earlier
// version of this loop, not the tensor pipe).  Between segments each producer thread adds its
// row of D (hi and lo columns) into FP32 running sums in its part of the shared-memory epilogue
// tile, so the MMAs wait only for that read; H is read and written once per flush.
// TMEM columns: D 0 .. 2NT-1, four A slots of 64 columns from 2NT (slot a, K-step ks: hi part at
// 2NT + 64 a + 16 ks, lo part 8 columns further; two frames per column).
// Every mbarrier wait is bounded; a wait that runs out records an error code in *status, the
// CTA stops issuing work, waits (bounded) for the MMAs it issued and frees its TMEM.
// This launch starts while the split pre-pass still runs (programmatic dependent launch), so
// everything earlier launches wrote (the group records and scan indices, the scales, H) is read
// after griddepcontrol.wait and through L2 (ld.global.cg), never through the non-coherent L1
// path: with several plans' work in flight on other streams, L1 lines of the previous flush's
// records were seen served to a later flush.  Only the phase table, fixed since the plan was
// built, is read through L1.

#include <algorithm>

#include <cuda_fp16.h>

#include "wdd_device.cuh"
#include "wdd_internal.h"

namespace wdd {

namespace {

constexpr int kTileV = 64;         // scan frequencies per CTA (Re and Im: MMA M = 128)
constexpr int kChunk = 64;         // frames per pipeline stage (four UMMA K-steps of 16)
constexpr int kKSteps = kChunk / 16;
constexpr int kProdWarps = 16;     // warps 0-15: four lane quarters x four K-steps
constexpr int kProducers = 32 * kProdWarps;
constexpr int kThreadsTC = kProducers + 64;   // + TMA warp + MMA warp
constexpr int kStages = 4;         // pipeline stages (A slots in TMEM, B slots in shared memory)
constexpr int kTmemCols = 512;
constexpr size_t kTcSmemRequest = 160 * 1024;

// Coefficient tile geometry.
template <int NT>
struct Tile {
    static constexpr int kKStepBytes = 2 * NT * 16 * 2;        // B: 2 NT rows x 16 frames, FP16
    static constexpr int kStageBytes = kKSteps * kKStepBytes;
    static constexpr int kColsD = 2 * NT;
    static constexpr int kRowBytes = NT * 4 + 16;              // epilogue tile row (floats + pad)
};

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

// D[tmem_d] (+)= A[tmem_a] * B[desc_b]: A from tensor memory, B from shared memory.
__device__ __forceinline__ void mma_f16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db,
                                           uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
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

// Phase index m = (v_y s_y mod S_y) my + (v_x s_x mod S_x) mx mod lcm of scan position s (any
// 32-bit value: the reductions keep m below lcm even for positions outside the scan).
__device__ __forceinline__ uint32_t phase_index(uint32_t s, uint32_t vy, uint32_t vx, FastMod fy,
                                                FastMod fx, uint32_t Sx, uint32_t my, uint32_t mx,
                                                uint32_t lcm) {
    const uint32_t sy = fastdiv(s, fx);
    const uint32_t sx = s - sy * Sx;
    uint32_t m = fastmod(vy * sy, fy) * my + fastmod(vx * sx, fx) * mx;
    return m >= lcm ? m - lcm : m;
}

// hi and lo FP16 parts of two FP32 values, packed (first value in the low half).
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

struct TcArgs {
    const uint16_t* csplit;   // B operand (see split_coeff_kernel), [k-tile][stage][stage bytes]
    const float* scale_inv;   // [Kp] 1 / column scale
    unsigned* colmax;         // [K] per-column max |c| (reset here for the next flush)
    const int32_t* idx;       // [n_pad] scan index of each staged frame
    const int2* grp;          // [n_pad / 16] per 16-frame group: (first scan index s0,
                              // (s0 mod S_x) << 1 | 1 if the 16 are consecutive positions of
                              // one scan row)
    const float2* tw;         // [lcm] exp(-2 pi i m / lcm), FP32 from FP64
    float2* H;                // [S_y S_x][K]
    unsigned* status;         // error word (0 = ok)
    int S, K, Sy, Sx, lcm, my, mx;   // S: frequencies processed, S_y x Sh (rows of the tiles)
    int Sh;                   // scan columns processed per row: S_x, or S_x / 2 + 1 when the
                              // rest follow from Hermitian symmetry (mirror_h_kernel)
    int stages_total;         // 64-frame stages of the flush
    int seg_stages;           // stages per TMEM accumulation segment
    int segments;             // ceil(stages_total / seg_stages)
    uint64_t wait_ns;
    FastMod mod_y, mod_x;
};

// Row of H of processed frequency number r (r = row Sh + column, column < Sh).
__device__ __forceinline__ size_t h_row(const TcArgs& a, int r) {
    const int ry = r / a.Sh;
    return (size_t)ry * a.Sx + (r - ry * a.Sh);
}

// Shared-memory layout (offsets from a 1024-byte aligned base).
struct TcLayout {
    size_t c, tile, bar, tmem, scale, total;
};
template <int NT>
__host__ __device__ inline TcLayout tc_layout() {
    TcLayout L;
    L.c = 0;
    L.tile = L.c + (size_t)kStages * Tile<NT>::kStageBytes;
    L.bar = L.tile + 2 * (size_t)kTileV * Tile<NT>::kRowBytes;   // Re and Im tiles
    L.tmem = L.bar + 8 * (size_t)(2 * kStages + 3);
    L.scale = (L.tmem + 16 + 15) & ~size_t(15);
    L.total = L.scale + 4 * (size_t)NT;
    return L;
}
// Dynamic shared memory requested per CTA: at least kTcSmemRequest, so that no CTA of another
// kernel that takes tensor memory (a projection) fits beside it and waits for the columns this
// CTA holds.
template <int NT>
inline size_t tc_smem_bytes() {
    const size_t need = 1024 + tc_layout<NT>().total;
    return need > kTcSmemRequest ? need : kTcSmemRequest;
}

// Named barrier among the producer threads (the epilogue phases).
__device__ __forceinline__ void epilogue_barrier() {
    asm volatile("bar.sync 1, %0;" ::"n"(kProducers) : "memory");
}

// 16 consecutive TMEM columns of this thread's lane <- r[0..15], and the wait for the store.
__device__ __forceinline__ void tmem_st16_wait(uint32_t t, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(t),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15])
        : "memory");
}

// Two 16-column TMEM loads of this thread's lane and the wait for them, in one statement.
__device__ __forceinline__ void tmem_ld16x2(uint32_t t0, uint32_t t1, float (&o0)[16],
                                            float (&o1)[16]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,"
        "%28,%29,%30,%31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(t0), "r"(t1)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        o0[i] = __uint_as_float(r[i]);
        o1[i] = __uint_as_float(r[16 + i]);
    }
}

template <int NT>
__device__ __forceinline__ void accumulate_stacked(const TcArgs& a, int bx, int by) {
    using TL = Tile<NT>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const TcLayout L = tc_layout<NT>();
    uint8_t* c_base = base + L.c;
    float* t_re = reinterpret_cast<float*>(base + L.tile);                     // [64][NT + 4]
    float* t_im = reinterpret_cast<float*>(base + L.tile + (size_t)kTileV * TL::kRowBytes);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + L.bar);   // stage filled (A and B)
    uint64_t* empty = full + kStages;                              // stage read by its MMAs
    uint64_t* dfull = empty + kStages;   // a segment's MMAs have completed (MMA warp -> epilogue)
    uint64_t* dfree = dfull + 1;         // the epilogue has read D (epilogue -> MMA warp)
    uint64_t* fin = dfree + 1;           // every issued MMA has completed (teardown)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.tmem);
    float* s_scale = reinterpret_cast<float*>(base + L.scale);
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int v0 = bx * kTileV;
    const int k0 = by * NT;
    const int T = a.stages_total;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], kProdWarps + 1);   // producer warps + the TMA arrival
            mbar_init(&empty[s], 1);
        }
        mbar_init(dfull, 1);
        mbar_init(dfree, kProdWarps);
        mbar_init(fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kProdWarps + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // The next launch may start now (this CTA holds its tensor memory): it waits
    // (griddepcontrol.wait) before touching anything this grid writes.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (warp < kProdWarps) {
        // ---------------- producers, and the epilogue between segments ---------------------
        const int quarter = warp & 3;
        const int ks = warp >> 2;                       // K-step of each stage this warp fills
        const bool imag = quarter >= 2;                 // rows 64-127: imaginary parts
        const int vi = (quarter & 1) * 32 + lane;       // frequency within the tile
        // Rows beyond S (last tile) generate v = 0; the epilogue never writes them.
        const int v = (v0 + vi < a.S) ? v0 + vi : 0;
        const uint32_t vy = (uint32_t)(v / a.Sh);
        const uint32_t vx = (uint32_t)(v % a.Sh);
        const uint32_t Sx = (uint32_t)a.Sx, my = (uint32_t)a.my, mx = (uint32_t)a.mx;
        const uint32_t lcm = (uint32_t)a.lcm;
        // w_v^j = exp(-2 pi i j vx / Sx), j = 0..8, from the table (index j vx mx mod lcm)
        float2 w[9];
        {
            const uint32_t d = vx * mx;   // < lcm
            uint32_t acc = 0;
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                w[j] = __ldg(a.tw + acc);
                acc += d;
                if (acc >= lcm) acc -= lcm;
            }
        }
        const uint32_t t_lane = tmem + ((uint32_t)(quarter * 32) << 16) +
                                (uint32_t)(TL::kColsD + ks * 16);
        // running sums of this thread's row (Re or Im of frequency vi) over the segments, for
        // coefficient columns cbase .. cbase + NT / 4 - 1 of the tile (FP32), kept in this
        // thread's part of the epilogue tile in shared memory: registers held across the stage
        // loop slow the producers (9-11 % per flush measured against register sums)
        const int cbase = ks * (NT / 4);
        float* srow = (imag ? t_im : t_re) + (size_t)vi * (TL::kRowBytes / 4) + cbase;
#pragma unroll
        for (int i = 0; i < NT / 4; i += 4)
            *reinterpret_cast<float4*>(srow + i) = make_float4(0.f, 0.f, 0.f, 0.f);
        // this warp's 16 frames of stage it form group 4 it + ks; the group records are written
        // by the split pre-pass.  Records run two stages ahead, the table entry of the group's
        // first position one stage ahead.
        const int2* gp = a.grp + ks;
        // phase-index step between a group and the group 64 positions further along the same
        // scan row: (64 vx mod Sx) mx mod lcm; when those 64 positions wrap into the next scan
        // row (raster order), the row step vy my is added as well
        const uint32_t d64 = fastmod(64u * vx, a.mod_x) * mx;   // < lcm
        const uint32_t dmy = vy * my;                           // < lcm (vy < S_y)
        int2 g0 = make_int2(0, 0), g1 = g0;
        uint32_t m0 = 0;
        float2 b0 = make_float2(1.f, 0.f);
        int ok = 1;   // warp-uniform: this warp has not given up
        int it = 0;
        for (int g = 0; g < a.segments; ++g) {
            const int it_end = (g + 1) * a.seg_stages < T ? (g + 1) * a.seg_stages : T;
            for (; it < it_end; ++it) {
                if (it == 0) {
                    // the records come from the split pre-pass, the launch before this one
                    asm volatile("griddepcontrol.wait;" ::: "memory");
                    g0 = __ldcg(gp);
                    if (T > 1) g1 = __ldcg(gp + kKSteps);
                    m0 = phase_index((uint32_t)g0.x, vy, vx, a.mod_y, a.mod_x, Sx, my, mx, lcm);
                    b0 = __ldg(a.tw + m0);
                }
                const int st = it & (kStages - 1);
                // prefetch: table entry of the next stage (its index one step along the row from
                // this one's in raster order), record of the one after
                float2 b1 = b0;
                uint32_t m1 = m0;
                int2 g2 = make_int2(0, 0);
                if (it + 1 < T) {
                    if (g1.x == g0.x + 64 && (g1.y >> 1) == (g0.y >> 1) + 64) {
                        m1 = m0 + d64;
                        if (m1 >= lcm) m1 -= lcm;
                    } else if (g1.x == g0.x + 64 && (g1.y >> 1) == (g0.y >> 1) + 64 - a.Sx) {
                        m1 = m0 + d64;
                        if (m1 >= lcm) m1 -= lcm;
                        m1 += dmy;
                        if (m1 >= lcm) m1 -= lcm;
                    } else {
                        m1 = phase_index((uint32_t)g1.x, vy, vx, a.mod_y, a.mod_x, Sx, my, mx, lcm);
                    }
                    b1 = __ldg(a.tw + m1);
                }
                if (it + 2 < T) g2 = __ldcg(gp + (size_t)(it + 2) * kKSteps);
                if (ok) {
                    int good = 1;
                    if (lane == 0) {
                        // the slot is free once the MMAs of stage it - 4 have completed
                        if (it >= kStages &&
                            !mbar_wait(&empty[st], ((it >> 2) - 1) & 1, a.wait_ns)) {
                            atomicExch(a.status, 1u);
                            s_abort = 1;
                        }
                        good = !s_abort;
                    }
                    ok = __shfl_sync(0xffffffffu, good, 0);
                }
                if (ok) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // Re or Im of the 16 phase factors, two halves of 8 frames
                    float x[16];
                    if (g0.y & 1) {
                        // consecutive positions of one scan row: E[v, s0] w^j, E[v, s0 + 8] w^j
                        const float2 b8 = make_float2(fmaf(b0.x, w[8].x, -b0.y * w[8].y),
                                                      fmaf(b0.x, w[8].y, b0.y * w[8].x));
                        if (imag) {
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                x[j] = fmaf(b0.x, w[j].y, b0.y * w[j].x);
                                x[8 + j] = fmaf(b8.x, w[j].y, b8.y * w[j].x);
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                x[j] = fmaf(b0.x, w[j].x, -b0.y * w[j].y);
                                x[8 + j] = fmaf(b8.x, w[j].x, -b8.y * w[j].y);
                            }
                        }
                    } else {
                        const int32_t* ip = a.idx + (size_t)it * kChunk + ks * 16;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float2 e = __ldg(a.tw + phase_index((uint32_t)__ldcg(ip + j), vy,
                                                                      vx, a.mod_y, a.mod_x, Sx, my,
                                                                      mx, lcm));
                            x[j] = imag ? e.y : e.x;
                        }
                    }
                    uint32_t r[16];   // hi part (8 frame pairs), then lo part
#pragma unroll
                    for (int c = 0; c < 8; ++c) split2(x[2 * c], x[2 * c + 1], r[c], r[8 + c]);
                    tmem_st16_wait(t_lane + (uint32_t)(st * 64), r);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full[st]);
                }
                g0 = g1; g1 = g2; b0 = b1; m0 = m1;
            }
            // ---------------- end of segment g: D is added into this thread's running sums ------
            int go = 0;
            if (ok) {
                int good = 1;
                if (lane == 0) {
                    good = mbar_wait(dfull, g & 1, a.wait_ns) ? 1 : 0;
                    if (!good) {
                        atomicExch(a.status, 4u);
                        s_abort = 1;
                    }
                    good = good && !s_abort;
                }
                go = __shfl_sync(0xffffffffu, good, 0);
                ok = go;
            }
            if (go) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
                for (int h = 0; h < NT / 64; ++h) {
                    const int c0 = cbase + 16 * h;
                    float hi[16], lo[16];
                    tmem_ld16x2(tl + (uint32_t)c0, tl + (uint32_t)(NT + c0), hi, lo);
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        float4 q = *reinterpret_cast<float4*>(srow + 16 * h + i);
                        q.x += hi[i] + lo[i];
                        q.y += hi[i + 1] + lo[i + 1];
                        q.z += hi[i + 2] + lo[i + 2];
                        q.w += hi[i + 3] + lo[i + 3];
                        *reinterpret_cast<float4*>(srow + 16 * h + i) = q;
                    }
                }
                // D has been read: the next segment's MMAs may overwrite it
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(dfree);
            }
        }
        // ---------------- epilogue: H[v, k] += sum / scale, once per flush ------------------
        // The scales come from the split pre-pass and H from the previous flush (both complete:
        // the producers passed griddepcontrol.wait at stage 0).
        for (int t = threadIdx.x; t < NT; t += kProducers) {
            const int k = k0 + t;
            s_scale[t] = (k < a.K) ? __ldcg(a.scale_inv + k) : 0.f;
        }
        epilogue_barrier();   // s_scale written, the tiles of running sums complete
        if (ok) {
            // warp w updates rows w, w + 16, w + 32, w + 48; lane l the coefficients l + 32 j
            constexpr int J = NT / 32;
            float2 hv[kTileV / kProdWarps][J];
#pragma unroll
            for (int i = 0; i < kTileV / kProdWarps; ++i) {
                const int vv = v0 + warp + kProdWarps * i;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int k = k0 + j * 32 + lane;
                    hv[i][j] = (vv < a.S && k < a.K) ? __ldcg(a.H + h_row(a, vv) * a.K + k)
                                                     : make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int i = 0; i < kTileV / kProdWarps; ++i) {
                const int vr = warp + kProdWarps * i;
                const int vv = v0 + vr;
                const float* rre = t_re + (size_t)vr * (TL::kRowBytes / 4);
                const float* rim = t_im + (size_t)vr * (TL::kRowBytes / 4);
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int kl = j * 32 + lane;
                    const int k = k0 + kl;
                    // (sum * scale) rounded, then added: no fused multiply-add
                    if (vv < a.S && k < a.K)
                        a.H[h_row(a, vv) * a.K + k] =
                            make_float2(__fadd_rn(hv[i][j].x, __fmul_rn(rre[kl], s_scale[kl])),
                                        __fadd_rn(hv[i][j].y, __fmul_rn(rim[kl], s_scale[kl])));
                }
            }
        }
    } else if (warp == kProdWarps) {
        // ---------------- B loader (TMA) ----------------
        if (lane == 0) {
            // the split coefficients come from the launch before (the split pre-pass)
            asm volatile("griddepcontrol.wait;" ::: "memory");
            const uint8_t* src = reinterpret_cast<const uint8_t*>(a.csplit) +
                                 (size_t)by * T * TL::kStageBytes;
            for (int it = 0; it < T; ++it) {
                const int st = it & (kStages - 1);
                if (it >= kStages && !mbar_wait(&empty[st], ((it >> 2) - 1) & 1, a.wait_ns)) {
                    atomicExch(a.status, 2u);
                    s_abort = 1;
                    break;
                }
                if (s_abort) break;
                mbar_arrive_tx(&full[st], TL::kStageBytes);
                tma_load_1d(c_base + (size_t)st * TL::kStageBytes,
                            src + (size_t)it * TL::kStageBytes, TL::kStageBytes, &full[st]);
            }
        }
    } else {
        // ---------------- MMA issuer: no division in this loop ----------------
        if (lane == 0) {
            const uint32_t id_full = instr_desc(128, 2 * NT);   // B = [c_hi | c_lo]
            const uint32_t id_hi = instr_desc(128, NT);         // B = c_hi
            const uint64_t dc0 = smem_desc(smem_u32(c_base), 128, 256);
            const int seg = a.seg_stages;
            int st = 0, seg_left = 0, g = 0;
            uint32_t ph = 0;
            for (int it = 0; it < T; ++it) {
                uint32_t acc = 1u;
                if (seg_left == 0) {
                    // a new segment: the epilogue must have read the previous one out of D
                    if (g > 0 && !mbar_wait(dfree, (uint32_t)(g - 1) & 1u, a.wait_ns)) {
                        atomicExch(a.status, 5u);
                        s_abort = 1;
                        break;
                    }
                    seg_left = seg;
                    acc = 0u;
                }
                if (!mbar_wait(&full[st], ph, a.wait_ns)) {
                    atomicExch(a.status, 3u);
                    s_abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t dbs = dc0 + (uint64_t)((st * TL::kStageBytes) >> 4);
                const uint32_t as = tmem + (uint32_t)(TL::kColsD + st * 64);
#pragma unroll
                for (int k2 = 0; k2 < kKSteps; ++k2) {
                    const uint64_t db = dbs + (uint64_t)((k2 * TL::kKStepBytes) >> 4);
                    const uint32_t a0 = as + (uint32_t)(k2 * 16);
                    mma_f16_ts(tmem, a0, db, id_full, k2 == 0 ? acc : 1u);   // A_hi [c_hi | c_lo]
                    mma_f16_ts(tmem, a0 + 8u, db, id_hi, 1u);                // A_lo c_hi
                }
                mma_commit(&empty[st]);   // frees the stage (A and B) once these MMAs have read it
                if (--seg_left == 0 || it + 1 == T) {
                    mma_commit(dfull);
                    ++g;
                    seg_left = 0;
                }
                st = (st + 1) & (kStages - 1);
                ph ^= (st == 0) ? 1u : 0u;
            }
            // teardown: every MMA issued above completes before TMEM is freed
            mma_commit(fin);
            if (!mbar_wait(fin, 0, a.wait_ns)) atomicExch(a.status, 6u);
        }
    }

    // column maxima for the next flush: reset by the producer warps, which have passed
    // griddepcontrol.wait, i.e. after the split pre-pass has read them
    if (bx == 0 && by == 0 && warp < kProdWarps)
        for (int t = threadIdx.x; t < a.K; t += kProducers) a.colmax[t] = 0u;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kProdWarps + 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
    }
}

template <int NT>
__global__ void __launch_bounds__(kThreadsTC, 1) accumulate_tc_kernel(const TcArgs a) {
    accumulate_stacked<NT>(a, blockIdx.x, blockIdx.y);
}

// ---- K <= 64: 128 frequencies x 64 coefficients per CTA ----------------------------------------
// For K <= 64 a CTA keeps 128 frequencies in the MMA rows and the real and imaginary parts in two
// accumulators instead: D_re = Re E [c_hi | c_lo] (TMEM columns 0-127), D_im = Im E [...]
// (128-255), four MMAs per K-step, two A slots of 128 columns at 256-511 (slot a, K-step ks, part
// p of Re_hi, Re_lo, Im_hi, Im_lo: column 256 + 128 a + 32 ks + 8 p).  With 64 coefficients this
// halves the CTAs (and their per-stage costs) for the same work; the stacked layout above only
// pays off when the generated values feed N = 256 MMAs.
constexpr int kNarrowV = 128;
constexpr int kNarrowK = 64;
constexpr int kNarrowColsD = 256;
constexpr int kSlotsA = 2;
constexpr int kNarrowStride = kNarrowK * 8 + 16;   // epilogue tile row: 64 float2 + 16 B pad

__host__ __device__ inline TcLayout narrow_layout() {
    TcLayout L;
    L.c = 0;
    L.tile = L.c + (size_t)kStages * Tile<64>::kStageBytes;
    L.bar = L.tile + (size_t)kNarrowV * kNarrowStride;
    L.tmem = L.bar + 8 * (size_t)(2 * kStages + 3);
    L.scale = (L.tmem + 16 + 15) & ~size_t(15);
    L.total = L.scale + 4 * (size_t)kNarrowK;
    return L;
}
inline size_t narrow_smem_bytes() {
    const size_t need = 1024 + narrow_layout().total;
    return need > kTcSmemRequest ? need : kTcSmemRequest;
}

// Four 4-column TMEM stores of this thread's lane (parts p at t + 8 p) and the wait for them.
__device__ __forceinline__ void tmem_st4x4_wait(uint32_t t, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%5], {%6,%7,%8,%9};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%10], {%11,%12,%13,%14};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%15], {%16,%17,%18,%19};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(t),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(t + 8u), "r"(r[4]), "r"(r[5]), "r"(r[6]),
        "r"(r[7]), "r"(t + 16u), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(t + 24u),
        "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

// Four 16-column TMEM loads of this thread's lane and the wait for them, in one statement.
__device__ __forceinline__ void tmem_ld16x4(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3,
                                            float (&o0)[16], float (&o1)[16], float (&o2)[16],
                                            float (&o3)[16]) {
    tmem_ld16x2(t0, t1, o0, o1);
    tmem_ld16x2(t2, t3, o2, o3);
}

__device__ __forceinline__ void accumulate_narrow(const TcArgs& a, int bx, int by) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const TcLayout L = narrow_layout();
    uint8_t* c_base = base + L.c;
    uint8_t* tile = base + L.tile;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + L.bar);   // stage filled (A and B)
    uint64_t* empty = full + kStages;                             // stage read by its MMAs
    uint64_t* dfull = empty + kStages;  // a segment's MMAs have completed (MMA warp -> epilogue)
    uint64_t* dfree = dfull + 1;         // the epilogue has read D (epilogue -> MMA warp)
    uint64_t* fin = dfree + 1;           // every issued MMA has completed (teardown)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.tmem);
    float* s_scale = reinterpret_cast<float*>(base + L.scale);
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int v0 = bx * kNarrowV;
    const int k0 = by * kNarrowK;
    const int T = a.stages_total;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], kProdWarps + 1);   // producer warps + the TMA arrival
            mbar_init(&empty[s], 1);
        }
        mbar_init(dfull, 1);
        mbar_init(dfree, kProdWarps);
        mbar_init(fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kProdWarps + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // The next launch may start now (this CTA holds its tensor memory): it waits
    // (griddepcontrol.wait) before touching anything this grid writes.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (warp < kProdWarps) {
        // ---------------- E producers, and the epilogue between segments ------------------
        const int quarter = warp & 3;
        const int ks = warp >> 2;                       // K-step of each stage this warp fills
        const int row = quarter * 32 + lane;            // TMEM lane = frequency in the tile
        // Rows beyond S (last tile) generate v = 0; the epilogue never writes them.
        const int v = (v0 + row < a.S) ? v0 + row : 0;
        const uint32_t vy = (uint32_t)(v / a.Sh);
        const uint32_t vx = (uint32_t)(v % a.Sh);
        const uint32_t Sx = (uint32_t)a.Sx, my = (uint32_t)a.my, mx = (uint32_t)a.mx;
        const uint32_t lcm = (uint32_t)a.lcm;
        // w_v^j = exp(-2 pi i j vx / Sx), j = 0..8, from the table (index j vx mx mod lcm)
        float2 w[9];
        {
            const uint32_t d = vx * mx;   // < lcm
            uint32_t acc = 0;
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                w[j] = __ldg(a.tw + acc);
                acc += d;
                if (acc >= lcm) acc -= lcm;
            }
        }
        const uint32_t t_lane = tmem + ((uint32_t)(quarter * 32) << 16) +
                                (uint32_t)(kNarrowColsD + ks * 32);
        // this warp's 16 frames of stage it form group 4 it + ks; the group records are written
        // by the split pre-pass.  Records run two stages ahead, the table entry of the group's
        // first position one stage ahead.
        const int2* gp = a.grp + ks;
        int2 g0 = make_int2(0, 0), g1 = g0;
        float2 b0 = make_float2(1.f, 0.f);
        int ok = 1;   // warp-uniform: this warp has not given up
        int it = 0;
        for (int g = 0; g < a.segments; ++g) {
            const int it_end = (g + 1) * a.seg_stages < T ? (g + 1) * a.seg_stages : T;
            for (; it < it_end; ++it) {
                if (it == 0) {
                    // the records come from the split pre-pass, the launch before this one
                    asm volatile("griddepcontrol.wait;" ::: "memory");
                    g0 = __ldcg(gp);
                    if (T > 1) g1 = __ldcg(gp + kKSteps);
                    b0 = __ldg(a.tw + phase_index((uint32_t)g0.x, vy, vx, a.mod_y, a.mod_x, Sx,
                                                  my, mx, lcm));
                }
                const int slot = it & (kSlotsA - 1);
                // prefetch: table entry of the next stage, record of the one after
                float2 b1 = b0;
                int2 g2 = make_int2(0, 0);
                if (it + 1 < T)
                    b1 = __ldg(a.tw + phase_index((uint32_t)g1.x, vy, vx, a.mod_y, a.mod_x, Sx, my,
                                                  mx, lcm));
                if (it + 2 < T) g2 = __ldcg(gp + (size_t)(it + 2) * kKSteps);
                if (ok) {
                    int good = 1;
                    if (lane == 0) {
                        // the A slot is free once the MMAs of stage it - 2 have completed
                        if (it >= kSlotsA &&
                            !mbar_wait(&empty[(it - 2) & (kStages - 1)], ((it - 2) >> 2) & 1,
                                       a.wait_ns)) {
                            atomicExch(a.status, 1u);
                            s_abort = 1;
                        }
                        good = !s_abort;
                    }
                    ok = __shfl_sync(0xffffffffu, good, 0);
                }
                if (ok) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t tcol = t_lane + (uint32_t)(slot * 128);
                    // two halves of 8 frames: phase factors, FP16 split, four 4-column stores
                    float2 bh = b0;                                   // E[v, s0 + 8 hf]
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        float2 e[8];
                        if (g0.y & 1) {
                            // consecutive positions of one scan row: E[v, s0] w^j
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                e[j] = make_float2(fmaf(bh.x, w[j].x, -bh.y * w[j].y),
                                                   fmaf(bh.x, w[j].y, bh.y * w[j].x));
                        } else {
                            const int32_t* ip = a.idx + (size_t)it * kChunk + ks * 16 + hf * 8;
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                e[j] = __ldg(a.tw + phase_index((uint32_t)__ldcg(ip + j), vy, vx,
                                                                a.mod_y, a.mod_x, Sx, my, mx, lcm));
                        }
                        uint32_t r[16];   // parts Re_hi, Re_lo, Im_hi, Im_lo: 4 frame pairs each
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            split2(e[2 * c].x, e[2 * c + 1].x, r[c], r[4 + c]);
                            split2(e[2 * c].y, e[2 * c + 1].y, r[8 + c], r[12 + c]);
                        }
                        tmem_st4x4_wait(tcol + (uint32_t)(hf * 4), r);
                        bh = make_float2(fmaf(b0.x, w[8].x, -b0.y * w[8].y),
                                         fmaf(b0.x, w[8].y, b0.y * w[8].x));
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full[it & (kStages - 1)]);
                }
                g0 = g1; g1 = g2; b0 = b1;
            }
            // ---------------- epilogue of segment g: H[v, k] += (D[k] + D[64 + k]) / scale ----
            // The scales come from the split pre-pass and H from the previous flush: wait for
            // the launch before this one (a no-op after the first time).
            asm volatile("griddepcontrol.wait;" ::: "memory");
            if (g == 0)
                for (int t = threadIdx.x; t < kNarrowK; t += kProducers) {
                    const int k = k0 + t;
                    s_scale[t] = (k < a.K) ? __ldcg(a.scale_inv + k) : 0.f;
                }
            int go = 0;
            if (ok) {
                int good = 1;
                if (lane == 0) {
                    good = mbar_wait(dfull, g & 1, a.wait_ns) ? 1 : 0;
                    if (!good) {
                        atomicExch(a.status, 4u);
                        s_abort = 1;
                    }
                    good = good && !s_abort;
                }
                go = __shfl_sync(0xffffffffu, good, 0);
                ok = go;
            }
            epilogue_barrier();   // s_scale written; the tile is free
            if (go) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
                float2* trow = reinterpret_cast<float2*>(tile + (size_t)row * kNarrowStride);
                const int c0 = (warp >> 2) * 16;   // this warp's 16 coefficient columns
                float rh[16], rl[16], ih[16], il[16];
                tmem_ld16x4(tl + (uint32_t)c0, tl + (uint32_t)(64 + c0), tl + (uint32_t)(128 + c0),
                            tl + (uint32_t)(192 + c0), rh, rl, ih, il);
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const float s0v = s_scale[c0 + i], s1v = s_scale[c0 + i + 1];
                    *reinterpret_cast<float4*>(trow + c0 + i) =
                        make_float4((rh[i] + rl[i]) * s0v, (ih[i] + il[i]) * s0v,
                                    (rh[i + 1] + rl[i + 1]) * s1v, (ih[i + 1] + il[i + 1]) * s1v);
                }
                // D has been read: the next segment's MMAs may overwrite it
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(dfree);
            }
            epilogue_barrier();   // the tile is complete
            if (go) {
                // warp w updates tile rows w, w + 16, ...; lane l the coefficients l and l + 32;
                // the H values of four rows are loaded before any is stored
#pragma unroll
                for (int i0 = 0; i0 < kNarrowV / kProdWarps; i0 += 4) {
                    float2 hv[4][2];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int vv = v0 + warp + kProdWarps * (i0 + i);
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const int k = k0 + hh * 32 + lane;
                            hv[i][hh] = (vv < a.S && k < a.K) ? __ldcg(a.H + h_row(a, vv) * a.K + k)
                                                              : make_float2(0.f, 0.f);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int vr = warp + kProdWarps * (i0 + i);
                        const int vv = v0 + vr;
                        const float2* trow =
                            reinterpret_cast<const float2*>(tile + (size_t)vr * kNarrowStride);
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const int kl = hh * 32 + lane;
                            const int k = k0 + kl;
                            if (vv < a.S && k < a.K) {
                                const float2 x = trow[kl];
                                a.H[h_row(a, vv) * a.K + k] =
                                    make_float2(hv[i][hh].x + x.x, hv[i][hh].y + x.y);
                            }
                        }
                    }
                }
            }
        }
    } else if (warp == kProdWarps) {
        // ---------------- B loader (TMA) ----------------
        if (lane == 0) {
            // the split coefficients come from the launch before (the split pre-pass)
            asm volatile("griddepcontrol.wait;" ::: "memory");
            const uint8_t* src = reinterpret_cast<const uint8_t*>(a.csplit) +
                                 (size_t)by * T * Tile<64>::kStageBytes;
            for (int it = 0; it < T; ++it) {
                const int st = it & (kStages - 1);
                if (it >= kStages && !mbar_wait(&empty[st], ((it >> 2) - 1) & 1, a.wait_ns)) {
                    atomicExch(a.status, 2u);
                    s_abort = 1;
                    break;
                }
                if (s_abort) break;
                mbar_arrive_tx(&full[st], Tile<64>::kStageBytes);
                tma_load_1d(c_base + (size_t)st * Tile<64>::kStageBytes, src + (size_t)it * Tile<64>::kStageBytes,
                            Tile<64>::kStageBytes, &full[st]);
            }
        }
    } else {
        // ---------------- MMA issuer: no division in this loop ----------------
        if (lane == 0) {
            const uint32_t id_full = instr_desc(128, 2 * kNarrowK);   // B = [c_hi | c_lo]
            const uint32_t id_hi = instr_desc(128, kNarrowK);         // B = c_hi
            const uint64_t dc0 = smem_desc(smem_u32(c_base), 128, 256);
            const uint32_t d_re = tmem, d_im = tmem + 128u;
            const int seg = a.seg_stages;
            int st = 0, seg_left = 0, g = 0;
            uint32_t ph = 0;
            for (int it = 0; it < T; ++it) {
                uint32_t acc = 1u;
                if (seg_left == 0) {
                    // a new segment: the epilogue must have read the previous one out of D
                    if (g > 0 && !mbar_wait(dfree, (uint32_t)(g - 1) & 1u, a.wait_ns)) {
                        atomicExch(a.status, 5u);
                        s_abort = 1;
                        break;
                    }
                    seg_left = seg;
                    acc = 0u;
                }
                if (!mbar_wait(&full[st], ph, a.wait_ns)) {
                    atomicExch(a.status, 3u);
                    s_abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t dbs = dc0 + (uint64_t)((st * Tile<64>::kStageBytes) >> 4);
                const uint32_t as = tmem + (uint32_t)(kNarrowColsD + (it & (kSlotsA - 1)) * 128);
#pragma unroll
                for (int k2 = 0; k2 < kKSteps; ++k2) {
                    const uint64_t db = dbs + (uint64_t)((k2 * Tile<64>::kKStepBytes) >> 4);
                    const uint32_t a0 = as + (uint32_t)(k2 * 32);
                    const uint32_t ac = k2 == 0 ? acc : 1u;
                    mma_f16_ts(d_re, a0, db, id_full, ac);           // Re_hi [c_hi | c_lo]
                    mma_f16_ts(d_im, a0 + 16u, db, id_full, ac);     // Im_hi [c_hi | c_lo]
                    mma_f16_ts(d_re, a0 + 8u, db, id_hi, 1u);        // Re_lo c_hi
                    mma_f16_ts(d_im, a0 + 24u, db, id_hi, 1u);       // Im_lo c_hi
                }
                mma_commit(&empty[st]);   // frees the stage (A and B) once these MMAs have read it
                if (--seg_left == 0 || it + 1 == T) {
                    mma_commit(dfull);
                    ++g;
                    seg_left = 0;
                }
                st = (st + 1) & (kStages - 1);
                ph ^= (st == 0) ? 1u : 0u;
            }
            // teardown: every MMA issued above completes before TMEM is freed
            mma_commit(fin);
            if (!mbar_wait(fin, 0, a.wait_ns)) atomicExch(a.status, 6u);
        }
    }

    // column maxima for the next flush: reset by the producer warps, which have passed
    // griddepcontrol.wait, i.e. after the split pre-pass has read them
    if (bx == 0 && by == 0 && warp < kProdWarps)
        for (int t = threadIdx.x; t < a.K; t += kProducers) a.colmax[t] = 0u;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kProdWarps + 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
    }
}

__global__ void __launch_bounds__(kThreadsTC, 1) accumulate_narrow_kernel(const TcArgs a) {
    accumulate_narrow(a, blockIdx.x, blockIdx.y);
}

// ---- several plans in one launch (wdd_flush_group) -----------------------------------------------
// The CTAs of plan j are the linear block indices first[j] .. first[j + 1] - 1 (its (v, k) tiles in
// the order of the single-plan grid, x fastest); each CTA runs exactly the single-plan kernel on
// its plan's arguments.
constexpr int kMaxGroup = 8;
struct TcGroup {
    TcArgs args[kMaxGroup];
    int first[kMaxGroup + 1];
    int xtiles[kMaxGroup];
    int kind[kMaxGroup];       // TcKind of each member
    int n;
};

__device__ __forceinline__ int group_member(const TcGroup& g, int b) {
    int j = 0;
    while (j + 1 < g.n && b >= g.first[j + 1]) ++j;
    return j;
}

// One launch for every member: a CTA runs the 128-frequency body for a member with K <= 64 and
// the stacked body otherwise (both need one CTA per SM and the same warp roles).
__global__ void __launch_bounds__(kThreadsTC, 1) accumulate_group_kernel(const TcGroup g) {
    const int j = group_member(g, blockIdx.x);
    const int local = blockIdx.x - g.first[j];
    if (g.kind[j] == 0)
        accumulate_narrow(g.args[j], local % g.xtiles[j], local / g.xtiles[j]);
    else if (g.kind[j] == 2)
        accumulate_stacked<64>(g.args[j], local % g.xtiles[j], local / g.xtiles[j]);
    else
        accumulate_stacked<128>(g.args[j], local % g.xtiles[j], local / g.xtiles[j]);
}

// Splits the staged FP32 coefficients into FP16 hi/lo parts with a power-of-two scale per column
// and writes them as the B operand of accumulate_tc_kernel<NT>, K-major core matrices:
//   [k-tile of NT][K-step of 16 frames][row group][core matrix b/8 % 2][row % 8][b % 8]
// where rows 0 .. NT-1 of a k-tile hold its coefficients' hi parts and rows NT .. 2NT-1 their lo
// parts (four consecutive K-steps form a 64-frame stage).  Frames beyond n and coefficients
// beyond K are zero.  One thread per (frame, column).  The thread of column 0 of every 16th frame
// also writes that 16-frame group's record.
struct SplitArgs {
    const float* c;
    const unsigned* colmax;
    uint16_t* out;
    float* scale_inv;
    const int32_t* idx;
    int2* grp;
    int n, n_pad, K, Kp, NT, Sx;
};

__device__ __forceinline__ void split_coeff(const SplitArgs& s, int t) {
    const float* __restrict__ c = s.c;
    const unsigned* __restrict__ colmax = s.colmax;
    uint16_t* __restrict__ out = s.out;
    float* __restrict__ scale_inv = s.scale_inv;
    const int32_t* __restrict__ idx = s.idx;
    int2* __restrict__ grp = s.grp;
    const int n = s.n, n_pad = s.n_pad, K = s.K, Kp = s.Kp, NT = s.NT, Sx = s.Sx;
    const int kk = t % Kp;
    const int b = t / Kp;
    if (b >= n_pad) return;
    if (kk == 0 && (b & 15) == 0) {
        // group record: first scan index, and whether the 16 frames are consecutive positions
        // of one scan row (frames beyond n have zero coefficients: any record serves them)
        const int32_t s0 = idx[b];
        const int32_t sx0 = s0 >= 0 ? s0 % Sx : 0;
        bool run = s0 >= 0 && sx0 + 15 < Sx;
        for (int j = 1; j < 16 && run; ++j) run = idx[b + j] == s0 + j;
        grp[b >> 4] = make_int2(s0, (run ? 1 : 0) | (sx0 << 1));
    }
    float cm = (kk < K) ? __uint_as_float(colmax[kk]) : 0.f;
    int e = 0;
    if (cm > 0.f) frexpf(cm, &e);
    const float sc = (cm > 0.f) ? ldexpf(1.f, 14 - e) : 1.f;
    if (b == 0) scale_inv[kk] = (kk < K && cm > 0.f) ? ldexpf(1.f, e - 14) : 0.f;
    const float x = (b < n && kk < K) ? c[(size_t)b * K + kk] * sc : 0.f;
    const __half hi = __float2half_rn(x);
    const __half lo = __float2half_rn(x - __half2float(hi));
    const int ktile = kk / NT, km = kk % NT;
    const int kstep = b >> 4, bk = b & 15;
    const int ksteps_total = n_pad >> 4;
    const size_t base = ((size_t)ktile * ksteps_total + kstep) * (size_t)(2 * NT * 16);
    const int rh = km, rl = NT + km;
    const size_t in_hi = (size_t)(rh >> 3) * 128 + (size_t)(bk >> 3) * 64 + (size_t)(rh & 7) * 8 + (bk & 7);
    const size_t in_lo = (size_t)(rl >> 3) * 128 + (size_t)(bk >> 3) * 64 + (size_t)(rl & 7) * 8 + (bk & 7);
    out[base + in_hi] = __half_as_ushort(hi);
    out[base + in_lo] = __half_as_ushort(lo);
}

__global__ void split_coeff_kernel(const SplitArgs s) {
    // the accumulation launched next sets up meanwhile; it reads this kernel's outputs only after
    // griddepcontrol.wait.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    split_coeff(s, blockIdx.x * blockDim.x + threadIdx.x);
}

// The split pre-pass of several plans: plan j takes threads first[j] .. first[j + 1] - 1.
struct SplitGroup {
    SplitArgs args[kMaxGroup];
    long long first[kMaxGroup + 1];
    int n;
};

__global__ void split_coeff_group_kernel(const SplitGroup g) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int j = 0;
    while (j + 1 < g.n && t >= g.first[j + 1]) ++j;
    if (t >= g.first[g.n]) return;
    split_coeff(g.args[j], (int)(t - g.first[j]));
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
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(accumulate_narrow_kernel));
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(accumulate_tc_kernel<128>));
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(accumulate_tc_kernel<64>));
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(accumulate_group_kernel));
    return e;
}

// Coefficients per CTA: 64 up to K = 64, else 128.
int split_tile_n(int K) { return K <= 64 ? 64 : 128; }

size_t split_smem_bytes(int NT) {
    if (NT != 64) return tc_smem_bytes<128>();
    return narrow_smem_bytes() > tc_smem_bytes<64>() ? narrow_smem_bytes() : tc_smem_bytes<64>();
}

int spectrum_cols(int Sx) { return Sx > 2 ? Sx / 2 + 1 : Sx; }

// Kernel launches of one flush: the split pre-pass and the accumulation.
int split_launch_count(int /*n*/, int /*segment*/) { return 2; }

size_t split_coeff_bytes(int K, int depth_pad) {
    const int NT = split_tile_n(K);
    const int Kp = (K + NT - 1) / NT * NT;
    return (size_t)Kp * depth_pad * 2 * 2;   // hi and lo halves
}

namespace {

SplitArgs make_split_args(const wdd_plan* P, const float* c, const int32_t* idx, int n,
                          long long* threads) {
    const int NT = split_tile_n(P->K);
    const int Kp = (P->K + NT - 1) / NT * NT;
    const int n_pad = (n + kChunk - 1) / kChunk * kChunk;
    SplitArgs s;
    s.c = c;
    s.colmax = P->d_colmax;
    s.out = reinterpret_cast<uint16_t*>(P->d_bsplit);
    s.scale_inv = P->d_scale_inv;
    s.idx = idx;
    s.grp = P->d_grp;
    s.n = n;
    s.n_pad = n_pad;
    s.K = P->K;
    s.Kp = Kp;
    s.NT = NT;
    s.Sx = P->Sx;
    *threads = (long long)n_pad * Kp;
    return s;
}

// Accumulation kernels: the 128-frequency kernel (K <= 64), the stacked kernel with 128 or 64
// coefficients per CTA.
enum TcKind { kNarrow = 0, kStacked128 = 1, kStacked64 = 2 };

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 148;
    return sms;
}

// Accumulation arguments of one plan, its grid (x: frequency tiles, y: coefficient tiles) and
// kernel.  Only the scan columns 0 .. S_x / 2 are accumulated (the rest follow from Hermitian
// symmetry, mirror_h_kernel).  For K <= 64 the 128-frequency kernel does the most work per
// generated phase factor, but when its tiles cannot fill the SMs once the 64-frequency stacked
// kernel, with twice the CTAs, finishes sooner.
TcArgs make_tc_args(const wdd_plan* P, const int32_t* idx, int n, dim3* grid, int* kind) {
    const int NT = split_tile_n(P->K);
    const int Kp = (P->K + NT - 1) / NT * NT;
    const int n_pad = (n + kChunk - 1) / kChunk * kChunk;
    TcArgs a;
    a.csplit = reinterpret_cast<const uint16_t*>(P->d_bsplit);
    a.scale_inv = P->d_scale_inv;
    a.colmax = P->d_colmax;
    a.idx = idx;
    a.grp = P->d_grp;
    a.tw = P->d_tw;
    a.H = P->d_H;
    a.status = P->d_status;
    a.Sh = spectrum_cols(P->Sx);
    a.S = P->Sy * a.Sh;
    a.K = P->K;
    a.Sx = P->Sx;
    a.Sy = P->Sy;
    a.lcm = P->lcm;
    a.my = P->lcm / P->Sy;
    a.mx = P->lcm / P->Sx;
    a.stages_total = n_pad / kChunk;
    a.seg_stages = P->segment / kChunk > 0 ? P->segment / kChunk : 1;
    a.segments = (a.stages_total + a.seg_stages - 1) / a.seg_stages;
    a.wait_ns = kDeviceWaitNs;
    a.mod_y = make_fastmod((uint32_t)P->Sy);
    a.mod_x = make_fastmod((uint32_t)P->Sx);
    if (NT != 64) {
        *kind = kStacked128;
        *grid = dim3((a.S + kTileV - 1) / kTileV, Kp / NT);
    } else if ((a.S + kNarrowV - 1) / kNarrowV >= sm_count()) {
        *kind = kNarrow;
        *grid = dim3((a.S + kNarrowV - 1) / kNarrowV, 1);
    } else {
        *kind = kStacked64;
        *grid = dim3((a.S + kTileV - 1) / kTileV, 1);
    }
    return a;
}

// The accumulation overlaps the split pre-pass (programmatic dependent launch): it allocates
// tensor memory and reads the phase table meanwhile, and reads the group records, the split
// coefficients, the scales and H only after griddepcontrol.wait.
template <typename Kern, typename Arg>
cudaError_t launch_dependent(Kern kern, const Arg& arg, dim3 grid, size_t smem, cudaStream_t st) {
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
    return cudaLaunchKernelEx(&cfg, kern, arg);
}

}  // namespace

cudaError_t launch_accumulate_split(const wdd_plan* P, const float* c, const int32_t* idx, int n,
                                    cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int n_pad = (n + kChunk - 1) / kChunk * kChunk;
    if (n_pad > P->depth_pad) return cudaErrorInvalidValue;
    // 1. split the coefficients (per-column scale from the projection's running max) and mark
    //    the 16-frame groups
    long long total = 0;
    const SplitArgs sa = make_split_args(P, c, idx, n, &total);
    split_coeff_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(sa);
    // 2. tensor-core accumulation of every staged frame, in TMEM segments of P->segment frames
    dim3 grid;
    int kind = kNarrow;
    const TcArgs a = make_tc_args(P, idx, n, &grid, &kind);
    cudaError_t e =
        kind == kNarrow ? launch_dependent(accumulate_narrow_kernel, a, grid, narrow_smem_bytes(), st)
        : kind == kStacked64
            ? launch_dependent(accumulate_tc_kernel<64>, a, grid, tc_smem_bytes<64>(), st)
            : launch_dependent(accumulate_tc_kernel<128>, a, grid, tc_smem_bytes<128>(), st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// H[v] = conj(H[-v]) for the scan columns S_x / 2 + 1 .. S_x - 1, whose mirror columns
// S_x - v_x lie in the accumulated half: with real coefficients the spectrum of Eq. 14 is
// Hermitian, H[-v, k] = sum_s conj(E[v, s]) c_s[k] = conj(H[v, k]).
__global__ void mirror_h_kernel(float2* H, int Sy, int Sx, int Sh, int K) {
    const int W = Sx - Sh;
    const long long n = (long long)Sy * W * K;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t % K);
        const long long r = t / K;
        const int vy = (int)(r / W), vx = Sh + (int)(r % W);
        const int my = vy == 0 ? 0 : Sy - vy, mx = Sx - vx;
        const float2 h = __ldcg(H + ((size_t)my * Sx + mx) * K + k);
        H[((size_t)vy * Sx + vx) * K + k] = make_float2(h.x, -h.y);
    }
}

int accum_kernel_of(const wdd_plan* P) {
    if (P->p.accum_mode == WDD_ACCUM_SEPARABLE) return WDD_ACCUM_KERNEL_SEPARABLE;
    if (P->p.precision != WDD_PREC_SPLIT) return WDD_ACCUM_KERNEL_FP32;
    dim3 grid;
    int kind = kNarrow;
    (void)make_tc_args(P, nullptr, kChunk, &grid, &kind);
    return kind == kNarrow ? WDD_ACCUM_KERNEL_NARROW
           : kind == kStacked64 ? WDD_ACCUM_KERNEL_STACKED64 : WDD_ACCUM_KERNEL_STACKED128;
}

bool mirror_needed(const wdd_plan* P) {
    return P->p.precision == WDD_PREC_SPLIT && P->p.accum_mode == WDD_ACCUM_DIRECT &&
           spectrum_cols(P->Sx) < P->Sx;
}

cudaError_t launch_mirror_h(const wdd_plan* P, cudaStream_t st) {
    const int Sh = spectrum_cols(P->Sx);
    const long long n = (long long)P->Sy * (P->Sx - Sh) * P->K;
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    mirror_h_kernel<<<(unsigned)blocks, 256, 0, st>>>(P->d_H, P->Sy, P->Sx, Sh, P->K);
    return cudaGetLastError();
}

int accumulate_group_max() { return kMaxGroup; }

cudaError_t launch_accumulate_group(wdd_plan* const* plans, int count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (count > kMaxGroup) return cudaErrorInvalidValue;
    SplitGroup sg{};
    TcGroup tg{};
    long long threads = 0;
    int ctas = 0;
    for (int j = 0; j < count; ++j) {
        const wdd_plan* P = plans[j];
        const int n = P->staged;
        long long t = 0;
        sg.args[j] = make_split_args(P, P->d_cstage, P->d_idxstage, n, &t);
        sg.first[j] = threads;
        threads += t;
        dim3 grid;
        int kind = kNarrow;
        tg.args[j] = make_tc_args(P, P->d_idxstage, n, &grid, &kind);
        tg.first[j] = ctas;
        tg.xtiles[j] = (int)grid.x;
        tg.kind[j] = kind;
        ctas += (int)(grid.x * grid.y);
    }
    sg.first[count] = threads;
    sg.n = count;
    tg.first[count] = ctas;
    tg.n = count;
    split_coeff_group_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(sg);
    const size_t smem = split_smem_bytes(64) > split_smem_bytes(128) ? split_smem_bytes(64)
                                                                     : split_smem_bytes(128);   // every kind fits
    cudaError_t e = launch_dependent(accumulate_group_kernel, tg, dim3((unsigned)ctas, 1, 1), smem, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace wdd
