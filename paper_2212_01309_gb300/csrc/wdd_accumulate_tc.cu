// Phase accumulation on the 5th-generation tensor cores (tcgen05, TMEM), split FP16 precision:
//   H[v, k] += sum_b E[v, s_b] c_b[k],  E = exp(-2 pi i m / lcm)  (Eq. outer_prod, Algorithm 2)
//
// Real form: D_re = Re(E) C and D_im = Im(E) C with one shared B operand C (frames x K).  Each
// operand is split into FP16 hi + lo parts and three products are accumulated in FP32 TMEM:
//   D = E_hi c_hi + E_lo c_hi + E_hi c_lo      (the dropped E_lo c_lo is ~2^-22 relative).
// The coefficients are scaled per column by a power of two before the split so that every
// column uses the FP16 range fully; the epilogue divides the scale out.
//
// Kernel structure (one CTA per 128 scan frequencies x NT coefficients):
//   warps 0-7  build the A operands (Re/Im, hi/lo of E) for their rows in shared memory, in the
//              no-swizzle K-major core-matrix layout, from the exact integer phase index and an
//              FP64-built table; warps 0-3 then run the epilogue (tcgen05.ld -> H += D / scale).
//   warp 8     streams the B operand (hi/lo coefficients, pre-arranged in the same layout by
//              split_coeff_kernel) into shared memory with 1-D TMA bulk copies.
//   warp 9     allocates TMEM and one elected lane issues tcgen05.mma; tcgen05.commit frees
//              each pipeline stage and finally signals the epilogue.
// Every mbarrier wait is bounded; a wait that runs out records an error code in *status and the
// CTA leaves the pipeline (after a bounded wait for its issued MMAs) and frees its TMEM.

#include <cuda_fp16.h>

#include "wdd_device.cuh"
#include "wdd_internal.h"

namespace wdd {

namespace {

constexpr int kTileM = 128;        // scan frequencies per CTA (UMMA M)
constexpr int kChunk = 32;         // frames per pipeline stage (two UMMA K-steps of 16)
constexpr int kProducers = 256;    // warps 0-7
constexpr int kThreadsTC = 320;    // + TMA warp + MMA warp
constexpr int kStages = 3;

// Bytes of one operand tile for one stage: kChunk/16 K-steps of 128 rows x 16 frames (FP16).
constexpr int kATileBytes = kTileM * kChunk * 2;   // 8 KB

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
    const uint32_t* bsplit;   // pre-arranged B operand (see split_coeff_kernel)
    const float* scale_inv;   // [Kp] 1 / column scale
    unsigned* colmax;         // [K] per-column max |c| (reset here for the next flush)
    const int32_t* idx;       // [n] scan index of each staged frame
    const uint2* tw16;        // [lcm] (re_hi | re_lo << 16, im_hi | im_lo << 16)
    float2* H;                // [S][K]
    unsigned* status;         // error word (0 = ok)
    int n_pad, S, K, NT, Sy, Sx, lcm, my, mx, stages_total, tmem_cols, tab_in_smem;
    uint64_t wait_ns;
    FastMod mod_y, mod_x;
};

__global__ void __launch_bounds__(kThreadsTC, 1) accumulate_tc_kernel(const TcArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned carve-up
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NT = a.NT;
    const int bTileBytes = NT * kChunk * 2;          // one hi or lo B tile per stage
    const int stageBytes = 4 * kATileBytes + 2 * bTileBytes;
    uint8_t* stage_base = base;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + kStages * stageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    float* s_scale = reinterpret_cast<float*>(tmem_slot + 4);   // [NT]
    uint2* s_tab = reinterpret_cast<uint2*>(
        (reinterpret_cast<uintptr_t>(s_scale + NT) + 15) & ~uintptr_t(15));   // [lcm] if it fits
    const uint2* tab = a.tab_in_smem ? s_tab : a.tw16;
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int v0 = blockIdx.x * kTileM;
    const int k0 = blockIdx.y * NT;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], kProducers + 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
        int k = k0 + t;
        s_scale[t] = (k < a.K) ? a.scale_inv[k] : 0.f;
    }
    if (a.tab_in_smem)
        for (int t = threadIdx.x; t < a.lcm; t += blockDim.x) s_tab[t] = a.tw16[t];
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

    if (warp < 8) {
        // ---------------- A producers ----------------
        const int row = threadIdx.x & (kTileM - 1);    // 0..127
        const int kstep = threadIdx.x >> 7;            // 0..1: which 16-frame K-step of a stage
        const int v = v0 + row;
        const bool vok = v < a.S;
        const uint32_t vy = vok ? (uint32_t)(v / a.Sx) : 0u;
        const uint32_t vx = vok ? (uint32_t)(v % a.Sx) : 0u;
        const int g = row >> 3, r = row & 7;
        for (int it = 0; it < a.stages_total; ++it) {
            const int st = it % kStages;
            if (it >= kStages) {
                if (!mbar_wait(&empty[st], ((it / kStages) - 1) & 1, a.wait_ns)) {
                    atomicExch(a.status, 1u);
                    s_abort = 1;
                    break;
                }
            }
            if (s_abort) break;
            // Phase index of this thread's 16 frames.  m = (vy sy mod Sy) my + (vx sx mod Sx) mx;
            // when a frame is the raster successor of the previous one, the two residues are
            // advanced by additions instead of being recomputed (the branch is warp-uniform).
            const int32_t* ip = a.idx + it * kChunk + kstep * 16;
            int32_t sv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) sv[j] = __ldg(ip + j);
            uint32_t sy = 0, sx = 0, myp = 0, mxp = 0;
            uint8_t* stg = stage_base + st * stageBytes;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    uint2 q[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int j = c * 8 + e + u;
                        if (j > 0 && sv[j] == sv[j - 1] + 1) {
                            ++sx;
                            mxp += vx;
                            if (mxp >= (uint32_t)a.Sx) mxp -= (uint32_t)a.Sx;
                            if (sx == (uint32_t)a.Sx) {
                                sx = 0;
                                mxp = 0;
                                ++sy;
                                myp += vy;
                                if (myp >= (uint32_t)a.Sy) myp -= (uint32_t)a.Sy;
                            }
                        } else {
                            const uint32_t s = (uint32_t)sv[j];
                            sy = fastdiv(s, a.mod_x);
                            sx = s - sy * (uint32_t)a.Sx;
                            myp = fastmod(vy * sy, a.mod_y);
                            mxp = fastmod(vx * sx, a.mod_x);
                        }
                        uint32_t m = myp * (uint32_t)a.my + mxp * (uint32_t)a.mx;
                        if (m >= (uint32_t)a.lcm) m -= (uint32_t)a.lcm;
                        q[u] = vok ? tab[m] : make_uint2(0u, 0u);
                    }
                    rh[e / 2] = __byte_perm(q[0].x, q[1].x, 0x5410);
                    rl[e / 2] = __byte_perm(q[0].x, q[1].x, 0x7632);
                    ih[e / 2] = __byte_perm(q[0].y, q[1].y, 0x5410);
                    il[e / 2] = __byte_perm(q[0].y, q[1].y, 0x7632);
                }
                const int off = kstep * 4096 + g * 256 + c * 128 + r * 16;
                *reinterpret_cast<uint4*>(stg + 0 * kATileBytes + off) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                *reinterpret_cast<uint4*>(stg + 1 * kATileBytes + off) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                *reinterpret_cast<uint4*>(stg + 2 * kATileBytes + off) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                *reinterpret_cast<uint4*>(stg + 3 * kATileBytes + off) = make_uint4(il[0], il[1], il[2], il[3]);
            }
            fence_async_smem();
            mbar_arrive(&full[st]);
        }
    } else if (warp == 8) {
        // ---------------- B loader (TMA) ----------------
        if (lane == 0) {
            const uint8_t* src = reinterpret_cast<const uint8_t*>(a.bsplit) +
                                 (size_t)blockIdx.y * a.stages_total * 2 * bTileBytes;
            for (int it = 0; it < a.stages_total; ++it) {
                const int st = it % kStages;
                if (it >= kStages && !mbar_wait(&empty[st], ((it / kStages) - 1) & 1, a.wait_ns)) {
                    atomicExch(a.status, 2u);
                    s_abort = 1;
                    break;
                }
                if (s_abort) break;
                uint8_t* dst = stage_base + st * stageBytes + 4 * kATileBytes;
                mbar_arrive_tx(&full[st], 2 * bTileBytes);
                tma_load_1d(dst, src + (size_t)it * 2 * bTileBytes, 2 * bTileBytes, &full[st]);
            }
        }
    } else {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc(kTileM, NT);
            const uint32_t d_re = tmem, d_im = tmem + (uint32_t)NT;
            uint32_t acc = 0;
            bool ok = true;
            for (int it = 0; it < a.stages_total; ++it) {
                const int st = it % kStages;
                if (!mbar_wait(&full[st], (it / kStages) & 1, a.wait_ns)) {
                    atomicExch(a.status, 3u);
                    s_abort = 1;
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sb = smem_u32(stage_base + st * stageBytes);
#pragma unroll
                for (int ks = 0; ks < kChunk / 16; ++ks) {
                    const uint32_t aoff = ks * 4096;
                    const uint64_t a_rh = smem_desc(sb + 0 * kATileBytes + aoff, 128, 256);
                    const uint64_t a_rl = smem_desc(sb + 1 * kATileBytes + aoff, 128, 256);
                    const uint64_t a_ih = smem_desc(sb + 2 * kATileBytes + aoff, 128, 256);
                    const uint64_t a_il = smem_desc(sb + 3 * kATileBytes + aoff, 128, 256);
                    const uint32_t bb = sb + 4 * kATileBytes + ks * (NT * 32);
                    const uint64_t b_h = smem_desc(bb, 128, 256);
                    const uint64_t b_l = smem_desc(bb + bTileBytes, 128, 256);
                    mma_f16(d_re, a_rh, b_h, idesc, acc);
                    mma_f16(d_re, a_rl, b_h, idesc, 1u);
                    mma_f16(d_re, a_rh, b_l, idesc, 1u);
                    mma_f16(d_im, a_ih, b_h, idesc, acc);
                    mma_f16(d_im, a_il, b_h, idesc, 1u);
                    mma_f16(d_im, a_ih, b_l, idesc, 1u);
                    acc = 1u;
                }
                mma_commit(&empty[st]);   // frees the stage once these MMAs have read it
            }
            mma_commit(done);              // all issued MMAs complete -> epilogue
            (void)ok;
        }
    }

    // ---------------- epilogue: warps 0-3 own TMEM lanes 0-127 ----------------
    if (warp < 4) {
        const bool ok = mbar_wait(done, 0, a.wait_ns);
        if (!ok) atomicExch(a.status, 4u);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = warp * 32 + lane;
        const int v = v0 + row;
        const bool go = __all_sync(0xffffffffu, ok && !s_abort);   // tcgen05.ld needs the whole warp
        if (go) {
            const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
            for (int c0 = 0; c0 < NT; c0 += 16) {
                float re[16], im[16];
                tmem_ld16(lane_addr + (uint32_t)c0, re);
                tmem_ld16(lane_addr + (uint32_t)(NT + c0), im);
                if (v < a.S) {
                    float2* h = a.H + (size_t)v * a.K + k0 + c0;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        int k = k0 + c0 + i;
                        if (k < a.K) {
                            float sc = s_scale[c0 + i];
                            float2 hv = h[i];
                            hv.x = fmaf(re[i], sc, hv.x);
                            hv.y = fmaf(im[i], sc, hv.y);
                            h[i] = hv;
                        }
                    }
                }
            }
        }
    }
    if (blockIdx.x == 0 && blockIdx.y == 0)
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
// and writes them in the B-operand layout of accumulate_tc_kernel:
//   [k-tile][stage][hi|lo][K-step][row group kk/8][core matrix b/8 % 2][kk % 8][b % 8]
// Frames beyond n and columns beyond K are zero.  One thread per (frame pair, column).
__global__ void split_coeff_kernel(const float* __restrict__ c, const unsigned* __restrict__ colmax,
                                   uint16_t* __restrict__ out, float* __restrict__ scale_inv,
                                   int n, int n_pad, int K, int Kp, int NT) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int kk = t % Kp;
    const int b = t / Kp;
    if (b >= n_pad) return;
    float cm = (kk < K) ? __uint_as_float(colmax[kk]) : 0.f;
    int e = 0;
    if (cm > 0.f) frexpf(cm, &e);
    const float sc = (cm > 0.f) ? ldexpf(1.f, 14 - e) : 1.f;
    if (b == 0 && kk < Kp) scale_inv[kk] = (kk < K && cm > 0.f) ? ldexpf(1.f, e - 14) : 0.f;
    float x = (b < n && kk < K) ? c[(size_t)b * K + kk] * sc : 0.f;
    __half hi = __float2half_rn(x);
    __half lo = __float2half_rn(x - __half2float(hi));
    const int ktile = kk / NT, kl = kk % NT;
    const int stage = b / kChunk, bs = b % kChunk;
    const int ks = bs / 16, bk = bs % 16;
    const int stages_total = n_pad / kChunk;
    const size_t bTile = (size_t)NT * kChunk;                 // halves per hi or lo tile
    const size_t base = ((size_t)ktile * stages_total + stage) * 2 * bTile;
    const size_t within = (size_t)ks * NT * 16 + (size_t)(kl >> 3) * 128 + (size_t)(bk >> 3) * 64 +
                          (size_t)(kl & 7) * 8 + (bk & 7);
    out[base + within] = __half_as_ushort(hi);
    out[base + bTile + within] = __half_as_ushort(lo);
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
    return allow_max_dynamic_smem(reinterpret_cast<const void*>(accumulate_tc_kernel));
}

int split_tile_n(int K) {
    int Kp = (K + 15) / 16 * 16;
    return Kp <= 256 ? Kp : 256;
}

size_t split_smem_bytes(int NT) {
    size_t stage = 4 * (size_t)kATileBytes + 2 * (size_t)NT * kChunk * 2;
    return 1024 + kStages * stage + 8 * (2 * kStages + 1) + 16 + 4 * (size_t)NT + 16;
}

// Shared-memory bytes of the phase table when it is kept on chip (0 when it does not fit).
static size_t split_table_bytes(int NT, int lcm) {
    const size_t limit = 226 * 1024;
    const size_t tab = 8 * (size_t)lcm;
    return split_smem_bytes(NT) + tab <= limit ? tab : 0;
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
        size_t total = (size_t)n_pad * Kp;
        split_coeff_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            c, P->d_colmax, reinterpret_cast<uint16_t*>(P->d_bsplit), P->d_scale_inv, n, n_pad,
            P->K, Kp, NT);
    }
    // 2. tensor-core accumulation
    TcArgs a;
    a.bsplit = reinterpret_cast<const uint32_t*>(P->d_bsplit);
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
    int cols = 32;
    while (cols < 2 * NT) cols <<= 1;
    a.tmem_cols = cols;
    a.wait_ns = kDeviceWaitNs;
    a.mod_y = make_fastmod((uint32_t)P->Sy);
    a.mod_x = make_fastmod((uint32_t)P->Sx);
    dim3 grid((P->S + kTileM - 1) / kTileM, Kp / NT);
    const size_t tab = split_table_bytes(NT, P->lcm);
    a.tab_in_smem = tab > 0 ? 1 : 0;
    accumulate_tc_kernel<<<grid, kThreadsTC, split_smem_bytes(NT) + tab, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wdd
