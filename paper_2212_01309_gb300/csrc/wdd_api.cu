// Host side of the C ABI declared in include/wdd.h: parameter validation, the plan-time
// geometry of Sect. 6.2, exact scan bookkeeping, staging of projected frames and the order of
// kernel launches for Algorithm 1 (plan), Algorithm 2 (push) and Eq. 3 (snapshot).
//
// Host floating point that decides an integer (aperture radius, frequency shifts, the
// overlap mask) is evaluated as a fixed sequence of IEEE double operations; this file is
// compiled without floating-point contraction so no fused multiply-add changes a rounding.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "wdd_internal.h"

namespace wdd {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

size_t frame_elem_bytes(int dtype) {
    switch (dtype) {
        case WDD_FRAME_U16: return 2;
        case WDD_FRAME_F32: return 4;
        case WDD_FRAME_F64: return 8;
        default: return 0;
    }
}

namespace {

// CODATA 2018 constants (SI).
constexpr double kPlanck = 6.62607015e-34;
constexpr double kElectronMass = 9.1093837015e-31;
constexpr double kCharge = 1.602176634e-19;
constexpr double kLight = 299792458.0;

int signed_freq(int v, int n) { return (v <= (n - 1) / 2) ? v : v - n; }

}  // namespace

double electron_wavelength(double volts) {
    double ev = kCharge * volts;
    double rel = 1.0 + ev / (2.0 * kElectronMass * kLight * kLight);
    return kPlanck / std::sqrt(2.0 * kElectronMass * ev * rel);
}

int scan_geometry(const wdd_params& p, double R, std::vector<double>& qy, std::vector<double>& qx,
                  std::vector<uint8_t>& mask) {
    const int Sy = p.scan_y, Sx = p.scan_x;
    qy.assign(Sy, 0.0);
    qx.assign(Sx, 0.0);
    double den_y = ((double)Sy * p.scan_step_m) * p.det_px_inv_m;
    double den_x = ((double)Sx * p.scan_step_m) * p.det_px_inv_m;
    for (int v = 0; v < Sy; ++v) qy[v] = (double)signed_freq(v, Sy) / den_y;
    for (int v = 0; v < Sx; ++v) qx[v] = (double)signed_freq(v, Sx) / den_x;
    mask.assign((size_t)Sy * Sx, 0);
    int n_active = 0;
    double lim = 4.0 * (R * R);
    for (int vy = 0; vy < Sy; ++vy)
        for (int vx = 0; vx < Sx; ++vx) {
            double a = qy[vy] * qy[vy];
            double b = qx[vx] * qx[vx];
            double d2 = a + b;
            uint8_t on = d2 < lim ? 1 : 0;
            mask[(size_t)vy * Sx + vx] = on;
            n_active += on;
        }
    return n_active;
}

cudaError_t allow_max_dynamic_smem(const void* func) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    return e;
}

cudaError_t prepare_kernels() {
    static cudaError_t status = [] {
        cudaError_t e = prepare_project_kernels();
        if (e == cudaSuccess) e = prepare_project_tc_kernels();
        if (e == cudaSuccess) e = prepare_project_rows_kernels();
        if (e == cudaSuccess) e = prepare_rows_kernels();
        if (e == cudaSuccess) e = prepare_reconstruct_kernels();
        if (e == cudaSuccess) e = prepare_split_kernels();
        return e;
    }();
    return status;
}

namespace {

wdd_status fail(wdd_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

wdd_status cuda_fail(cudaError_t e, const char* where) {
    return fail(WDD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define WDD_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Energy-ordered pairs (Eq. 10): first K of (n_y, n_x) by n_y + n_x, ties by smaller n_y.
std::vector<std::pair<int, int>> energy_pairs(int K) {
    std::vector<std::pair<int, int>> out;
    for (int e = 0; (int)out.size() < K; ++e)
        for (int ny = 0; ny <= e && (int)out.size() < K; ++ny) out.push_back({ny, e - ny});
    return out;
}

template <typename T>
wdd_status alloc(wdd_plan* P, T** ptr, size_t count) {
    size_t bytes = sizeof(T) * (count ? count : 1);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(WDD_ERR_OUT_OF_MEMORY, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    P->allocs.push_back({p, bytes});
    P->device_bytes += (int64_t)bytes;
    *ptr = static_cast<T*>(p);
    return WDD_OK;
}

void release(wdd_plan* P) {
    for (auto& a : P->allocs) cudaFree(a.ptr);
    P->allocs.clear();
    for (auto& r : P->ring) {
        if (r.done) cudaEventDestroy(r.done);
        if (r.h_frames) cudaFreeHost(r.h_frames);
        r = wdd::RingSlot{};
    }
    if (P->handoff) cudaEventDestroy(P->handoff);
    P->handoff = nullptr;
    for (auto& t : P->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    P->timed.clear();
    for (auto ev : P->event_pool) cudaEventDestroy(ev);
    P->event_pool.clear();
}

// Device-memory footprint planned for these sizes (checked against the budget before any
// allocation happens).
int64_t planned_bytes(const wdd_plan* P) {
    int64_t b = 0;
    b += 16LL * (P->Ny * P->Ly + P->Nx * P->Lx);           // FP64 bases
    b += 8LL * (P->Sy + P->Sx);                             // shifts
    b += 16LL * P->S * P->M;                                // chi (plan time)
    b += 8LL * (P->Ny * P->Ly + P->Nx * P->Lx);             // FP32 bases
    b += 8LL * P->K;                                        // coefficient table
    b += 8LL * P->S * P->K * 2;                             // W and H
    b += (int64_t)P->S;                                     // mask
    b += 16LL * P->lcm + 8LL * (P->Sy + P->Sx);             // tables
    b += 4LL * P->depth * P->K + 4LL * P->depth;            // staging
    b += 16LL * P->S;                                       // spectrum + DFT scratch
    b += 8LL * P->depth_pad * (P->K + 256) + 8LL * P->K;    // FP16 split coefficients
    b += (int64_t)P->depth_pad / 2;                         // 16-frame group records
    if (P->proj_tc)                                                          // basis image, By
        b += 2LL * (int64_t)proj_tc_bimg_halves(P->Nx, P->Lx) + 4LL * ((P->Ny * P->Ly + 3) / 4 * 4);
    if (P->proj_rows)                                                        // By, Bx (FP32), table
        b += 4LL * P->Ny * proj_rows_lyp(P->Ly) + 4LL * P->Nx * proj_rows_lxp(P->Lx) + 4LL * P->K;
    if (P->p.accum_mode == WDD_ACCUM_SEPARABLE) {                            // row slots, G
        const int64_t R = rows_slots(P->Sy, P->depth_pad);
        b += 8LL * R * P->Sx * P->K + 12LL * R + 4LL * P->depth_pad + 4;
    }
    return b;
}

cudaEvent_t pool_event(wdd_plan* P) {
    if (!P->event_pool.empty()) {
        cudaEvent_t e = P->event_pool.back();
        P->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Runs `launch` (which enqueues `count` kernels of one stage on P->stream), with event timing
// around it when enabled, and counts the launches.
template <typename F>
cudaError_t staged_launch(wdd_plan* P, int stage, int count, F&& launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    // inside stream capture the events become event-record nodes of the graph
    unsigned flags = cudaEventRecordDefault;
    if (P->timing) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(P->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
            flags = cudaEventRecordExternal;
        a = pool_event(P);
        b = pool_event(P);
        cudaError_t er = cudaEventRecordWithFlags(a, P->stream, flags);
        if (er != cudaSuccess) return er;
    }
    cudaError_t e = launch();
    if (e != cudaSuccess) return e;
    P->launches_total += count;
    if (P->timing) {
        cudaError_t er = cudaEventRecordWithFlags(b, P->stream, flags);
        if (er != cudaSuccess) return er;
        P->timed.push_back({stage, count, a, b});
    }
    return cudaSuccess;
}

// Projects the pushes gathered for one launch (coalesce_frames), on the plan's stream.
wdd_status launch_pending(wdd_plan* P) {
    wdd::PendingLaunch& q = P->pend;
    if (q.n == 0) return WDD_OK;
    q.segs.first[q.segs.nseg] = q.n;
    float* c_out = P->d_cstage + (size_t)q.slot0 * P->K;
    int32_t* i_out = P->d_idxstage + q.slot0;
    cudaError_t e = staged_launch(P, WDD_STAGE_PROJECT, 1, [&] {
        if (P->proj_rows)
            return launch_project_rows(P, q.segs, P->p.frame_dtype, q.n, P->p.overlap_pushes != 0,
                                       q.ids, c_out, i_out, P->stream);
        return launch_project_tc(P, q.segs, P->p.frame_dtype, q.n, P->p.overlap_pushes != 0, q.ids,
                                 c_out, i_out, P->stream);
    });
    if (e != cudaSuccess) return cuda_fail(e, "projection");
    P->last_coeff_off = q.slot0;
    P->last_coeff_n = q.n;
    q.n = 0;
    q.segs.nseg = 0;
    return WDD_OK;
}

wdd_status flush(wdd_plan* P) {
    {
        wdd_status ls = launch_pending(P);
        if (ls != WDD_OK) return ls;
    }
    if (P->staged == 0) return WDD_OK;
    const bool rows = P->p.accum_mode == WDD_ACCUM_SEPARABLE;
    const int count = rows ? 3
                           : P->p.precision == WDD_PREC_SPLIT ? split_launch_count(P->staged, P->segment)
                                                              : 1;
    cudaError_t e = staged_launch(P, WDD_STAGE_ACCUMULATE, count, [&] {
        if (rows) return launch_accumulate_rows(P, P->d_cstage, P->d_idxstage, P->staged, P->stream);
        return P->p.precision == WDD_PREC_SPLIT
                   ? launch_accumulate_split(P, P->d_cstage, P->d_idxstage, P->staged, P->stream)
                   : launch_accumulate_fp32(P, P->d_cstage, P->d_idxstage, P->staged, P->stream);
    });
    if (e != cudaSuccess) return cuda_fail(e, "phase accumulation");
    P->staged = 0;
    return WDD_OK;
}

wdd_status acquire_slot(wdd_plan* P, wdd::RingSlot** out) {
    wdd::RingSlot& s = P->ring[P->ring_next];
    P->ring_next = (P->ring_next + 1) % wdd::kRingSlots;
    if (s.used) WDD_CUDA(cudaEventSynchronize(s.done));
    *out = &s;
    return WDD_OK;
}

// Makes `st` the plan's stream, ordering it after everything enqueued on the previous one.
wdd_status switch_stream(wdd_plan* P, cudaStream_t st) {
    if (P->stream_set && st != P->stream) {
        // gathered pushes belong to the old stream
        wdd_status ls = launch_pending(P);
        if (ls != WDD_OK) return ls;
        WDD_CUDA(cudaEventRecord(P->handoff, P->stream));
        WDD_CUDA(cudaStreamWaitEvent(st, P->handoff, 0));
    }
    P->stream = st;
    P->stream_set = true;
    return WDD_OK;
}

wdd_status reconstruct(wdd_plan* P, wdd_result* out) {
    if (!out || !out->obj) return fail(WDD_ERR_INVALID_ARG, "result buffer is NULL");
    wdd_status st = flush(P);
    if (st != WDD_OK) return st;
    // the split path accumulates half the scan columns: the rest of H follows by symmetry
    const bool mirror = mirror_needed(P);
    cudaError_t e = staged_launch(P, WDD_STAGE_DECONVOLVE, mirror ? 2 : 1, [&] {
        if (mirror) {
            cudaError_t m = launch_mirror_h(P, P->stream);
            if (m != cudaSuccess) return m;
        }
        return launch_deconvolve(P, P->stream);
    });
    if (e != cudaSuccess) return cuda_fail(e, "deconvolution");
    e = staged_launch(P, WDD_STAGE_IDFT, 2, [&] {
        return launch_inverse_dft(P, static_cast<float2*>(out->obj), out->phase, P->stream);
    });
    if (e != cudaSuccess) return cuda_fail(e, "inverse DFT");
    out->frames_seen = P->frames_seen;
    out->positions_covered = P->covered;
    return WDD_OK;
}

}  // namespace
}  // namespace wdd

using namespace wdd;

extern "C" {

int32_t wdd_version(void) { return (0 << 16) | 1; }

const char* wdd_status_string(wdd_status s) {
    switch (s) {
        case WDD_OK: return "WDD_OK";
        case WDD_ERR_INVALID_ARG: return "WDD_ERR_INVALID_ARG";
        case WDD_ERR_OUT_OF_MEMORY: return "WDD_ERR_OUT_OF_MEMORY";
        case WDD_ERR_CUDA: return "WDD_ERR_CUDA";
        case WDD_ERR_SCAN_INDEX: return "WDD_ERR_SCAN_INDEX";
        case WDD_ERR_STATE: return "WDD_ERR_STATE";
        case WDD_ERR_TIMEOUT: return "WDD_ERR_TIMEOUT";
        case WDD_ERR_UNSUPPORTED: return "WDD_ERR_UNSUPPORTED";
    }
    return "WDD_ERR_UNKNOWN";
}

const char* wdd_last_error(void) { return g_last_error.c_str(); }

wdd_status wdd_params_default(wdd_params* p) {
    if (!p) return fail(WDD_ERR_INVALID_ARG, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->epsilon = 1e-3;
    p->basis = WDD_BASIS_HG_TENSOR;
    p->precision = WDD_PREC_FP32;
    p->frame_dtype = WDD_FRAME_F32;
    p->max_batch = 256;
    p->accum_depth = 0;
    p->det_center_y = -1.0;
    p->det_center_x = -1.0;
    return WDD_OK;
}

namespace {
// Creates a plan, or (footprint != NULL) only validates the parameters and reports the device
// bytes the plan would hold, without touching the GPU.
wdd_status plan_create_impl(const wdd_params* prm, wdd_plan** out, int64_t* footprint) {
    if (!prm || !out) return fail(WDD_ERR_INVALID_ARG, "params or out is NULL");
    *out = nullptr;
    const wdd_params& p = *prm;
    if (p.scan_y <= 0 || p.scan_x <= 0 || p.det_y <= 0 || p.det_x <= 0)
        return fail(WDD_ERR_INVALID_ARG, "scan and detector sizes must be positive");
    if (p.scan_y > 4096 || p.scan_x > 4096)
        return fail(WDD_ERR_UNSUPPORTED, "scan side above 4096");
    if (p.det_y > 1024 || p.det_x > 1024)
        return fail(WDD_ERR_UNSUPPORTED, "detector side above 1024");
    if (!(p.scan_step_m > 0) || !(p.det_px_inv_m > 0) || !(p.voltage_v > 0) ||
        !(p.semiconv_rad > 0) || !std::isfinite(p.defocus_m))
        return fail(WDD_ERR_INVALID_ARG, "step, sampling, voltage and angle must be positive");
    if (!(p.epsilon >= 0) || !std::isfinite(p.epsilon))
        return fail(WDD_ERR_INVALID_ARG, "epsilon must be finite and non-negative");
    if (p.frame_dtype < WDD_FRAME_U16 || p.frame_dtype > WDD_FRAME_F64)
        return fail(WDD_ERR_INVALID_ARG, "unknown frame dtype");
    if (p.precision != WDD_PREC_FP32 && p.precision != WDD_PREC_SPLIT)
        return fail(WDD_ERR_INVALID_ARG, "unknown precision");
    if (p.max_batch <= 0 || p.max_batch > 65536)
        return fail(WDD_ERR_INVALID_ARG, "max_batch must be in [1, 65536]");
    if (p.accum_depth < 0 || p.accum_depth > (1 << 20))
        return fail(WDD_ERR_INVALID_ARG, "accum_depth must be in [0, 2^20]");
    if (p.rank_k <= 0) return fail(WDD_ERR_INVALID_ARG, "rank_k must be positive");
    if (p.proj_cluster < 0 || p.proj_cluster > 8 || (p.proj_cluster & (p.proj_cluster - 1)))
        return fail(WDD_ERR_INVALID_ARG, "proj_cluster must be 0, 1, 2, 4 or 8");
    if (p.accum_segment < 0 || p.accum_segment > 8192)
        return fail(WDD_ERR_INVALID_ARG, "accum_segment must be in [0, 8192]");
    if (p.accum_mode != WDD_ACCUM_DIRECT && p.accum_mode != WDD_ACCUM_SEPARABLE)
        return fail(WDD_ERR_INVALID_ARG, "unknown accumulation mode");
    if (p.coalesce_frames < 0 || p.coalesce_frames > kLaunchFrames)
        return fail(WDD_ERR_INVALID_ARG, "coalesce_frames must be in [0, 4096]");
    if (!std::isfinite(p.scan_rotation_rad))
        return fail(WDD_ERR_INVALID_ARG, "scan_rotation_rad must be finite");
    if (p.proj_engine < WDD_PROJ_AUTO || p.proj_engine > WDD_PROJ_STREAM)
        return fail(WDD_ERR_INVALID_ARG, "unknown projection engine");
    if (p.precision == WDD_PREC_SPLIT && !split_path_available())
        return fail(WDD_ERR_UNSUPPORTED, "split-precision tensor-core path not built");

    wdd_plan* P = new wdd_plan();
    P->p = p;
    P->Sy = p.scan_y;
    P->Sx = p.scan_x;
    P->S = p.scan_y * p.scan_x;
    P->Ny = p.det_y;
    P->Nx = p.det_x;
    P->cy = p.det_center_y >= 0 ? p.det_center_y : (double)(p.det_y / 2);
    P->cx = p.det_center_x >= 0 ? p.det_center_x : (double)(p.det_x / 2);
    P->K = p.rank_k;
    P->max_batch = p.max_batch;
    P->chunk = std::min(p.max_batch, kLaunchFrames);
    P->depth = p.accum_depth > 0 ? std::max(p.accum_depth, p.max_batch) : p.max_batch;
    P->depth_pad = (P->depth + 63) / 64 * 64;
    P->segment = p.accum_segment > 0 ? (p.accum_segment + 63) / 64 * 64 : 1024;
    if (p.precision == WDD_PREC_SPLIT && P->depth_pad > 8192) {
        delete P;
        return fail(WDD_ERR_INVALID_ARG, "split precision stages at most 8192 frames");
    }
    P->lcm = std::lcm(P->Sy, P->Sx);
    if (!footprint) cudaGetDevice(&P->device);

    // ---- geometry (Sect. 6.2) ------------------------------------------------------------
    P->lambda = electron_wavelength(p.voltage_v);
    P->R = p.semiconv_rad / (P->lambda * p.det_px_inv_m);

    // ---- basis family and coefficient table ----------------------------------------------
    std::vector<int32_t>& kt = P->h_ktab;
    if (p.basis == WDD_BASIS_FOURIER_FULL) {
        if (P->Ny > 64 || P->Nx > 64) {
            delete P;
            return fail(WDD_ERR_UNSUPPORTED, "FOURIER_FULL needs detector sides <= 64");
        }
        P->complex_basis = 1;
        P->Ly = P->Ny;
        P->Lx = P->Nx;
        for (int ry = 0; ry < P->Ny; ++ry)
            for (int rx = 0; rx < P->Nx; ++rx) {
                int m = ry * P->Nx + rx;
                int n = ((P->Ny - ry) % P->Ny) * P->Nx + (P->Nx - rx) % P->Nx;
                if (m > n) continue;
                kt.push_back(m); kt.push_back(0);
                if (m != n) { kt.push_back(m); kt.push_back(1); }
            }
        if ((int)kt.size() / 2 != P->K) {
            delete P;
            return fail(WDD_ERR_INVALID_ARG, "FOURIER_FULL needs rank_k = det_y * det_x");
        }
    } else if (p.basis == WDD_BASIS_HG_TENSOR || p.basis == WDD_BASIS_HG_ENERGY) {
        int L;
        std::vector<std::pair<int, int>> pairs;
        if (p.basis == WDD_BASIS_HG_TENSOR) {
            L = (int)std::lround(std::sqrt((double)P->K));
            if (L * L != P->K) {
                delete P;
                return fail(WDD_ERR_INVALID_ARG, "HG_TENSOR needs a square rank_k");
            }
            for (int a = 0; a < L; ++a)
                for (int b = 0; b < L; ++b) pairs.push_back({a, b});
        } else {
            pairs = energy_pairs(P->K);
            L = 0;
            for (auto& q : pairs) L = std::max(L, std::max(q.first, q.second) + 1);
        }
        if (L > 32) {
            delete P;
            return fail(WDD_ERR_INVALID_ARG, "Hermite-Gauss order above 32 per axis");
        }
        if (L > P->Ny || L > P->Nx) {
            delete P;
            return fail(WDD_ERR_INVALID_ARG, "more Hermite-Gauss functions than detector pixels");
        }
        P->Ly = P->Lx = L;
        P->sigma = P->R / std::sqrt(2.0 * (L - 1) + 1.0);
        for (auto& q : pairs) { kt.push_back(q.first * L + q.second); kt.push_back(0); }
    } else {
        delete P;
        return fail(WDD_ERR_INVALID_ARG, "unknown basis");
    }
    P->M = P->Ly * P->Lx;
    {
        // shared-memory footprints of the plan and projection kernels (227 KB per CTA)
        const size_t lim = 227u * 1024u;
        size_t chi = 16u * ((size_t)P->Nx * P->Lx + 8u * P->Nx + 8u * P->Lx);
        P->proj = make_proj_geom(P->Ny, P->Nx, P->Ly, P->Lx, P->K, P->complex_basis,
                                 std::min(p.max_batch, kLaunchFrames), p.proj_cluster);
        size_t proj = proj_smem_bytes(P->proj) + 1024;
        size_t tc = p.precision == WDD_PREC_SPLIT ? split_smem_bytes(split_tile_n(P->K)) : 0;
        if (chi > lim || proj > lim || tc > lim) {
            delete P;
            return fail(WDD_ERR_UNSUPPORTED, "detector width times basis order too large");
        }
        // split precision: the streaming FP32 projection wherever it applies (unless the tensor
        // cores or the staged SIMT kernel were asked for), else the tensor cores where they
        // apply, else the staged SIMT kernel; FP32 plans keep the staged SIMT kernel
        const bool split = p.precision == WDD_PREC_SPLIT;
        const bool rows_ok = split &&
                             proj_rows_supported(P->Ny, P->Nx, P->Ly, P->Lx, P->K,
                                                 P->complex_basis, p.frame_dtype);
        const bool tc_ok = split && proj_tc_supported(P->Nx, P->Lx, P->complex_basis, p.frame_dtype) &&
                           proj_tc_smem_bytes(P->Ny, P->Nx, P->Ly, P->Lx, P->K) + 1024 <= lim;
        const int want = p.proj_engine;
        if (want == WDD_PROJ_TENSOR && tc_ok) P->proj_tc = 1;
        else if (want == WDD_PROJ_SIMT && split) P->proj_tc = 0;
        else if (rows_ok) P->proj_rows = 1;
        else if (tc_ok) P->proj_tc = 1;
    }
    if (P->K > 4096) {
        delete P;
        return fail(WDD_ERR_UNSUPPORTED, "rank above 4096");
    }

    // ---- shifts and active mask (Sect. 6.2, Eq. 15; R8: |q_v| < 2 R strictly) ----------------------
    std::vector<double> qy, qx;
    std::vector<uint8_t> mask;
    P->n_active = scan_geometry(p, P->R, qy, qx, mask);

    // ---- memory budget -----------------------------------------------------------------
    int64_t need = planned_bytes(P);
    if (footprint) {
        *footprint = need;
        delete P;
        return WDD_OK;
    }
    if (p.hbm_budget_bytes > 0 && need > p.hbm_budget_bytes) {
        delete P;
        char buf[160];
        std::snprintf(buf, sizeof buf, "plan needs %lld bytes, budget is %lld",
                      (long long)need, (long long)p.hbm_budget_bytes);
        return fail(WDD_ERR_OUT_OF_MEMORY, buf);
    }

    {
        cudaError_t pe = prepare_kernels();
        if (pe != cudaSuccess) {
            delete P;
            return cuda_fail(pe, "kernel attributes");
        }
    }

    wdd_status st = WDD_OK;
#define WDD_ALLOC(ptr, n)                         \
    do {                                          \
        st = alloc(P, &(ptr), (n));               \
        if (st != WDD_OK) { release(P); delete P; return st; } \
    } while (0)
    WDD_ALLOC(P->d_By, (size_t)P->Ny * P->Ly);
    WDD_ALLOC(P->d_Bx, (size_t)P->Nx * P->Lx);
    WDD_ALLOC(P->d_qy, P->Sy);
    WDD_ALLOC(P->d_qx, P->Sx);
    WDD_ALLOC(P->d_chi, (size_t)P->S * P->M);
    WDD_ALLOC(P->d_By32, (size_t)P->Ny * P->Ly);
    WDD_ALLOC(P->d_Bx32, (size_t)P->Nx * P->Lx);
    WDD_ALLOC(P->d_ktab, P->K);
    WDD_ALLOC(P->d_W, (size_t)P->S * P->K);
    WDD_ALLOC(P->d_mask, P->S);
    WDD_ALLOC(P->d_H, (size_t)P->S * P->K);
    WDD_ALLOC(P->d_tw, P->lcm);
    WDD_ALLOC(P->d_tw16, P->lcm);
    WDD_ALLOC(P->d_twy, P->Sy);
    WDD_ALLOC(P->d_twx, P->Sx);
    WDD_ALLOC(P->d_cstage, (size_t)P->depth_pad * P->K);
    WDD_ALLOC(P->d_idxstage, P->depth_pad);
    WDD_ALLOC(P->d_status, 1);
    WDD_ALLOC(P->d_o, P->S);
    WDD_ALLOC(P->d_tmp, P->S);
    if (p.precision == WDD_PREC_SPLIT) {
        int NT = split_tile_n(P->K);
        int Kp = (P->K + NT - 1) / NT * NT;
        WDD_ALLOC(P->d_bsplit, split_coeff_bytes(P->K, P->depth_pad) / 2);
        WDD_ALLOC(P->d_scale_inv, Kp);
        WDD_ALLOC(P->d_grp, P->depth_pad / 16);
        WDD_ALLOC(P->d_colmax, P->K);
    }
    if (P->proj_tc) {
        WDD_ALLOC(P->d_bimg, proj_tc_bimg_halves(P->Nx, P->Lx));
        WDD_ALLOC(P->d_Byre, ((size_t)P->Ny * P->Ly + 3) / 4 * 4);
    }
    if (P->proj_rows) {
        WDD_ALLOC(P->d_Byp, (size_t)P->Ny * proj_rows_lyp(P->Ly));
        WDD_ALLOC(P->d_Bxp, (size_t)P->Nx * proj_rows_lxp(P->Lx));
        WDD_ALLOC(P->d_kpad, P->K);
    }
    if (p.accum_mode == WDD_ACCUM_SEPARABLE) {
        const int R = rows_slots(P->Sy, P->depth_pad);
        WDD_ALLOC(P->d_G, (size_t)R * P->Sx * P->K);
        WDD_ALLOC(P->d_slotrow, R);
        WDD_ALLOC(P->d_slotfirst, R);
        WDD_ALLOC(P->d_slotlast, R);
        WDD_ALLOC(P->d_frameslot, P->depth_pad);
        WDD_ALLOC(P->d_nslots, 1);
    }
#undef WDD_ALLOC

    cudaStream_t s0 = nullptr;
    auto bail = [&](wdd_status s) { release(P); delete P; return s; };
    auto cbail = [&](cudaError_t e, const char* w) { cuda_fail(e, w); release(P); delete P; return WDD_ERR_CUDA; };
    cudaError_t e;
    if ((e = cudaMemcpy(P->d_qy, qy.data(), 8 * P->Sy, cudaMemcpyHostToDevice))) return cbail(e, "copy shifts");
    if ((e = cudaMemcpy(P->d_qx, qx.data(), 8 * P->Sx, cudaMemcpyHostToDevice))) return cbail(e, "copy shifts");
    if ((e = cudaMemcpy(P->d_mask, mask.data(), P->S, cudaMemcpyHostToDevice))) return cbail(e, "copy mask");
    if ((e = cudaMemcpy(P->d_ktab, kt.data(), 8 * P->K, cudaMemcpyHostToDevice))) return cbail(e, "copy table");

    // ---- bases (FP64 on the GPU) -------------------------------------------------------
    if (P->complex_basis) {
        if ((e = launch_fourier_basis(P->d_By, P->Ny, P->cy, s0))) return cbail(e, "Fourier basis");
        if ((e = launch_fourier_basis(P->d_Bx, P->Nx, P->cx, s0))) return cbail(e, "Fourier basis");
    } else {
        if ((e = launch_hg_basis(P->d_By, P->Ny, P->Ly, P->sigma, P->cy, s0))) return cbail(e, "HG basis");
        if ((e = launch_hg_basis(P->d_Bx, P->Nx, P->Lx, P->sigma, P->cx, s0))) return cbail(e, "HG basis");
    }
    if (P->proj_tc && (e = launch_build_bimg(P, P->d_bimg, s0))) return cbail(e, "projection basis image");
    {
        std::vector<double2> by((size_t)P->Ny * P->Ly), bx((size_t)P->Nx * P->Lx);
        if ((e = cudaMemcpy(by.data(), P->d_By, 16 * by.size(), cudaMemcpyDeviceToHost))) return cbail(e, "basis copy");
        if ((e = cudaMemcpy(bx.data(), P->d_Bx, 16 * bx.size(), cudaMemcpyDeviceToHost))) return cbail(e, "basis copy");
        std::vector<float2> fy(by.size()), fx(bx.size());
        for (size_t i = 0; i < by.size(); ++i) fy[i] = make_float2((float)by[i].x, (float)by[i].y);
        for (size_t i = 0; i < bx.size(); ++i) fx[i] = make_float2((float)bx[i].x, (float)bx[i].y);
        if ((e = cudaMemcpy(P->d_By32, fy.data(), 8 * fy.size(), cudaMemcpyHostToDevice))) return cbail(e, "basis copy");
        if ((e = cudaMemcpy(P->d_Bx32, fx.data(), 8 * fx.size(), cudaMemcpyHostToDevice))) return cbail(e, "basis copy");
        if (P->d_Byre) {
            std::vector<float> re((by.size() + 3) / 4 * 4, 0.f);
            for (size_t i = 0; i < by.size(); ++i) re[i] = (float)by[i].x;
            if ((e = cudaMemcpy(P->d_Byre, re.data(), 4 * re.size(), cudaMemcpyHostToDevice))) return cbail(e, "basis copy");
        }
        if (P->proj_rows) {
            // real parts, zero-padded to the streaming projection's widths, and each
            // coefficient's place in a padded LYP x LXP block
            const int LYP = proj_rows_lyp(P->Ly), LXP = proj_rows_lxp(P->Lx);
            std::vector<float> yp((size_t)P->Ny * LYP, 0.f), xp((size_t)P->Nx * LXP, 0.f);
            for (int i = 0; i < P->Ny; ++i)
                for (int l = 0; l < P->Ly; ++l) yp[(size_t)i * LYP + l] = (float)by[(size_t)i * P->Ly + l].x;
            for (int i = 0; i < P->Nx; ++i)
                for (int l = 0; l < P->Lx; ++l) xp[(size_t)i * LXP + l] = (float)bx[(size_t)i * P->Lx + l].x;
            std::vector<int32_t> kp(P->K);
            for (int k = 0; k < P->K; ++k) kp[k] = kt[2 * k] / P->Lx * LXP + kt[2 * k] % P->Lx;
            if ((e = cudaMemcpy(P->d_Byp, yp.data(), 4 * yp.size(), cudaMemcpyHostToDevice))) return cbail(e, "basis copy");
            if ((e = cudaMemcpy(P->d_Bxp, xp.data(), 4 * xp.size(), cudaMemcpyHostToDevice))) return cbail(e, "basis copy");
            if ((e = cudaMemcpy(P->d_kpad, kp.data(), 4 * kp.size(), cudaMemcpyHostToDevice))) return cbail(e, "copy table");
        }
    }

    // ---- Algorithm 1: chi_v, eps_eff, Wiener weights ------------------------------------
    unsigned long long* d_max = nullptr;
    if ((e = cudaMalloc(&d_max, sizeof(unsigned long long)))) return cbail(e, "alloc");
    cudaMemset(d_max, 0, sizeof(unsigned long long));
    e = launch_chi(P, d_max, s0);
    unsigned long long maxbits = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&maxbits, d_max, 8, cudaMemcpyDeviceToHost);
    cudaFree(d_max);
    if (e) return cbail(e, "probe autocorrelation projection");
    double maxchi;
    std::memcpy(&maxchi, &maxbits, 8);
    P->eps_eff = p.eps_absolute ? p.epsilon : p.epsilon * maxchi;
    if (!(P->eps_eff > 0) && p.epsilon > 0) return bail(fail(WDD_ERR_INVALID_ARG, "probe autocorrelation is zero everywhere"));
    if ((e = launch_weights(P, s0))) return cbail(e, "Wiener weights");
    if ((e = launch_tables(P, s0))) return cbail(e, "phase tables");
    if ((e = cudaMemset(P->d_H, 0, 8 * (size_t)P->S * P->K))) return cbail(e, "zero accumulator");
    if ((e = cudaMemset(P->d_idxstage, 0, 4 * (size_t)P->depth_pad))) return cbail(e, "zero staging");
    if ((e = cudaMemset(P->d_cstage, 0, 4 * (size_t)P->depth_pad * P->K))) return cbail(e, "zero staging");
    if ((e = cudaMemset(P->d_status, 0, 4))) return cbail(e, "zero status");
    if (P->d_colmax && (e = cudaMemset(P->d_colmax, 0, 4 * (size_t)P->K))) return cbail(e, "zero column max");
    if ((e = cudaDeviceSynchronize())) return cbail(e, "plan build");

    // keep chi for inspection only when it is small
    if ((size_t)P->S * P->M * 16 > (256u << 20)) {
        for (auto it = P->allocs.begin(); it != P->allocs.end(); ++it)
            if (it->ptr == P->d_chi) {
                cudaFree(it->ptr);
                P->device_bytes -= (int64_t)it->bytes;
                P->allocs.erase(it);
                break;
            }
        P->d_chi = nullptr;
    }

    for (auto& r : P->ring)
        if ((e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming))) return cbail(e, "ring event");
    if ((e = cudaEventCreateWithFlags(&P->handoff, cudaEventDisableTiming))) return cbail(e, "event");
    P->hits.assign(P->S, 0u);
    *out = P;
    return WDD_OK;
}

}  // namespace

wdd_status wdd_plan_create(const wdd_params* prm, wdd_plan** out) {
    return plan_create_impl(prm, out, nullptr);
}

wdd_status wdd_plan_footprint(const wdd_params* prm, int64_t* bytes) {
    if (!bytes) return fail(WDD_ERR_INVALID_ARG, "bytes is NULL");
    wdd_plan* unused = nullptr;
    return plan_create_impl(prm, &unused, bytes);
}

wdd_status wdd_flush(wdd_plan* P) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    return flush(P);
}

int32_t wdd_flush_group_max(void) { return accumulate_group_max(); }

wdd_status wdd_flush_group(wdd_plan* const* plans, int32_t count, wdd_stream_t stream) {
    if (!plans) return fail(WDD_ERR_INVALID_ARG, "plans is NULL");
    if (count < 1 || count > accumulate_group_max())
        return fail(WDD_ERR_INVALID_ARG, "group size out of range");
    for (int j = 0; j < count; ++j) {
        const wdd_plan* P = plans[j];
        if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
        for (int i = 0; i < j; ++i)
            if (plans[i] == P) return fail(WDD_ERR_INVALID_ARG, "plan repeated in the group");
        if (P->p.precision != WDD_PREC_SPLIT || P->p.accum_mode != WDD_ACCUM_DIRECT)
            return fail(WDD_ERR_INVALID_ARG, "grouped flush needs SPLIT plans with DIRECT accumulation");
        if (P->finished) return fail(WDD_ERR_STATE, "plan already finalized");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int j = 0; j < count; ++j) {
        wdd_status ss = switch_stream(plans[j], st);
        if (ss != WDD_OK) return ss;
    }
    // gathered pushes: streaming-projection plans of one class share launches, the others
    // project their own
    wdd_plan* rows[wdd::kProjGroupMax];
    int nr = 0;
    for (int j = 0; j < count; ++j) {
        wdd_plan* P = plans[j];
        if (P->pend.n == 0) continue;
        if (P->proj_rows && nr < wdd::kProjGroupMax) {
            rows[nr++] = P;
        } else {
            wdd_status ls = launch_pending(P);
            if (ls != WDD_OK) return ls;
        }
    }
    bool taken[wdd::kProjGroupMax] = {};
    for (int i = 0; i < nr; ++i) {
        if (taken[i]) continue;
        wdd_plan* grp[wdd::kProjGroupMax];
        int ng = 0, frames = 0, nseg = 0;
        for (int k = i; k < nr; ++k) {
            wdd_plan* P = rows[k];
            if (taken[k] || wdd::proj_rows_class(P) != wdd::proj_rows_class(rows[i])) continue;
            if (frames + P->pend.n > wdd::kLaunchFrames || nseg + P->pend.segs.nseg > wdd::kMaxSegs)
                continue;
            grp[ng++] = P;
            frames += P->pend.n;
            nseg += P->pend.segs.nseg;
            taken[k] = true;
        }
        cudaError_t e = staged_launch(grp[0], WDD_STAGE_PROJECT, 1, [&] {
            return wdd::launch_project_rows_group(grp, ng, st);
        });
        if (e != cudaSuccess) return cuda_fail(e, "grouped projection");
        for (int k = 0; k < ng; ++k) {
            wdd::PendingLaunch& q = grp[k]->pend;
            grp[k]->last_coeff_off = q.slot0;
            grp[k]->last_coeff_n = q.n;
            q.n = 0;
            q.segs.nseg = 0;
        }
    }
    wdd_plan* active[64];
    int m = 0;
    for (int j = 0; j < count; ++j)
        if (plans[j]->staged > 0) active[m++] = plans[j];
    if (m == 0) return WDD_OK;
    cudaError_t e = staged_launch(active[0], WDD_STAGE_ACCUMULATE, 2, [&] {
        return launch_accumulate_group(active, m, st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "grouped phase accumulation");
    for (int j = 0; j < m; ++j) active[j]->staged = 0;
    return WDD_OK;
}

wdd_status wdd_plan_destroy(wdd_plan* P) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    if (P->stream) cudaStreamSynchronize(P->stream);
    release(P);
    delete P;
    return WDD_OK;
}

wdd_status wdd_push_frames(wdd_plan* P, const void* frames, const int32_t* scan_idx, int64_t n,
                           wdd_stream_t stream) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    if (P->finished) return fail(WDD_ERR_STATE, "plan is finalized");
    if (n < 0) return fail(WDD_ERR_INVALID_ARG, "negative frame count");
    if (n == 0) return WDD_OK;
    if (!frames || !scan_idx) return fail(WDD_ERR_INVALID_ARG, "frames or scan_idx is NULL");
    for (int64_t i = 0; i < n; ++i)
        if (scan_idx[i] < 0 || scan_idx[i] >= P->S) {
            char buf[128];
            std::snprintf(buf, sizeof buf, "scan index %d at position %lld outside [0, %d)",
                          scan_idx[i], (long long)i, P->S);
            return fail(WDD_ERR_SCAN_INDEX, buf);
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // where do the frames live?
    cudaPointerAttributes attr{};
    cudaError_t e = cudaPointerGetAttributes(&attr, frames);
    if (e != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    const char* src = nullptr;
    bool pageable = false;
    bool device_src = false;
    if (attr.type == cudaMemoryTypeDevice) {
        src = static_cast<const char*>(frames);
        device_src = true;
    } else if (attr.type == cudaMemoryTypeManaged) {
        src = static_cast<const char*>(frames);
    } else if (attr.type == cudaMemoryTypeHost) {
        src = static_cast<const char*>(attr.devicePointer ? attr.devicePointer : frames);
    } else {
        pageable = true;
    }
    const size_t fbytes = frame_elem_bytes(P->p.frame_dtype) * (size_t)P->Ny * P->Nx;
    if (pageable && P->frame_slot_bytes == 0) {
        size_t slot = fbytes * P->chunk;
        for (auto& r : P->ring) {
            if (r.used) WDD_CUDA(cudaEventSynchronize(r.done));
            e = cudaMallocHost(&r.h_frames, slot);
            if (e != cudaSuccess) return fail(WDD_ERR_OUT_OF_MEMORY, "pinned staging for pageable frames");
        }
        P->frame_slot_bytes = slot;
    }

    {
        wdd_status ss = switch_stream(P, st);
        if (ss != WDD_OK) return ss;
    }
    const bool coalesce = P->p.coalesce_frames > 0 && (P->proj_tc || P->proj_rows) && !pageable &&
                          (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
    if (coalesce) {
        // gather into the pending launch (at most kLaunchFrames frames from kMaxSegs pushes,
        // and no more than the staging depth)
        wdd::PendingLaunch& q = P->pend;
        const int cap = std::min(kLaunchFrames, P->depth);
        for (int64_t off = 0; off < n;) {
            if (q.n == cap || q.segs.nseg == kMaxSegs) {
                wdd_status ls = launch_pending(P);
                if (ls != WDD_OK) return ls;
            }
            int nb = (int)std::min<int64_t>(cap - q.n, n - off);
            if (P->staged + nb > P->depth) {
                wdd_status fs = flush(P);   // launches the pending frames first
                if (fs != WDD_OK) return fs;
                nb = (int)std::min<int64_t>(cap, n - off);
            }
            if (q.n == 0) q.slot0 = P->staged;
            q.segs.ptr[q.segs.nseg] = src + fbytes * off;
            q.segs.first[q.segs.nseg] = q.n;
            ++q.segs.nseg;
            std::memcpy(q.ids.s + q.n, scan_idx + off, sizeof(int32_t) * nb);
            q.n += nb;
            P->staged += nb;
            off += nb;
        }
        if (q.n >= P->p.coalesce_frames) {
            wdd_status ls = launch_pending(P);
            if (ls != WDD_OK) return ls;
        }
        if (P->p.accum_depth == 0) {
            wdd_status fs = flush(P);
            if (fs != WDD_OK) return fs;
        }
    } else {
        wdd_status ls = launch_pending(P);   // keep launches in push order
        if (ls != WDD_OK) return ls;
    }
    for (int64_t off = 0; off < n && !coalesce; off += P->chunk) {
        int nb = (int)std::min<int64_t>(P->chunk, n - off);
        bool flushed = false;
        if (P->staged + nb > P->depth) {
            wdd_status fs = flush(P);
            if (fs != WDD_OK) return fs;
            flushed = true;
        }
        IndexBlock ids;
        std::memcpy(ids.s, scan_idx + off, sizeof(int32_t) * nb);
        wdd::RingSlot* slot = nullptr;
        const void* fsrc;
        if (pageable) {
            wdd_status ss = acquire_slot(P, &slot);
            if (ss != WDD_OK) return ss;
            std::memcpy(slot->h_frames, static_cast<const char*>(frames) + fbytes * off, fbytes * nb);
            void* dp = nullptr;
            WDD_CUDA(cudaHostGetDevicePointer(&dp, slot->h_frames, 0));
            fsrc = dp;
        } else {
            fsrc = src + fbytes * off;
        }
        float* c_out = P->d_cstage + (size_t)P->staged * P->K;
        int32_t* i_out = P->d_idxstage + P->staged;
        e = staged_launch(P, WDD_STAGE_PROJECT, 1, [&] {
            // overlap with the previous kernel only when that kernel was launched by this call (a
            // projection of an earlier chunk, or the flush just above, which itself started only
            // after all earlier work on the stream), or when the caller allowed overlap across
            // pushes
            const bool overlap = off > 0 || flushed || P->p.overlap_pushes != 0;
            if ((P->proj_tc || P->proj_rows) && (reinterpret_cast<uintptr_t>(fsrc) & 15u) == 0) {
                wdd::FrameSegs one{};
                one.ptr[0] = fsrc;
                one.first[0] = 0;
                one.first[1] = nb;
                one.nseg = 1;
                if (P->proj_rows)
                    return launch_project_rows(P, one, P->p.frame_dtype, nb, overlap, ids, c_out,
                                               i_out, st);
                return launch_project_tc(P, one, P->p.frame_dtype, nb, overlap, ids, c_out, i_out,
                                         st);
            }
            return launch_project(P, fsrc, P->p.frame_dtype, nb, device_src, overlap, ids, c_out,
                                  i_out, st);
        });
        if (e != cudaSuccess) return cuda_fail(e, "projection");
        if (slot) {
            WDD_CUDA(cudaEventRecord(slot->done, st));
            slot->used = true;
        }
        P->last_coeff_off = P->staged;
        P->last_coeff_n = nb;
        P->staged += nb;
        if (P->p.accum_depth == 0 && (off + nb == n || P->staged + P->chunk > P->depth)) {
            wdd_status fs = flush(P);
            if (fs != WDD_OK) return fs;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        if (P->hits[scan_idx[i]]++ == 0u) ++P->covered;
    }
    P->frames_seen += n;
    return WDD_OK;
}

wdd_status wdd_snapshot(wdd_plan* P, wdd_result* out) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    return reconstruct(P, out);
}

wdd_status wdd_finalize(wdd_plan* P, wdd_result* out) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    if (P->finished) return fail(WDD_ERR_STATE, "plan already finalized");
    wdd_status s = reconstruct(P, out);
    if (s == WDD_OK) P->finished = true;
    return s;
}

wdd_status wdd_set_stream(wdd_plan* P, wdd_stream_t stream) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    return switch_stream(P, static_cast<cudaStream_t>(stream));
}

wdd_status wdd_reset(wdd_plan* P) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    WDD_CUDA(cudaMemsetAsync(P->d_H, 0, 8 * (size_t)P->S * P->K, P->stream));
    if (P->d_colmax) WDD_CUDA(cudaMemsetAsync(P->d_colmax, 0, 4 * (size_t)P->K, P->stream));
    P->staged = 0;
    P->pend.n = 0;             // gathered pushes are dropped with the staged frames
    P->pend.segs.nseg = 0;
    P->frames_seen = 0;
    P->covered = 0;
    P->finished = false;
    std::fill(P->hits.begin(), P->hits.end(), 0u);
    return WDD_OK;
}

wdd_status wdd_plan_get_info(const wdd_plan* P, wdd_plan_info* out) {
    if (!P || !out) return fail(WDD_ERR_INVALID_ARG, "plan or out is NULL");
    out->rank_k = P->K;
    out->basis_ly = P->Ly;
    out->basis_lx = P->Lx;
    out->n_active = P->n_active;
    out->eps_eff = P->eps_eff;
    out->wavelength_m = P->lambda;
    out->bf_radius_px = P->R;
    out->hg_sigma_px = P->sigma;
    out->device_bytes = P->device_bytes;
    out->frames_seen = P->frames_seen;
    out->positions_covered = P->covered;
    out->kernel_launches = P->launches_total;
    out->staged = P->staged;
    out->finished = P->finished ? 1 : 0;
    out->proj_tensor = P->proj_tc;
    out->proj_engine = P->proj_tc ? WDD_PROJ_TENSOR : P->proj_rows ? WDD_PROJ_STREAM : WDD_PROJ_SIMT;
    out->accum_mode = P->p.accum_mode;
    out->pending = P->pend.n;
    out->accum_kernel = accum_kernel_of(P);
    out->spectrum_cols = mirror_needed(P) ? spectrum_cols(P->Sx) : P->Sx;
    return WDD_OK;
}

wdd_status wdd_set_stage_timing(wdd_plan* P, int32_t enable) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    P->timing = enable != 0;
    return WDD_OK;
}

wdd_status wdd_get_stage_times(wdd_plan* P, double* ms_out, int64_t* launches_out) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    WDD_CUDA(cudaStreamSynchronize(P->stream));
    double ms[WDD_STAGE_COUNT] = {0, 0, 0, 0};
    int64_t cnt[WDD_STAGE_COUNT] = {0, 0, 0, 0};
    for (auto& t : P->timed) {
        float f = 0.f;
        WDD_CUDA(cudaEventElapsedTime(&f, t.a, t.b));
        ms[t.stage] += f;
        cnt[t.stage] += t.launches;
        P->event_pool.push_back(t.a);
        P->event_pool.push_back(t.b);
    }
    P->timed.clear();
    for (int s = 0; s < WDD_STAGE_COUNT; ++s) {
        if (ms_out) ms_out[s] = ms[s];
        if (launches_out) launches_out[s] = cnt[s];
    }
    return WDD_OK;
}

wdd_status wdd_check_device(wdd_plan* P) {
    if (!P) return fail(WDD_ERR_INVALID_ARG, "plan is NULL");
    WDD_CUDA(cudaStreamSynchronize(P->stream));
    unsigned code = 0;
    WDD_CUDA(cudaMemcpy(&code, P->d_status, 4, cudaMemcpyDeviceToHost));
    if (code == 9u) {
        WDD_CUDA(cudaMemset(P->d_status, 0, 4));
        return fail(WDD_ERR_UNSUPPORTED,
                    "a float32 frame value is outside the FP16 split range |I| < 65520 of the "
                    "tensor-core projection (use the FP32 precision path for such frames)");
    }
    if (code != 0) {
        WDD_CUDA(cudaMemset(P->d_status, 0, 4));
        char buf[96];
        std::snprintf(buf, sizeof buf, "a device wait gave up (code %u)", code);
        return fail(WDD_ERR_TIMEOUT, buf);
    }
    return WDD_OK;
}

wdd_status wdd_selftest_bounded_wait(int64_t wait_ns) {
    if (wait_ns <= 0 || wait_ns > 10000000000LL) return fail(WDD_ERR_INVALID_ARG, "wait_ns out of range");
    unsigned* d = nullptr;
    WDD_CUDA(cudaMalloc(&d, 4));
    cudaError_t e = cudaMemset(d, 0, 4);
    if (e == cudaSuccess) e = launch_bounded_wait_selftest(d, (uint64_t)wait_ns, nullptr);
    unsigned code = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&code, d, 4, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self test");
    if (code == 7u) return fail(WDD_ERR_TIMEOUT, "the device wait gave up as designed");
    return WDD_OK;
}

wdd_status wdd_reconstruct_noalloc(const void* weights, const void* accum, int32_t scan_y,
                                   int32_t scan_x, int32_t rank_k, void* obj, float* phase,
                                   wdd_stream_t stream) {
    if (!weights || !accum || !obj)
        return fail(WDD_ERR_INVALID_ARG, "weights, accum and obj must not be NULL");
    if (scan_y <= 0 || scan_x <= 0 || rank_k <= 0 || scan_y > 4096 || scan_x > 4096)
        return fail(WDD_ERR_INVALID_ARG, "scan sizes must be in [1, 4096] and rank_k positive");
    const size_t S = (size_t)scan_y * scan_x;
    const size_t need = 16 * S + 8 * ((size_t)scan_y + scan_x);
    if (need > noalloc_scratch_limit()) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "scan %d x %d needs %zu bytes of scratch; the built-in scratch holds %zu "
                      "(at most about 524,000 scan positions)",
                      scan_y, scan_x, need, noalloc_scratch_limit());
        return fail(WDD_ERR_INVALID_ARG, buf);
    }
    int dev = 0;
    WDD_CUDA(cudaGetDevice(&dev));
    void* scratch = nullptr;
    WDD_CUDA(noalloc_scratch(dev, &scratch));
    cudaError_t e = launch_reconstruct_noalloc(scratch, static_cast<const float2*>(weights),
                                               static_cast<const float2*>(accum), scan_y, scan_x,
                                               rank_k, static_cast<float2*>(obj), phase,
                                               static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "reconstruction without allocation");
    return WDD_OK;
}

wdd_status wdd_detector_center(const void* frames, int64_t n, int32_t det_y, int32_t det_x,
                               int32_t frame_dtype, double* center_y, double* center_x,
                               wdd_stream_t stream) {
    if (!frames || !center_y || !center_x)
        return fail(WDD_ERR_INVALID_ARG, "frames and outputs must not be NULL");
    if (n < 1 || det_y <= 0 || det_x <= 0 || det_y > 1024 || det_x > 1024)
        return fail(WDD_ERR_INVALID_ARG, "n must be positive and detector sides in [1, 1024]");
    if (frame_dtype < WDD_FRAME_U16 || frame_dtype > WDD_FRAME_F64)
        return fail(WDD_ERR_INVALID_ARG, "unknown frame dtype");
    cudaPointerAttributes attr{};
    cudaError_t e = cudaPointerGetAttributes(&attr, frames);
    if (e != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    const void* src = nullptr;
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)
        src = frames;
    else if (attr.type == cudaMemoryTypeHost)
        src = attr.devicePointer ? attr.devicePointer : frames;
    else
        return fail(WDD_ERR_INVALID_ARG, "frames must be in device or pinned host memory");
    double sums[3] = {0.0, 0.0, 0.0};
    e = launch_detector_center(src, n, det_y, det_x, frame_dtype, sums,
                               static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "detector centre of mass");
    if (!(sums[0] > 0.0) || !std::isfinite(sums[0]))
        return fail(WDD_ERR_INVALID_ARG, "frames must have a positive finite total");
    *center_y = sums[1] / sums[0];
    *center_x = sums[2] / sums[0];
    return WDD_OK;
}

wdd_status wdd_get_hit_counts(const wdd_plan* P, uint32_t* host_out, int64_t n) {
    if (!P || !host_out) return fail(WDD_ERR_INVALID_ARG, "plan or output is NULL");
    if (n < P->S) return fail(WDD_ERR_INVALID_ARG, "output shorter than the scan");
    std::memcpy(host_out, P->hits.data(), sizeof(uint32_t) * P->S);
    return WDD_OK;
}

wdd_status wdd_copy_array(wdd_plan* P, int32_t which, void* dst, int64_t bytes, int64_t* written) {
    if (!P || !dst) return fail(WDD_ERR_INVALID_ARG, "plan or destination is NULL");
    const void* src = nullptr;
    size_t size = 0;
    std::vector<int32_t> host;
    switch (which) {
        case WDD_ARRAY_WEIGHTS: src = P->d_W; size = 8ull * P->S * P->K; break;
        case WDD_ARRAY_CHI:
            if (!P->d_chi) return fail(WDD_ERR_UNSUPPORTED, "chi was released (too large)");
            src = P->d_chi; size = 16ull * P->S * P->M; break;
        case WDD_ARRAY_ACCUM: {
            wdd_status s = flush(P);
            if (s != WDD_OK) return s;
            if (mirror_needed(P)) WDD_CUDA(launch_mirror_h(P, P->stream));
            src = P->d_H; size = 8ull * P->S * P->K; break;
        }
        case WDD_ARRAY_COEFF:
            src = P->d_cstage + (size_t)P->last_coeff_off * P->K;
            size = 4ull * P->last_coeff_n * P->K; break;
        case WDD_ARRAY_SPECTRUM: src = P->d_o; size = 8ull * P->S; break;
        case WDD_ARRAY_BASIS_Y: src = P->d_By; size = 16ull * P->Ny * P->Ly; break;
        case WDD_ARRAY_BASIS_X: src = P->d_Bx; size = 16ull * P->Nx * P->Lx; break;
        case WDD_ARRAY_MASK: src = P->d_mask; size = (size_t)P->S; break;
        case WDD_ARRAY_COEFF_INDEX: size = 8ull * P->K; break;
        default: return fail(WDD_ERR_INVALID_ARG, "unknown array");
    }
    if ((int64_t)size > bytes) return fail(WDD_ERR_INVALID_ARG, "destination too small");
    if (which == WDD_ARRAY_COEFF_INDEX) {
        std::memcpy(dst, P->h_ktab.data(), size);
    } else {
        if (P->stream) WDD_CUDA(cudaStreamSynchronize(P->stream));
        WDD_CUDA(cudaDeviceSynchronize());
        WDD_CUDA(cudaMemcpy(dst, src, size, cudaMemcpyDeviceToHost));
    }
    if (written) *written = (int64_t)size;
    return WDD_OK;
}

}  // extern "C"
