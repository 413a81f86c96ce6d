// Internal declarations shared by the translation units of libwdd.so.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "wdd.h"  // include/ is on the include path

namespace wdd {

// Threads per block used by most kernels.
constexpr int kThreads = 256;
// Raw frame bytes per projection row block (two blocks are double buffered in shared memory).
constexpr int kRowBlockBytes = 32 * 1024;

// Launch geometry of the projection kernel (fixed per plan except the frame-type dependent
// rows per block and the copy path).
struct ProjGeom {
    int Ny, Nx, Ly, Lx, K, CW;  // detector, basis sizes, rank, 2 for a complex basis
    int G;                      // groups of 8 basis rows (re/im counted separately)
    int P;                      // row parts of the first contraction
    int SP;                     // slices of the second contraction per coefficient
    int CS;                     // CTAs per frame (thread-block cluster size, 1..8)
    int rows_cta;               // detector rows per CTA
    int RB;                     // rows per shared-memory block
    int buf_bytes;              // bytes of one of the two row-block buffers
    int use_tma;                // 1: device frames copied by cp.async.bulk
};
// Frames per projection launch; their scan indices travel as a kernel parameter block.
constexpr int kLaunchFrames = 4096;
struct IndexBlock {
    int32_t s[kLaunchFrames];
};
// Frames of one tensor-core projection launch, possibly from several pushes: CTA b projects
// frame b - first[j] of segment j, where first[j] <= b < first[j + 1].
constexpr int kMaxSegs = 64;
// Most plans in one grouped projection launch.
constexpr int kProjGroupMax = 8;
struct FrameSegs {
    const void* ptr[kMaxSegs];
    int32_t first[kMaxSegs + 1];
    int32_t nseg;
};
// Pushes gathered for one launch (wdd_params.coalesce_frames).
struct PendingLaunch {
    FrameSegs segs{};
    IndexBlock ids{};
    int n = 0;          // frames gathered
    int slot0 = 0;      // staging slot of the first of them
};
// Pinned ring slots for host-side staging of pageable frames.
constexpr int kRingSlots = 4;

struct RingSlot {
    void* h_frames = nullptr;      // pinned, allocated on first pageable push
    cudaEvent_t done = nullptr;    // recorded after the slot's last reader
    bool used = false;
};

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace wdd

struct wdd_plan {
    wdd_params p{};
    int S = 0, Sy = 0, Sx = 0, Ny = 0, Nx = 0, K = 0, Ly = 0, Lx = 0, M = 0;
    int complex_basis = 0;   // 1 = Fourier basis (complex 1-D functions)
    int lcm = 0;             // lcm(Sy, Sx): length of the scan-phase table
    int depth = 0;           // staging depth (frames accumulated per flush)
    int max_batch = 0;
    int chunk = 0;           // frames per projection launch (<= kLaunchFrames)
    wdd::ProjGeom proj{};    // projection launch geometry
    double lambda = 0, R = 0, sigma = 0, eps_eff = 0, cy = 0, cx = 0;
    int n_active = 0;

    // FP64 plan arrays
    double2* d_By = nullptr;     // [Ny][Ly] complex (imag 0 for Hermite-Gauss)
    double2* d_Bx = nullptr;     // [Nx][Lx]
    double* d_qy = nullptr;      // [Sy] probe shift per frequency row, detector pixels
    double* d_qx = nullptr;      // [Sx]
    double2* d_chi = nullptr;    // [S][M] (freed after the plan is built unless kept)
    // FP32 streaming arrays
    float2* d_By32 = nullptr;    // [Ny][Ly] (complex, imag 0 for Hermite-Gauss)
    float2* d_Bx32 = nullptr;    // [Nx][Lx]
    int2* d_ktab = nullptr;      // [K] (flat index m, component)
    float2* d_W = nullptr;       // [S][K]
    uint8_t* d_mask = nullptr;   // [S]
    float2* d_H = nullptr;       // [S][K] accumulator
    float2* d_tw = nullptr;      // [lcm] exp(-2 pi i m / lcm)
    uint2* d_tw16 = nullptr;     // [lcm] FP16 hi/lo split of exp(-2 pi i m / lcm), packed
    float2* d_twy = nullptr;     // [Sy] exp(+2 pi i m / Sy)  (inverse DFT)
    float2* d_twx = nullptr;     // [Sx]
    float* d_cstage = nullptr;   // [depth][K] staged coefficients
    int32_t* d_idxstage = nullptr;  // [depth]
    float2* d_o = nullptr;       // [S] spectrum
    float2* d_tmp = nullptr;     // [S] inverse-DFT intermediate
    uint16_t* d_bsplit = nullptr;  // split path: FP16 hi/lo coefficients in the UMMA A layout
    float* d_scale_inv = nullptr;  // split path: [Kp] inverse power-of-two column scales
    int2* d_grp = nullptr;         // split path: [depth_pad / 16] 16-frame group records
    unsigned* d_colmax = nullptr;  // split path: [K] running max |c| per column (float bits)
    unsigned* d_status = nullptr;  // device error word (bounded waits that gave up)
    uint16_t* d_bimg = nullptr;    // tensor-core projection: FP16 hi/lo basis image (B operand)
    float* d_Byre = nullptr;       // tensor-core projection: real parts of By, [Ny * Ly] padded to 4
    float* d_Byp = nullptr;        // streaming projection: real parts of By, [Ny][LYP] zero-padded
    float* d_Bxp = nullptr;        // streaming projection: real parts of Bx, [Nx][LXP] zero-padded
    int32_t* d_kpad = nullptr;     // streaming projection: ly * LXP + lx of each coefficient
    // SEPARABLE accumulation: per-flush row slots and row DFTs
    float2* d_G = nullptr;          // [slots][Sx][K]
    int32_t* d_slotrow = nullptr;   // [slots] scan row of each slot
    int32_t* d_slotfirst = nullptr; // [slots] first / last staged frame of each slot
    int32_t* d_slotlast = nullptr;
    int32_t* d_frameslot = nullptr; // [depth_pad] slot of each staged frame
    int32_t* d_nslots = nullptr;    // [1] slots in use
    int proj_tc = 0;               // 1: projection on the tensor cores
    int proj_rows = 0;             // 1: streaming FP32 projection (wdd_project_rows.cu)
    int depth_pad = 0;             // staging depth rounded up to the split kernel's 64-frame stage
    int segment = 1024;            // split path: frames per TMEM accumulation segment
    wdd::PendingLaunch pend;       // pushes gathered for one projection launch

    // host bookkeeping (exact)
    std::vector<uint32_t> hits;
    std::vector<int32_t> h_ktab;
    int64_t frames_seen = 0;
    int64_t covered = 0;
    int staged = 0;
    int last_coeff_n = 0;
    int last_coeff_off = 0;
    bool finished = false;
    cudaStream_t stream = nullptr;
    bool stream_set = false;
    cudaEvent_t handoff = nullptr;  // orders work when the caller switches streams
    int device = 0;

    wdd::RingSlot ring[wdd::kRingSlots];
    int ring_next = 0;
    size_t frame_slot_bytes = 0;

    std::vector<wdd::DevBuf> allocs;
    int64_t device_bytes = 0;

    // launch accounting and optional per-stage event timing
    int64_t launches_total = 0;
    bool timing = false;
    struct Timed { int stage; int launches; cudaEvent_t a, b; };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
    int64_t untimed_launches[4] = {0, 0, 0, 0};
};

namespace wdd {

void set_error(const std::string& msg);
// Raises the dynamic shared-memory limit of every kernel once per process (not per launch, so
// launches stay legal inside stream capture).
cudaError_t prepare_kernels();
// Sets a kernel's dynamic shared-memory limit to the device opt-in maximum minus its static use.
cudaError_t allow_max_dynamic_smem(const void* func);
cudaError_t prepare_project_kernels();
cudaError_t prepare_reconstruct_kernels();
cudaError_t prepare_split_kernels();
size_t frame_elem_bytes(int dtype);

// ---- plan kernels (FP64) -----------------------------------------------------------------
cudaError_t launch_hg_basis(double2* B, int n, int L, double sigma, double center, cudaStream_t st);
cudaError_t launch_fourier_basis(double2* B, int n, double center, cudaStream_t st);
cudaError_t launch_chi(const wdd_plan* P, unsigned long long* d_maxbits, cudaStream_t st);
// Sum of all frame values and the row- and column-weighted sums (frames readable by the device,
// n >= 1); synchronises `st`.
cudaError_t launch_detector_center(const void* frames, int64_t n, int Ny, int Nx, int dtype,
                                   double sums[3], cudaStream_t st);
cudaError_t launch_weights(const wdd_plan* P, cudaStream_t st);
cudaError_t launch_tables(const wdd_plan* P, cudaStream_t st);

// ---- streaming kernels ---------------------------------------------------------------------
ProjGeom make_proj_geom(int Ny, int Nx, int Ly, int Lx, int K, int complex_basis,
                        int frames_per_launch, int cluster);
void proj_set_frame_bytes(ProjGeom& g, int elem_bytes);  // RB and buffer size for a frame type
size_t proj_smem_bytes(const ProjGeom& g);
// `overlap`: launch with programmatic stream serialization (see the projection kernel).
cudaError_t launch_project(const wdd_plan* P, const void* frames, int dtype, int n,
                           bool device_src, bool overlap, const IndexBlock& idx, float* c_out,
                           int32_t* idx_out, cudaStream_t st);  // also folds |c| into d_colmax
// Tensor-core projection (split precision, real basis, uint16/float32 frames, Nx % 16 == 0).
bool proj_tc_supported(int Nx, int Lx, int complex_basis, int frame_dtype);
size_t proj_tc_smem_bytes(int Ny, int Nx, int Ly, int Lx, int K);
size_t proj_tc_bimg_halves(int Nx, int Lx);
cudaError_t prepare_project_tc_kernels();
cudaError_t launch_build_bimg(const wdd_plan* P, uint16_t* img, cudaStream_t st);
cudaError_t launch_project_tc(const wdd_plan* P, const FrameSegs& segs, int dtype, int n,
                              bool overlap, const IndexBlock& idx, float* c_out, int32_t* idx_out,
                              cudaStream_t st);
// Streaming FP32 projection (real basis, L_y <= 16, uint16/float32 frames, N_x % 4 == 0).
bool proj_rows_supported(int Ny, int Nx, int Ly, int Lx, int K, int complex_basis, int frame_dtype);
// Padded basis widths of the streaming projection: By is stored [Ny][proj_rows_lyp(Ly)] and Bx
// [Nx][proj_rows_lxp(Lx)], zero beyond Ly / Lx.
int proj_rows_lyp(int Ly);
int proj_rows_lxp(int Lx);
cudaError_t prepare_project_rows_kernels();
cudaError_t launch_project_rows(const wdd_plan* P, const FrameSegs& segs, int dtype, int n,
                                bool overlap, const IndexBlock& idx, float* c_out,
                                int32_t* idx_out, cudaStream_t st);
// Plans whose gathered pushes may share one grouped projection launch have equal classes.
int proj_rows_class(const wdd_plan* P);
// One launch projecting the gathered pushes of several streaming-projection plans of one class
// (at most kProjGroupMax plans, kLaunchFrames frames and kMaxSegs pushes in all); each plan's
// coefficients go to its own staging slots.  Leaves the plans' pending lists unchanged.
cudaError_t launch_project_rows_group(wdd_plan* const* plans, int count, cudaStream_t st);
// Row-factorised accumulation (SEPARABLE mode).
int rows_slots(int Sy, int depth_pad);   // slots a flush of depth_pad frames can need
cudaError_t prepare_rows_kernels();
cudaError_t launch_accumulate_rows(const wdd_plan* P, const float* c, const int32_t* idx, int n,
                                   cudaStream_t st);
cudaError_t launch_accumulate_fp32(const wdd_plan* P, const float* c, const int32_t* idx, int n,
                                   cudaStream_t st);
// Device-side waits give up after this long and report WDD_ERR_TIMEOUT.
constexpr uint64_t kDeviceWaitNs = 2000000000ull;
bool split_path_available();
int split_tile_n(int K);
size_t split_smem_bytes(int NT);
// Scan columns the tensor-core accumulation computes (S_x / 2 + 1 when S_x > 2): the split path
// accumulates only these and mirrors the rest (H[-v] = conj H[v]) before H is read.
int spectrum_cols(int Sx);
bool mirror_needed(const wdd_plan* P);
int accum_kernel_of(const wdd_plan* P);   // wdd_accum_kernel
cudaError_t launch_mirror_h(const wdd_plan* P, cudaStream_t st);
size_t split_coeff_bytes(int K, int depth_pad);   // bytes of the split coefficient operand
int split_launch_count(int n, int segment);       // kernel launches of a flush of n frames
cudaError_t launch_bounded_wait_selftest(unsigned* status, uint64_t wait_ns, cudaStream_t st);
cudaError_t launch_accumulate_split(const wdd_plan* P, const float* c, const int32_t* idx, int n,
                                    cudaStream_t st);
// One split pre-pass and one accumulation launch over the staged frames of several split plans.
int accumulate_group_max();
cudaError_t launch_accumulate_group(wdd_plan* const* plans, int count, cudaStream_t st);
cudaError_t launch_deconvolve(const wdd_plan* P, cudaStream_t st);
cudaError_t launch_inverse_dft(const wdd_plan* P, float2* obj, float* phase, cudaStream_t st);
// The normalisation and conjugated inverse DFT of Eq. 3 on any spectrum o [Sy][Sx] (tmp: [S]
// scratch; twy/twx: exp(+2 pi i m / n) tables written by launch_idft_tables).
cudaError_t launch_idft_tables(float2* twy, int Sy, float2* twx, int Sx, cudaStream_t st);
cudaError_t launch_idft(const float2* o, const float2* twx, const float2* twy, float2* tmp, int Sy,
                        int Sx, float2* obj, float* phase, cudaStream_t st);

// ---- host geometry shared by the live and the classical plans (Sect. 6.2) -------------------
double electron_wavelength(double volts);
// Probe shift per scan frequency (detector pixels along the scan axes) and the overlap mask
// |q_v| < 2 R (Eq. 15, strict); returns the number of active frequencies.
int scan_geometry(const wdd_params& p, double R, std::vector<double>& qy, std::vector<double>& qx,
                  std::vector<uint8_t>& mask);

// Reconstruction that allocates nothing (see wdd_reconstruct_noalloc): the device address of the
// file-scope scratch array for `device` (resolved on first use), its size, and the launcher.
cudaError_t noalloc_scratch(int device, void** out);
size_t noalloc_scratch_limit();
cudaError_t launch_reconstruct_noalloc(void* scratch, const float2* W, const float2* H, int Sy,
                                       int Sx, int K, float2* obj, float* phase, cudaStream_t st);

}  // namespace wdd
