/*
 * wdd.h -- C ABI of the GB300 live Wigner Distribution Deconvolution library (libwdd.so).
 *
 * The library reconstructs the object transfer function of a 4D-STEM scan while the frames
 * stream in (live WDD, Sect. 6 of Bangun et al., arXiv 2212.01309):
 *
 *   plan    (Algorithm 1)  reduced detector basis P, probe autocorrelation Y_v for every scan
 *                          frequency v, chi_v = P vec(Y_v), Wiener filter
 *                          W_v = conj(chi_v) / (|chi_v|^2 + eps_eff), active-frequency mask
 *                          (Sect. 6.2, Eq. 15).  Built once, in FP64 on the GPU.
 *   push    (Algorithm 2)  per frame: c_s = P vec(I_s) (Sect. 5, operator H of Eq. 12), then
 *                          H[v,k] += exp(-2 pi i (v_y s_y / S_y + v_x s_x / S_x)) c_s[k]
 *                          (Eq. 14: partial sums of F_2D I over the frames at hand).
 *   snapshot / finalize    o_v = sum_k W_v[k] H[v,k]  (Hadamard product with K_v and sum of all
 *                          elements, Algorithm 2), o <- o / sqrt(o_0) (Eq. 3), and
 *                          O = conj(IFFT2(o)) (Algorithm 2, last step), at any time in the scan.
 *
 * Every entry point returns a wdd_status; WDD_OK is 0.  On any error nothing is enqueued on the
 * GPU and the plan's state is unchanged; wdd_last_error() returns a one-line explanation
 * (thread-local, valid until the next call on the same thread).
 *
 * Threading: a plan may be used by one host thread at a time.  Different plans are independent.
 * Memory: a plan owns all its device buffers; callers own frames and result buffers.
 */
#ifndef WDD_H
#define WDD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle (cudaStream_t) passed as an opaque pointer; NULL = legacy default stream. */
typedef void* wdd_stream_t;

typedef enum {
    WDD_OK = 0,
    WDD_ERR_INVALID_ARG = 1,   /* a pointer is NULL, a size is out of range, a flag is unknown */
    WDD_ERR_OUT_OF_MEMORY = 2, /* device allocation failed or would exceed hbm_budget_bytes */
    WDD_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in wdd_last_error) */
    WDD_ERR_SCAN_INDEX = 4,    /* a scan index is outside [0, scan_y * scan_x) */
    WDD_ERR_STATE = 5,         /* push after finalize, or use of a destroyed plan */
    WDD_ERR_TIMEOUT = 6,       /* a bounded wait gave up */
    WDD_ERR_UNSUPPORTED = 7    /* a valid request the library cannot serve (sizes, basis, dtype) */
} wdd_status;

/* Reduced detector bases.
 *  FOURIER_FULL  K = det_y * det_x real cos/sin rows of the detector inverse DFT.  Live WDD with
 *                this basis equals classical WDD (Eq. 2, Eq. 3) exactly.  det_y, det_x <= 64.
 *  HG_TENSOR     the operator H of Sect. 5: L x L Hermite-Gauss functions (Eq. 7), K = L * L.
 *  HG_ENERGY     the first K tensor pairs (n_y, n_x) ordered by oscillator energy n_y + n_x
 *                (Eq. 10), ties broken by smaller n_y; L is the smallest that holds them.
 * Hermite-Gauss width: sigma = R_bf / sqrt(2 (L - 1) + 1), R_bf = semiconv / (lambda * dk)
 * pixels, sampled at x_j = j - det_center; each column has unit discrete L2 norm. */
typedef enum { WDD_BASIS_FOURIER_FULL = 0, WDD_BASIS_HG_TENSOR = 1, WDD_BASIS_HG_ENERGY = 2 } wdd_basis;

/* Arithmetic of the streaming steps.
 *  FP32   projection and phase accumulation in FP32 FMA on the SIMT cores.
 *  SPLIT  tensor cores: phase factors and coefficients split into hi + lo FP16 parts, the
 *         hi*hi, hi*lo and lo*hi products accumulated in FP32 (the lo*lo term lies below FP32
 *         rounding); frames and the projection basis likewise on the tensor cores where the
 *         frame type and detector width allow (see wdd_plan_info.proj_tensor).  Staged frames
 *         are accumulated accum_depth at a time, in TMEM segments of accum_segment frames. */
typedef enum { WDD_PREC_FP32 = 0, WDD_PREC_SPLIT = 1 } wdd_precision;

/* How staged frames are added into the accumulator H.
 *  DIRECT     H[v, k] += sum_s F_2D[v, s] c_s[k] over every scan frequency v for every frame
 *             (Eq. 14, Algorithm 2): 4 S K flops per frame, on the tensor cores (SPLIT) or the
 *             SIMT cores (FP32).
 *  SEPARABLE  the scan DFT factorised by scan rows (not in the paper): for each scan row s_y
 *             touched by the staged frames, G[v_x, k] = sum over its frames of
 *             exp(-2 pi i v_x s_x / S_x) c_s[k], then H[(v_y, v_x), k] +=
 *             sum over rows of exp(-2 pi i v_y s_y / S_y) G_{s_y}[v_x, k].  The same H up to
 *             rounding, in 4 S_x K flops per frame plus 8 S K per touched row (64x fewer at a
 *             128 x 128 scan in raster order); FP32 on the SIMT cores for either precision. */
typedef enum { WDD_ACCUM_DIRECT = 0, WDD_ACCUM_SEPARABLE = 1 } wdd_accum_mode;

/* Element type of the frames passed to wdd_push_frames. */
typedef enum { WDD_FRAME_U16 = 0, WDD_FRAME_F32 = 1, WDD_FRAME_F64 = 2 } wdd_frame_dtype;

typedef struct {
    int32_t scan_y, scan_x;   /* scan grid S_y x S_x; position s = s_y * scan_x + s_x        */
    double scan_step_m;       /* scan step Delta in metres (equal on both axes, Sect. 6.2)     */
    int32_t det_y, det_x;     /* detector pixels N_y x N_x                                     */
    double det_px_inv_m;      /* detector sampling dk in reciprocal metres per pixel           */
    double voltage_v;         /* acceleration voltage (sets lambda, relativistic)              */
    double semiconv_rad;      /* semiconvergence angle theta                                   */
    double defocus_m;         /* probe defocus df: p(k) = A(k) exp(-i pi lambda df |k|^2)      */
    double epsilon;           /* Wiener epsilon (relative unless eps_absolute)                 */
    int32_t rank_k;           /* reduced rank K                                                */
    int32_t basis;            /* wdd_basis                                                     */
    int32_t precision;        /* wdd_precision                                                 */
    int32_t frame_dtype;      /* wdd_frame_dtype                                               */
    int32_t max_batch;        /* most frames per internal launch (at most 4096); larger pushes
                                 are split                                                     */
    int32_t accum_depth;      /* frames staged before the phase accumulation runs; 0 = every
                                 push is accumulated at once (the plain path)                  */
    double det_center_y;      /* detector zero-frequency pixel; negative = det_y / 2 (integer) */
    double det_center_x;
    int32_t eps_absolute;     /* 1: eps_eff = epsilon; 0: eps_eff = epsilon * max |chi|^2     */
    int32_t proj_cluster;     /* CTAs per frame in the projection (1, 2, 4 or 8); 0 = automatic */
    int64_t hbm_budget_bytes; /* refuse plans whose device footprint exceeds this; 0 = none   */
    int32_t overlap_pushes;   /* 1: a push's first projection may start before the previous
                                 kernel on the stream has finished (programmatic dependent
                                 launch).  Set it only when no kernel that produces the frames
                                 runs on the stream right before a push, e.g. frames written by
                                 a detector DMA or by copies.  Later chunks of one push always
                                 overlap (their predecessor is the push's own projection). */
    int32_t accum_segment;    /* SPLIT: staged frames summed in the tensor cores' FP32 accumulators
                                 before they are added into H in FP32 (rounded up to a multiple
                                 of 64; all segments of a flush run in one launch).  The
                                 accumulator error grows linearly with the segment (relative
                                 3.2e-7 at 256 frames, 7.6e-7 at 1024, 3.8e-6 at 4096 on a
                                 128x128 scan); longer segments run slightly faster.  0 = 1024. */
    int32_t accum_mode;       /* wdd_accum_mode: how staged frames are added into H            */
    int32_t coalesce_frames;  /* tensor-core and streaming projections: device or pinned-host pushes are gathered
                                 until this many frames are pending (at most 4096, from at most 64
                                 pushes) and projected in one launch.  The caller must then keep a
                                 push's frames unchanged until the plan's next wdd_flush,
                                 wdd_snapshot, wdd_finalize, wdd_reset or wdd_set_stream, or until
                                 wdd_plan_info reports pending == 0.  0 = every push is projected
                                 when it is made. */
    double scan_rotation_rad; /* scan axes against the detector axes (the rotation of Tables 2
                                 and 3): a scan frequency (q_y, q_x) along the scan axes shifts
                                 the probe by (q_y cos - q_x sin, q_y sin + q_x cos) on the
                                 detector, so +pi/2 matches detector images turned a quarter
                                 turn as numpy's rot90 over the detector axes does.  0 = aligned. */
    int32_t proj_engine;      /* wdd_proj_engine: which kernel projects the frames (SPLIT plans;
                                 FP32 plans always use WDD_PROJ_SIMT)                          */
} wdd_params;

/* Projection kernels (wdd_params.proj_engine, reported in wdd_plan_info.proj_engine).
 *  AUTO    SPLIT plans: STREAM where it applies, else TENSOR, else SIMT; FP32 plans: SIMT.
 *  TENSOR  T = I Bx on the tensor cores with FP16 hi/lo splits of frame and basis, then
 *          By^T T on the SIMT cores (real basis, uint16/float32 frames, det_x a multiple of
 *          16).
 *  SIMT    FP32 on the SIMT cores, frames staged in shared memory (any basis and frame type).
 *  STREAM  FP32 on the SIMT cores, one warp per frame (teams of det_x / 128 warps for wider
 *          detectors), each lane streaming four detector columns down the rows with coalesced
 *          loads and the second contraction combined across lanes by shuffles (real basis with
 *          at most 16 functions per axis and K <= 256, uint16/float32 frames, det_x a multiple
 *          of 4 from 16 to 512): the projection reads each frame byte once and does about
 *          2 L_y flops per pixel, so it is bound by the frame read.  A requested engine that
 *          does not apply falls back as AUTO does. */
typedef enum {
    WDD_PROJ_AUTO = 0,
    WDD_PROJ_TENSOR = 1,
    WDD_PROJ_SIMT = 2,
    WDD_PROJ_STREAM = 3
} wdd_proj_engine;

/* Fills *p with defaults: FP32, HG_TENSOR, F32 frames, max_batch 256, accum_depth 0, centre at
 * N/2, relative epsilon 1e-3, no overlap across pushes, accum_segment 0 (1024), no scan
 * rotation.  Geometry fields are zeroed and must be
 * set by the caller. */
wdd_status wdd_params_default(wdd_params* p);

typedef struct wdd_plan wdd_plan;

/* Builds a plan (Algorithm 1 and the initialisation of Algorithm 2): bases, Wiener filter and
 * mask in FP64 on the current CUDA device, then zeroes the accumulator.  Blocks until the plan
 * is built.  *out receives the plan (owned by the library, freed by wdd_plan_destroy).
 * Errors: INVALID_ARG (NULL, non-positive sizes, rank not matching the basis, L > 32,
 * epsilon < 0), UNSUPPORTED (FOURIER_FULL with a detector side > 64, det side > 1024),
 * OUT_OF_MEMORY, CUDA. */
wdd_status wdd_plan_create(const wdd_params* p, wdd_plan** out);

/* Validates *p exactly as wdd_plan_create does and reports in *bytes the device memory such a
 * plan would hold, without touching the GPU (admission control by memory budget).  Returns the
 * status wdd_plan_create would return for these parameters (memory-independent errors only). */
wdd_status wdd_plan_footprint(const wdd_params* p, int64_t* bytes);

/* Releases every device and host buffer of the plan (synchronises with its last stream). */
wdd_status wdd_plan_destroy(wdd_plan* plan);

/* Wiener filter update from a recovered probe (Sect. 10): rebuilds chi_v, eps_eff and the
 * weights of Algorithm 1 with Y_v(q) = A(q) conj A(q + q_v), A(k) = [|k| <= theta / lambda]
 * exp(i arg P(k)), P(k) = sum_s probe_s exp(-2 pi i dk k . r_s) the spectrum of `probe` at
 * detector-pixel frequencies: the condenser aperture is kept, the recovered probe gives the
 * phase inside it.  `probe` is complex64 [scan_y][scan_x] on the scan grid with its origin at
 * index 0 (the out->obj of wdd_offline_reconstruct on a probe plan), in device or pinned host
 * memory, read during the call only.  The accumulator and the counters are kept, so the next
 * snapshot deconvolves every frame pushed so far with the updated filter; this includes a
 * finalized plan, whose acquisition is complete (wdd_snapshot still reconstructs it).
 * Synchronous: waits for all queued device work first and returns when the weights are
 * rebuilt.  Errors: INVALID_ARG (NULL or pageable probe, an autocorrelation that is zero
 * everywhere), UNSUPPORTED (scan_rotation_rad != 0, bases too large), OUT_OF_MEMORY, CUDA; on
 * an error after the weights were started they are undefined. */
wdd_status wdd_plan_set_probe(wdd_plan* plan, const void* probe);

/* Streams n frames into the plan (the loop body of Algorithm 2).
 *  frames    n x det_y x det_x elements of frame_dtype, row-major, zero frequency at
 *            (det_center_y, det_center_x) (i.e. fftshifted).  Device memory, pinned host memory
 *            (read by the kernels directly over the host link) or pageable host memory (copied
 *            through a plan-owned pinned ring).  Borrowed: it must stay valid and unchanged
 *            until `stream` has passed this push.
 *  scan_idx  n int32 scan positions s in [0, S), host memory, read before the call returns.
 *            Duplicate positions accumulate (the method is linear in the frames).
 *  stream    CUDA stream the work is enqueued on; the plan remembers it for snapshots.
 * Returns immediately after enqueuing.  Errors: INVALID_ARG, SCAN_INDEX (nothing enqueued,
 * counters unchanged), STATE (plan finalized), CUDA. */
wdd_status wdd_push_frames(wdd_plan* plan, const void* frames, const int32_t* scan_idx,
                           int64_t n, wdd_stream_t stream);

typedef struct {
    void* obj;                  /* in: device buffer, complex64 [scan_y][scan_x] (re, im)    */
    float* phase;               /* in: device buffer f32 [scan_y][scan_x] or NULL             */
    int64_t frames_seen;        /* out: frames pushed so far (host count, exact)              */
    int64_t positions_covered;  /* out: scan positions with at least one frame                */
} wdd_result;

/* Reconstructs from every frame pushed so far (Algorithm 2 after any number of iterations):
 * deconvolution, normalisation by sqrt(o_0) (principal root; skipped while o_0 == 0), conjugated
 * inverse FFT (numpy ifft2 normalisation 1/S) and phase = atan2(im, re).  Enqueued on the
 * plan's last stream; out->obj and out->phase are written in stream order.  The plan continues
 * to accept frames.  Errors: INVALID_ARG (out or out->obj NULL), STATE, CUDA. */
wdd_status wdd_snapshot(wdd_plan* plan, wdd_result* out);

/* As wdd_snapshot, then marks the plan finished: later pushes return WDD_ERR_STATE.  An
 * incomplete scan is not an error; positions_covered reports the coverage. */
wdd_status wdd_finalize(wdd_plan* plan, wdd_result* out);

/* Accumulates the frames staged so far (Algorithm 2 loop body for them) on the plan's stream.
 * After it, a snapshot enqueues only the deconvolution and the inverse DFT, a fixed sequence of
 * launches that can be captured once in a CUDA graph and replayed. */
wdd_status wdd_flush(wdd_plan* plan);

/* wdd_flush for several plans at once.  The pushes the plans have gathered (coalesce_frames) are
 * projected (Eq. 12) by shared launches: streaming-projection plans with equal frame type and
 * basis width share one launch of up to 4096 frames from up to 64 pushes; other plans project
 * their own.  Then the frames staged by every plan are accumulated (the sum of Eq. 14 over each
 * plan's frames, Sect. 6.3) by one coefficient-split launch and one tensor-core accumulation
 * launch whose CTAs cover all the plans' tiles, instead of two launches per plan.  This is how a
 * server that holds many small sessions keeps the GPU's SMs filled: each session alone stages too
 * few frames and frequency tiles to occupy them.
 *  plans   count distinct plans, host array.  Every plan must use precision SPLIT with the
 *          direct accumulation (accum_mode DIRECT), be unfinished, and belong to the device
 *          that is current.
 *  count   1 .. wdd_flush_group_max().
 *  stream  every plan's stream becomes `stream` (as wdd_set_stream); their gathered pushes are
 *          projected and the accumulation runs on it.
 * Plans with nothing staged are skipped.  Each shared launch is counted, and timed when timing
 * is on, on the first plan it serves.  Results equal those of wdd_flush on each plan.
 * Errors: INVALID_ARG (NULL or repeated plan, count out of range, a plan not SPLIT/DIRECT;
 * nothing enqueued), STATE (a plan finalized; nothing enqueued), CUDA. */
wdd_status wdd_flush_group(wdd_plan* const* plans, int32_t count, wdd_stream_t stream);

/* Most plans one wdd_flush_group call takes. */
int32_t wdd_flush_group_max(void);

/* Sets the stream on which the plan's next snapshot, finalize or reset is enqueued (pushes set
 * it too).  Work already enqueued on the previous stream is ordered before later work on the
 * new one. */
wdd_status wdd_set_stream(wdd_plan* plan, wdd_stream_t stream);

/* Zeroes the accumulator, the staged frames and the hit counters so the plan can take a new
 * acquisition with the same geometry (the Wiener filter is kept).  Enqueued on the plan's last
 * stream.  Clears the finished state. */
wdd_status wdd_reset(wdd_plan* plan);

typedef struct {
    int32_t rank_k;          /* K                                                            */
    int32_t basis_ly;        /* basis functions along detector rows (L_y)                    */
    int32_t basis_lx;        /* along detector columns (L_x)                                 */
    int32_t n_active;        /* active scan frequencies (Sect. 6.2 overlap criterion)        */
    double eps_eff;          /* epsilon actually added to |chi|^2                            */
    double wavelength_m;     /* lambda                                                       */
    double bf_radius_px;     /* bright-field radius R_bf in detector pixels                  */
    double hg_sigma_px;      /* Hermite-Gauss sigma (0 for the Fourier basis)                */
    int64_t device_bytes;    /* device memory held by the plan                               */
    int64_t frames_seen;
    int64_t positions_covered;
    int64_t kernel_launches; /* hot-path kernel launches since the plan was created          */
    int32_t staged;          /* frames projected but not yet accumulated                     */
    int32_t finished;
    int32_t proj_tensor;     /* 1: frames are projected on the tensor cores (proj_engine
                                TENSOR); 0: on the SIMT cores in FP32                         */
    int32_t accum_mode;      /* wdd_accum_mode of the plan                                   */
    int32_t pending;         /* frames gathered for a projection launch (coalesce_frames)    */
    int32_t proj_engine;     /* wdd_proj_engine the plan projects with (never AUTO)          */
    int32_t accum_kernel;    /* wdd_accum_kernel the plan's flushes run                      */
    int32_t spectrum_cols;   /* scan columns the accumulation computes: S_x / 2 + 1 on the
                                SPLIT direct path (the rest of H follows from H[-v] =
                                conj H[v], Eq. 14 with real coefficients, filled before H is
                                read), else S_x                                              */
} wdd_plan_info;

/* Accumulation kernels (wdd_plan_info.accum_kernel): FP32 SIMT (FP32 plans), the row-factorised
 * SIMT kernels (SEPARABLE), and the tensor-core kernels of the SPLIT path: 128 scan frequencies
 * x 64 coefficients per CTA (K <= 64 on scans large enough to fill the GPU), the stacked kernel
 * with 128 coefficients per CTA (K > 64), and with 64 (K <= 64 on smaller scans). */
typedef enum {
    WDD_ACCUM_KERNEL_FP32 = 0,
    WDD_ACCUM_KERNEL_SEPARABLE = 1,
    WDD_ACCUM_KERNEL_NARROW = 2,
    WDD_ACCUM_KERNEL_STACKED128 = 3,
    WDD_ACCUM_KERNEL_STACKED64 = 4
} wdd_accum_kernel;

/* Reports the plan's derived constants and counters (host-side, no GPU work). */
wdd_status wdd_plan_get_info(const wdd_plan* plan, wdd_plan_info* out);

/* Hot-path stages, for wdd_get_stage_times. */
typedef enum {
    WDD_STAGE_PROJECT = 0,     /* frame ingest + projection (one launch per internal batch)  */
    WDD_STAGE_ACCUMULATE = 1,  /* phase accumulation (one launch per flush)                   */
    WDD_STAGE_DECONVOLVE = 2,  /* Wiener deconvolution (one launch per snapshot)              */
    WDD_STAGE_IDFT = 3,        /* inverse DFT + phase (two launches per snapshot)             */
    WDD_STAGE_COUNT = 4
} wdd_stage;

/* Enables (1) or disables (0) CUDA-event timing of every hot-path launch on the plan's stream.
 * Timing adds two event records per launch; it is off by default. */
wdd_status wdd_set_stage_timing(wdd_plan* plan, int32_t enable);

/* Synchronises the plan's stream, then reports per stage the summed device time (ms) and the
 * number of kernel launches timed since the previous call, and clears them.  ms_out and
 * launches_out each hold WDD_STAGE_COUNT entries (either may be NULL). */
wdd_status wdd_get_stage_times(wdd_plan* plan, double* ms_out, int64_t* launches_out);

/* Synchronises the plan's stream and reports whether any of its kernels gave up a bounded
 * device wait (tensor-core pipeline barriers wait at most ~2 s).  Returns WDD_ERR_TIMEOUT and
 * clears the flag if one did; the CUDA context stays usable and the accumulator must be
 * considered invalid (wdd_reset).  Returns WDD_ERR_UNSUPPORTED (and clears the flag) when the
 * tensor-core projection met a float32 frame value at or above the FP16 overflow threshold
 * (|I| >= 65520) or a non-finite one, outside the range of its FP16
 * hi/lo split; the coefficients of that frame are then invalid. */
wdd_status wdd_check_device(wdd_plan* plan);

/* Runs the library's bounded device wait on a barrier that nothing completes, with a limit of
 * wait_ns nanoseconds (1 .. 1e10).  Returns WDD_ERR_TIMEOUT when the wait gave up as designed
 * (the expected result), WDD_OK if it did not, WDD_ERR_CUDA on a CUDA error. */
wdd_status wdd_selftest_bounded_wait(int64_t wait_ns);

/* Reconstruction for callers that must not allocate device memory.
 *
 * The paper has no counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc: code that runs while a CUDA graph is being captured (allocation is not a legal
 * stream-capture operation), real-time acquisition threads that must not block on the
 * allocator (which may synchronise the whole device), and applications whose device memory is
 * fixed up front by a memory pool or budget that this library must not grow.
 *
 * It computes the same result as wdd_snapshot from a plan's Wiener weights and accumulator:
 * o_v = sum_k W_v[k] H[v,k], O = conj(IFFT2(o / sqrt(o_0))) (numpy ifft2 normalisation),
 * phase = atan2(Im O, Re O), with the same kernels.  The caller passes everything:
 *   weights  device complex64 [scan_y * scan_x][rank_k] (W, e.g. read with WDD_ARRAY_WEIGHTS)
 *   accum    device complex64 [scan_y * scan_x][rank_k] (H, e.g. WDD_ARRAY_ACCUM)
 *   obj      device complex64 [scan_y][scan_x] output;  phase: device f32 [scan_y][scan_x] or NULL
 * Its working memory (spectrum, inverse-DFT intermediate, twiddle tables: 16 S + 8 (S_y + S_x)
 * bytes) lives in a fixed 8 MiB array compiled into the library, held on every GPU that loads
 * it until the process exits; scans needing more (above about 524,000 positions) are rejected
 * with WDD_ERR_INVALID_ARG before anything is enqueued.
 * The first call on each device resolves the array's device address (cudaGetSymbolAddress)
 * and keeps it for the life of the process; make that first call before any stream capture.
 * Resetting a device (cudaDeviceReset) after that call is not supported: the kept address would
 * no longer belong to the new context.  All calls share the one array and every call
 * writes all of the scratch it reads, so nothing needs clearing, but calls whose work may
 * overlap on the GPU (different streams without ordering) race on it.
 * Errors: INVALID_ARG (NULL, sizes, scratch too small), CUDA. */
wdd_status wdd_reconstruct_noalloc(const void* weights, const void* accum, int32_t scan_y,
                                   int32_t scan_x, int32_t rank_k, void* obj, float* phase,
                                   wdd_stream_t stream);

/* Copies the per-position hit counts (uint32 [S], exact host bookkeeping) into host memory. */
wdd_status wdd_get_hit_counts(const wdd_plan* plan, uint32_t* host_out, int64_t n);

/* Adds an exported state to the plan (checkpoint/resume and partition merge): Eq. 14 is linear
 * in the frames, so the accumulator of a set of frames is the sum of the accumulators of any
 * partition of it (the merge by summation of Sect. 6.3).  accum: complex64 [S][K] in device or
 * pinned host memory (read with wdd_copy_array(WDD_ARRAY_ACCUM) from a plan with the same
 * parameters), borrowed until the plan's stream has passed the merge; hits: host uint32 [S]
 * (wdd_get_hit_counts), summing to frames_seen, read before the call returns.  Adds accum to the
 * accumulator (one kernel enqueued on the plan's last stream, after everything the plan has
 * enqueued; nothing is allocated and nothing else is waited for), hits to the hit counters and
 * frames_seen to the frame count; merged into a freshly created (or reset) plan it resumes the
 * acquisition exactly.  Errors: INVALID_ARG (NULL pointers, pageable accum, a negative
 * frames_seen, hits that do not add up to frames_seen, a counter that would overflow), STATE (a
 * finalized plan: wdd_reset it first), CUDA; on an error nothing is enqueued and the counters
 * are unchanged. */
wdd_status wdd_merge_state(wdd_plan* plan, const void* accum, const uint32_t* hits,
                           int64_t frames_seen);

/* Internal arrays that wdd_copy_array can read back (tests and diagnostics). */
typedef enum {
    WDD_ARRAY_WEIGHTS = 0,   /* complex64 [S][K]   W_v[k] (zero rows for inactive v)           */
    WDD_ARRAY_CHI = 1,       /* complex128 [S][M]  chi_v[m] = H(Y_v), M = L_y * L_x (FP64)      */
    WDD_ARRAY_ACCUM = 2,     /* complex64 [S][K]   H[v][k] accumulated so far (staged frames
                                                   are flushed first)                         */
    WDD_ARRAY_COEFF = 3,     /* float32 [n][K]     coefficients c of the most recent push's
                                                   last internal launch (n = its frame count) */
    WDD_ARRAY_SPECTRUM = 4,  /* complex64 [S]      o_v of the most recent snapshot            */
    WDD_ARRAY_BASIS_Y = 5,   /* float64 [N_y][L_y] (complex128 for FOURIER_FULL)               */
    WDD_ARRAY_BASIS_X = 6,   /* float64 [N_x][L_x] (complex128 for FOURIER_FULL)               */
    WDD_ARRAY_MASK = 7,      /* uint8 [S]          1 = active frequency                        */
    WDD_ARRAY_COEFF_INDEX = 8 /* int32 [K][2]      (flat basis index m, 0 = real / 1 = imag)   */
} wdd_array;

/* Synchronously copies an internal array into host memory.  `bytes` must be at least the
 * array's size; *written receives the bytes copied.  Errors: INVALID_ARG, CUDA. */
wdd_status wdd_copy_array(wdd_plan* plan, int32_t which, void* host_dst, int64_t bytes,
                          int64_t* written);

/* Centre of mass of n detector frames (row, column, in pixels): sum over frames and pixels of
 * I[i][j] (i, j) / sum of I, accumulated in FP64 in a fixed order (bit-reproducible).  This is
 * the data-estimated centre of the basis sampling grid (Sect. 5 samples the Hermite-Gauss
 * functions around the centre of mass); pass it as det_center_y / det_center_x to
 * wdd_plan_create.  frames: n x det_y x det_x values of frame_dtype, row-major, in device or
 * pinned host memory (read in place), borrowed for the call.  Runs on `stream` and returns when
 * the result is on the host; allocates a small scratch buffer.  Errors: INVALID_ARG (NULL
 * pointers, n < 1, sizes out of range, pageable frames, a total that is not positive), CUDA. */
wdd_status wdd_detector_center(const void* frames, int64_t n, int32_t det_y, int32_t det_x,
                               int32_t frame_dtype, double* center_y, double* center_x,
                               wdd_stream_t stream);

/* ---- Classical (offline) WDD on the whole 4-D dataset (Eq. 2 and 3) --------------------------
 * The method live WDD reformulates, run on the GPU for comparison and validation:
 *   G(v, q)  = forward FFT over both scan axes of I_s(q)                         (Eq. 2)
 *   W_O(v,r) = IFFT_q(ifftshift_q G(v, .)) conj(W_P) / (|W_P|^2 + eps_eff),
 *              W_P = IFFT_q(ifftshift_q Y_v), Y_v(q) = p(q) conj p(q + q_v)       (Eq. 2)
 *   o_v      = sum_r W_O(v, r) (F_r(W_O) at q = 0), 0 for inactive v             (Eq. 3)
 * then the normalisation by sqrt(o_0) and conjugated inverse DFT of wdd_snapshot.  Inverse
 * transforms carry numpy's 1/(N_y N_x) factor; eps_eff = epsilon * max_{v,r} |W_P|^2 unless
 * eps_absolute.  FP32 transforms (twiddles built in FP64), Y_v in FP64.
 * Parameters used: scan_y, scan_x, scan_step_m, det_y, det_x, det_px_inv_m, voltage_v,
 * semiconv_rad, defocus_m, epsilon, eps_absolute, frame_dtype, scan_rotation_rad,
 * hbm_budget_bytes; the detector centre must be the default det / 2 (the zero frequency moves to
 * pixel 0 by an integer roll).  Other fields are ignored.  Device memory: two complex64
 * [S][det_y][det_x] arrays (the scan spectrum and the Wiener kernel) plus O(S). */
typedef struct wdd_offline_plan wdd_offline_plan;

/* Builds the Wiener kernel for every scan frequency (synchronous).  Errors: INVALID_ARG,
 * UNSUPPORTED (detector centre not det / 2, sizes), OUT_OF_MEMORY (budget or allocation), CUDA. */
wdd_status wdd_offline_plan_create(const wdd_params* p, wdd_offline_plan** out);
/* Probe reconstruction (Sect. 10): a classical plan with the roles of probe and object swapped.
 * The Wiener kernel is built from an object estimate `obj` (complex64 [scan_y][scan_x], e.g. the
 * out->obj of a reconstruction; device or pinned host memory, read during this call only):
 * Omega_v(q) = Psi(q) conj Psi(q - q_v) with Psi(k) = sum_s obj_s exp(-2 pi i dk k . r_s) the
 * estimate's spectrum at detector-pixel frequencies, W_O = IFFT2(ifftshift Omega_v), and
 * conj(W_O) / (|W_O|^2 + eps_v) with eps_v = epsilon * max_r |W_O(v, r)|^2 per frequency (or
 * epsilon when eps_absolute).  wdd_offline_reconstruct on this plan then writes the probe
 * IFFT2(conj(p_v / sqrt(p_0))) on the scan grid (origin at index 0) to out->obj and its phase
 * to out->phase; WDD_OFFLINE_SPECTRUM holds p_v, and get_info's eps_eff the largest eps_v.
 * Holds the classical plan's memory plus two scan-axis tables and the object's x sums.
 * Errors: as wdd_offline_plan_create; INVALID_ARG for a NULL or pageable `obj` or an estimate
 * whose autocorrelation is zero everywhere; UNSUPPORTED for scan_rotation_rad != 0 (the
 * estimate's spectrum is taken one scan axis at a time). */
wdd_status wdd_offline_probe_plan_create(const wdd_params* p, const void* obj,
                                         wdd_offline_plan** out);
/* Device bytes such a plan would hold, without touching the GPU. */
wdd_status wdd_offline_footprint(const wdd_params* p, int64_t* bytes);
/* Reconstructs from all S = scan_y * scan_x frames: frames [S][det_y][det_x] of frame_dtype in
 * raster scan order (s = s_y * scan_x + s_x), in device or pinned host memory, borrowed until
 * `stream` has passed the call.  Writes out->obj (complex64 [scan_y][scan_x]) and out->phase
 * (f32, may be NULL) in stream order; frames_seen = positions_covered = S.  Calls on one plan
 * must be ordered (one stream, or synchronised).  Errors: INVALID_ARG (NULL pointers, pageable
 * frames), CUDA. */
wdd_status wdd_offline_reconstruct(wdd_offline_plan* plan, const void* frames, wdd_result* out,
                                   wdd_stream_t stream);
typedef enum {
    WDD_OFFLINE_SPECTRUM = 0, /* complex64 [S] o_v of the last reconstruction (before the
                                 normalisation by sqrt(o_0))                                */
    WDD_OFFLINE_WIENER = 1,   /* complex64 [S][det_y][det_x] conj(W_P) / (|W_P|^2 + eps_eff),
                                 r in numpy ifft2 order, zero for inactive v               */
    WDD_OFFLINE_MASK = 2      /* uint8 [S] 1 = active frequency                             */
} wdd_offline_array;
/* Synchronously copies an array into host memory (bytes >= its size; *written = bytes copied). */
wdd_status wdd_offline_copy_array(wdd_offline_plan* plan, int32_t which, void* host_dst,
                                  int64_t bytes, int64_t* written);
/* Device bytes held, active frequencies, 1 if one CTA transforms a whole detector plane, and
 * eps_eff.  Any output pointer may be NULL. */
wdd_status wdd_offline_get_info(const wdd_offline_plan* plan, int64_t* device_bytes,
                                int32_t* n_active, int32_t* fused, double* eps_eff);
/* Frees the plan (synchronises the device first). */
wdd_status wdd_offline_plan_destroy(wdd_offline_plan* plan);

/* Status name ("WDD_OK", ...) and the calling thread's last error detail. */
const char* wdd_status_string(wdd_status s);
const char* wdd_last_error(void);

/* Library version: (major << 16) | minor. */
int32_t wdd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WDD_H */
