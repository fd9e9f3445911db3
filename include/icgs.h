/*
 * icgs.h -- C ABI of the GB300-native instant-colorization library (libicgs.so).
 *
 * The library computes, for a fixed Gaussian-splat scene and a set of calibrated target images,
 * the per-Gaussian spherical-harmonic coefficients of the visibility-weighted least-squares problem
 * of arXiv 2604.17155 (Sec. 3, Eq. 10-15, Alg. 1 lines 1-6):
 *
 *     c_i = (G_i + w_i Lambda)^-1 b_i,   G_i = sum_j V_i^j Y_ij Y_ij^T,   b_i = sum_j Y_ij S_ij^T,
 *     w_i = sum_j V_i^j,  V_i^j = sum_{x,y} alpha_i T_i,  S_ij^k = sum_{x,y} alpha_i T_i t^{j,k}_{x,y},
 *
 * where alpha_i T_i is the front-to-back blend weight of Gaussian i in pixel (x,y) of camera j
 * (Eq. 2, Eq. 4) and Y_ij is the real SH basis (Eq. 3) at the direction from camera j's centre to
 * Gaussian i's mean (Sec. 3, below Eq. 9). It also renders (Eq. 1-3) and differentiates the
 * coefficients with respect to the target images and the opacities.
 *
 * Rendering conventions (the paper renders "following Kerbl et al."; these are the 3DGS ones):
 *   - camera: pinhole, looks down +z, image y axis down, world_to_cam = row-major [R|t]; pixel
 *     (x,y) has its centre at (x+0.5, y+0.5); Gaussians with camera-space z <= near_z are culled;
 *   - 2D covariance J W Sigma W^T J^T + 0.3 I, Jacobian taken at the mean with x/z, y/z clamped to
 *     1.3 * (width/2)/fx, 1.3 * (height/2)/fy;
 *   - alpha = min(0.99, opacity * exp(-q/2)); pairs with alpha < 1/255 are skipped; the walk of a
 *     pixel stops before the first Gaussian that would bring T below 1e-4;
 *   - depth order: ascending float32 key fma(W22, z, fma(W21, y, fma(W20, x, W23))), three
 *     correctly rounded float32 fused multiply-adds (the near-plane test uses the same key); equal
 *     keys in ascending Gaussian index;
 *   - SH: real orthonormal harmonics, index l*l+l+m (m = -l..l), degree 1 = sqrt(3/(4 pi))*(y,z,x);
 *     no 0.5 colour offset and no clamp (Eq. 3 is linear).
 *
 * Memory and threading:
 *   - Pointers named "device" are CUDA device pointers owned by the caller; "host" pointers are
 *     read during the call only. The library never allocates device memory: every call takes a
 *     caller-owned workspace of at least the size returned by the matching *_workspace_size call.
 *   - All work is enqueued on `stream` (a cudaStream_t, NULL = legacy default stream). The plain
 *     calls end by copying a small status block back to the host and synchronising `stream`, so
 *     results are complete when the call returns ICGS_OK. Their *_async twins (icgs_colorize_async,
 *     icgs_colorize_backward_async, icgs_colorize_refine_async, icgs_render_async) never
 *     synchronise: they check the arguments on the host, enqueue the work and return; the device
 *     status (capacity overflow, timeouts, non-finite targets) stays in the workspace until
 *     icgs_async_status reads it.
 *   - Calls on different streams with different workspaces may run concurrently.
 *   - On error the call returns a negative icgs_status; icgs_last_error() gives a message (per host
 *     thread). Outputs are then unspecified.
 */
#ifndef ICGS_H
#define ICGS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ICGS_API __attribute__((visibility("default")))
#else
#define ICGS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ICGS_OK = 0,
  ICGS_ERR_INVALID_ARG = -1,          /* bad shape, pointer, degree, dtype or option */
  ICGS_ERR_WORKSPACE_TOO_SMALL = -2,  /* workspace_bytes below the *_workspace_size result */
  ICGS_ERR_CUDA = -3,                 /* a CUDA runtime call failed (message has the CUDA error) */
  ICGS_ERR_CAPACITY = -4,             /* more (Gaussian, tile) instances than the workspace was sized
                                         for; icgs_last_required_instances() gives the count to pass
                                         as icgs_options.instance_capacity */
  ICGS_ERR_UNSUPPORTED = -5,          /* valid request the library does not implement; also reported
                                         after the work when the tensor-core walk found its dynamic
                                         shared memory base not 128-byte aligned (that walk then did
                                         nothing; results are unspecified) */
  ICGS_ERR_DEVICE_TIMEOUT = -6,       /* a bounded wait inside a kernel gave up (the kernel freed its
                                         resources and returned; results are unspecified) */
  ICGS_ERR_NONFINITE_INPUT = -7       /* a target value that a walk read (a pixel of a tile that some
                                         Gaussian's support box reaches) is NaN or infinite; the
                                         results are unspecified. Detected by the accumulate walks of
                                         colorize and refine */
} icgs_status;

typedef enum { ICGS_F32 = 0, ICGS_BF16 = 1, ICGS_F16 = 2 } icgs_dtype;

typedef enum {
  ICGS_PRECISION_PLAIN = 0, /* FP32 weights, CUDA-core contraction, plain FP32 fold and Cholesky */
  ICGS_PRECISION_MIXED = 1  /* fold with exact float-float products and compensated sums, FP32
                               Cholesky refined in float-float against them; below cond_tau
                               solved in FP64; 16-bit targets with >= 16 channels contract on
                               tcgen05 tensor cores (BF16/FP16 in, FP32 acc) */
} icgs_precision;

/* Per-Gaussian status written to status_out. */
enum { ICGS_GAUSSIAN_OK = 0, ICGS_GAUSSIAN_UNSEEN = 1, ICGS_GAUSSIAN_FP64 = 2 };

/* The fixed scene (Alg. 1 "Data": Gaussian means and covariances; Sec. 3 Eq. 1). All device,
 * float32, contiguous. quats are (w,x,y,z) and are normalised inside; scales are linear (> 0). */
typedef struct {
  int64_t n;
  const float* means;    /* device [n,3] */
  const float* scales;   /* device [n,3] */
  const float* quats;    /* device [n,4] */
  const float* opacity;  /* device [n], in (0,1) */
} icgs_scene;

/* Calibrated cameras P_j (Alg. 1 "Data": camera poses). All cameras share one image size. */
typedef struct {
  int32_t n_cams;
  int32_t width, height;
  float near_z;                /* <= 0 selects 0.2 */
  const float* intrinsics;     /* host [n_cams,4]: fx, fy, cx, cy (pixels) */
  const float* world_to_cam;   /* host [n_cams,12]: row-major 3x4 [R|t] */
} icgs_cameras;

/* Target images t^{j,k}_{x,y} (Alg. 1 "Data": GT images; Sec. 3: any number of channels). */
typedef struct {
  icgs_dtype dtype;
  int32_t channels;            /* K >= 1 */
  const void* data;            /* device [n_cams,height,width,channels], contiguous */
} icgs_targets;

typedef struct {
  int32_t sh_degree;           /* L in 0..3; (L+1)^2 coefficients per channel */
  const float* lambda;         /* host [(L+1)^2] Tikhonov weights lambda_m (Eq. 14); NULL selects
                                  the paper's values (Sec. 4): 1e-5 / 1e-4 / 1e-3 / 1e-2 per band */
  int32_t precision;           /* icgs_precision */
  float cond_tau;              /* MIXED: FP64 for a Gaussian when min_k pivot_k / A_kk < cond_tau
                                  (<= 0 selects 1e-3); for a re-folded Gaussian (below) the test
                                  is against cond_tau * 1e-2 */
  float refold_tau;            /* MIXED, every camera in one pass: a Gaussian whose pivot ratio is
                                  below refold_tau is re-folded from its per-camera sums (a second,
                                  independent float-float evaluation of its G, b, w) before the
                                  solve. The MIXED fold itself forms every product and sum exactly
                                  in float-float, so this is a cross-check, off by default: <= 0
                                  selects none; > 1 re-folds every Gaussian */
  int32_t cam_batch;           /* cameras accumulated per pass; <= 0 selects min(n_cams, 128) */
  int64_t instance_capacity;   /* (Gaussian, tile) instances per pass the workspace holds; <= 0
                                  selects an estimate (see ICGS_ERR_CAPACITY) */
} icgs_options;

/* Bytes of workspace icgs_colorize / icgs_colorize_backward need for these arguments. */
ICGS_API size_t icgs_workspace_size(const icgs_scene* scene, const icgs_cameras* cams,
                           const icgs_targets* targets, const icgs_options* opt);

/* Colorize (Alg. 1 lines 1-6, Eq. 14). Writes
 *   coeffs_out  device [n,(L+1)^2,K] float32: c_i (zero for Gaussians no pixel sees),
 *   status_out  device [n] uint8 (nullable): ICGS_GAUSSIAN_{OK,UNSEEN,FP64},
 *   chol_out    device [n, 3P] float32 (nullable), P = B(B+1)/2 with B = (L+1)^2: the solve record
 *               that icgs_colorize_backward and icgs_colorize_refine take. Per Gaussian: the
 *               row-packed lower Cholesky factor of A_i = G_i + w_i Lambda (P floats; row r holds
 *               L_r0..L_rr), then A_i itself in float-float, row-packed lower triangle, P hi parts
 *               followed by P lo parts (A = hi + lo; lo is 0 in PLAIN precision). The adjoint refines
 *               its solve with A_i against the factor's rounding. Unseen Gaussians: all zero. */
ICGS_API icgs_status icgs_colorize(const icgs_scene* scene, const icgs_cameras* cams,
                          const icgs_targets* targets, const icgs_options* opt,
                          void* workspace, size_t workspace_bytes,
                          float* coeffs_out, uint8_t* status_out, float* chol_out, void* stream);

/* Several target sets on one geometry (Sec. 4: the same scene captured under different lightings;
 * Sec. 3: the inverse of G_i + w_i Lambda is shared by every channel). sets[0..n_sets-1] are target
 * image stacks of the same cameras, each with its own dtype and channel count K_s (1 <= n_sets <=
 * 64). The projection, binning and depth sort run once per camera pass for all sets, each set is
 * walked once (the tensor-core walk where it applies to that set), and one factorisation of A_i
 * solves every set's channels as right-hand sides. Writes
 *   coeffs_out  device [n,(L+1)^2,sum_s K_s] float32: the sets' coefficients, channels in set order
 *               (identical arithmetic to icgs_colorize on the concatenated channels),
 *   status_out, chol_out as for icgs_colorize (one record: the factorisation is shared),
 *   keep_out    device [n, sum_s K_s] uint8 (nullable; needs sh_degree 0): the segmentation
 *               threshold of Sec. 5, fused into the solve: 1 where the Gaussian's colour
 *               c_i0 Y_0 >= threshold (the paper filters Gaussians below 0.6), 0 elsewhere and for
 *               unseen Gaussians; with sh_degree > 0 ICGS_ERR_UNSUPPORTED.
 * Workspace: icgs_sets_workspace_size() bytes (the colorize workspace of all channels plus one
 * accumulator per set). Synchronises `stream`. The pair count of icgs_last_stats sums the sets. */
ICGS_API size_t icgs_sets_workspace_size(const icgs_scene* scene, const icgs_cameras* cams, int32_t n_sets,
                                         const icgs_targets* sets, const icgs_options* opt);
ICGS_API icgs_status icgs_colorize_sets(const icgs_scene* scene, const icgs_cameras* cams, int32_t n_sets,
                                        const icgs_targets* sets, const icgs_options* opt, void* workspace,
                                        size_t workspace_bytes, float* coeffs_out, uint8_t* status_out,
                                        float* chol_out, float threshold, uint8_t* keep_out, void* stream);

/* Iterative refinement (Alg. 1 lines 7-10). Repeats n_steps times: render the images of the current
 * coefficients (Eq. 1-3), accumulate the visibility-weighted residual targets t - img as in Eq. 6
 * (V, Y and w are those of the fixed geometry), and update
 *     c_i <- c_i + A_i^-1 (sum_j Y_ij S_res_ij^T - w_i Lambda c_i)
 * with the factor of A_i = G_i + w_i Lambda in the solve record icgs_colorize returned (chol, [n, 3P]). coeffs_inout (device
 * [n,(L+1)^2,K] float32) holds the coefficients of icgs_colorize on entry and the refined ones on
 * return. The residual walk always runs on CUDA cores (FP32), whatever the target dtype. Needs the
 * workspace size icgs_refine_workspace_size returns. */
ICGS_API size_t icgs_refine_workspace_size(const icgs_scene* scene, const icgs_cameras* cams,
                                           const icgs_targets* targets, const icgs_options* opt);
ICGS_API icgs_status icgs_colorize_refine(const icgs_scene* scene, const icgs_cameras* cams,
                                          const icgs_targets* targets, const icgs_options* opt,
                                          int32_t n_steps, const float* chol, void* workspace,
                                          size_t workspace_bytes, float* coeffs_inout, void* stream);

/* Adjoint of icgs_colorize for a loss L(c): given dL/dc (grad_coeffs, device [n,(L+1)^2,K]),
 * the coefficients and solve records (chol, [n, 3P]) returned by icgs_colorize on the same inputs,
 * writes
 *   grad_targets  device [n_cams,height,width,K] float32 (nullable): dL/dt,
 *   grad_opacity  device [n] float32 (nullable): dL/d(opacity) (overwritten, not accumulated).
 * The blend lists are recomputed, not stored. With u_i = A_i^-1 dL/dc_i (the factor's solve, refined
 * twice in float-float against the record's A_i): dL/dS_ij = Y_ij^T u_i,
 * dL/dV_ij = -sum_k u_ik^T (Y_ij Y_ij^T + Lambda) c_ik, and the per-pixel walk applies
 * d(alpha_m T_m)/d(alpha_n) (Eq. 2). Threshold decisions (alpha >= 1/255, the T stop, the 0.99 cap)
 * are held fixed, as in any rasterizer's gradient. */
ICGS_API icgs_status icgs_colorize_backward(const icgs_scene* scene, const icgs_cameras* cams,
                                   const icgs_targets* targets, const icgs_options* opt,
                                   const float* coeffs, const float* chol, const float* grad_coeffs,
                                   void* workspace, size_t workspace_bytes,
                                   float* grad_targets, float* grad_opacity, void* stream);

/* Bytes of workspace icgs_render needs. */
ICGS_API size_t icgs_render_workspace_size(const icgs_scene* scene, const icgs_cameras* cams,
                                  int32_t sh_degree, int32_t channels, int64_t instance_capacity);

/* Render (Eq. 1-3): images_out device [n_cams,height,width,channels] float32 from coeffs device
 * [n,(L+1)^2,channels]; background 0. (L+1)^2 x channels must be at most 12287
 * (ICGS_ERR_UNSUPPORTED otherwise); the same limit applies to icgs_colorize_refine. */
ICGS_API icgs_status icgs_render(const icgs_scene* scene, const icgs_cameras* cams, int32_t sh_degree,
                        int32_t channels, const float* coeffs, int64_t instance_capacity,
                        void* workspace, size_t workspace_bytes, float* images_out, void* stream);

/* Colorize without a caller workspace -- no counterpart in the paper; this is a library service.
 *
 * For callers that cannot allocate device memory: a plugin inside an application that owns every
 * byte of device memory through its own allocator, or a latency-critical loop that may not
 * allocate (or risk failing to) once it runs. Such callers cannot hand icgs_colorize a workspace,
 * so this call takes it from a fixed scratch array of icgs_noalloc_scratch_bytes() (64 MiB) that
 * the library places on every GPU that loads it and keeps until the process exits. It allocates
 * nothing itself; inputs, outputs and `stream` are as for icgs_colorize, and so are the results.
 *   - The first call on a device resolves the scratch's device address for that device; make that
 *     first call before any stream capture.
 *   - A problem whose workspace does not fit returns ICGS_ERR_WORKSPACE_TOO_SMALL (or
 *     ICGS_ERR_CAPACITY when the Gaussian-tile instances of one pass do not fit), with a message
 *     naming the limit; use icgs_colorize with a caller workspace then. opt->instance_capacity <= 0
 *     gives the instance buffers all the scratch the other regions leave free.
 *   - Every call on a device shares the one array and leaves its contents behind (each call
 *     clears what must start at zero). Calls that overlap on the GPU -- on two streams, or from
 *     two host threads -- race on it and must not be issued. */
ICGS_API icgs_status icgs_colorize_noalloc(const icgs_scene* scene, const icgs_cameras* cams,
                                           const icgs_targets* targets, const icgs_options* opt,
                                           float* coeffs_out, uint8_t* status_out, float* chol_out,
                                           void* stream);

/* icgs_colorize with the targets in HOST memory and the coefficients and status written to HOST
 * memory: the call a user makes when the images and results live on the host. There is no paper
 * counterpart; it computes exactly what icgs_colorize computes (Alg. 1 lines 1-6).
 *   targets->data  HOST pointer to [n_cams, H, W, channels] of targets->dtype, row-major. Page-locked
 *                  (pinned) memory lets the copies run asynchronously; pageable memory works but the
 *                  driver stages it.
 *   coeffs_host    HOST [n, (L+1)^2, channels] float32, written before the call returns.
 *   status_host    HOST [n] ICGS_GAUSSIAN_*, or NULL.
 *   chol_out       DEVICE, as for icgs_colorize (for icgs_colorize_backward), or NULL.
 *   workspace      DEVICE, 256-byte aligned, icgs_colorize_host_workspace_size() bytes: the
 *                  colorize workspace followed by the staged targets, coefficients and status.
 * The targets are copied to the device in chunks of cameras, alternating between two copy streams
 * owned by the library (one pair per host thread and device), and each chunk's walk waits only for
 * its own copy, so the copies overlap the projection, binning and the walk of earlier chunks. Each
 * copy is enqueued two chunks ahead of its walk: with pageable memory, where an enqueue holds the
 * host until the copy is done, the walks already enqueued still run meanwhile. The call synchronises
 * `stream` before returning. The staging region is overwritten only after the work already queued
 * on `stream` has finished. Errors as for icgs_colorize. */
ICGS_API size_t icgs_colorize_host_workspace_size(const icgs_scene* scene, const icgs_cameras* cams,
                                                  const icgs_targets* targets, const icgs_options* opt);
ICGS_API icgs_status icgs_colorize_host(const icgs_scene* scene, const icgs_cameras* cams,
                                        const icgs_targets* targets, const icgs_options* opt, void* workspace,
                                        size_t workspace_bytes, float* coeffs_host, uint8_t* status_host,
                                        float* chol_out, void* stream);

/* Camera sharding of the normal equations (Eq. 12-14). The sums over cameras split over any
 * partition of the cameras: a caller with several GPUs (or several calls on one GPU) accumulates
 * each subset with icgs_accumulate, sums the results elementwise (across GPUs a reduce-scatter over
 * contiguous Gaussian ranges, so each GPU receives the totals of its own range), and solves each
 * range with icgs_solve. The paper has no such split; it is the same arithmetic in two steps.
 *
 * Packed layout, per Gaussian, icgs_normal_size(L, K) = P + B K + 1 doubles (B = (L+1)^2,
 * P = B(B+1)/2): the upper triangle of G_i = sum_j V_ij Y_ij Y_ij^T row by row (row r holds columns
 * r..B-1), then b_i = sum_j Y_ij S_ij^T as [B,K] row-major, then w_i = sum_j V_ij. MIXED returns its
 * compensated sums (hi + lo) rounded once to double; add shards in double.
 *
 * icgs_accumulate: these cameras' sums, sums_out DEVICE [n, icgs_normal_size(L,K)] float64.
 *   Workspace: icgs_workspace_size() bytes (DEVICE, 256-byte aligned). Synchronises `stream`. */
ICGS_API int64_t icgs_normal_size(int32_t sh_degree, int32_t channels);
ICGS_API icgs_status icgs_accumulate(const icgs_scene* scene, const icgs_cameras* cams,
                                     const icgs_targets* targets, const icgs_options* opt, void* workspace,
                                     size_t workspace_bytes, double* sums_out, void* stream);

/* icgs_solve: c_i = (G_i + w_i Lambda)^-1 b_i (Eq. 14) for n Gaussians from their packed float64
 * device sums (any contiguous range of rows icgs_accumulate wrote, or their sum over shards), with
 * the precision, lambda and cond_tau of opt (scene and camera fields are not used). MIXED
 * factorises in FP32 and refines in float-float against the sums split into (hi, lo); below
 * cond_tau it solves in FP64. There is no exact re-fold: the per-camera sums are not available here.
 * Outputs as for icgs_colorize (device, n rows). Workspace: icgs_solve_workspace_size() bytes
 * (DEVICE, 256-byte aligned). Synchronises `stream`. */
ICGS_API size_t icgs_solve_workspace_size(int64_t n, int32_t sh_degree, int32_t channels, const icgs_options* opt);
ICGS_API icgs_status icgs_solve(int64_t n, int32_t sh_degree, int32_t channels, const double* sums,
                                const icgs_options* opt, void* workspace, size_t workspace_bytes, float* coeffs_out,
                                uint8_t* status_out, float* chol_out, void* stream);

/* Enqueue-only forms of icgs_colorize, icgs_colorize_backward, icgs_colorize_refine and
 * icgs_render: the same arguments, checks and work, but the call returns as soon as the work is on
 * `stream`, with no synchronisation and no device-to-host copy (the camera table and lambda reach
 * the device as kernel parameters). A returned ICGS_OK means only that the arguments were valid and
 * every launch was accepted; outputs and workspace must stay allocated, and the host arrays
 * (cameras, lambda) may be released at once. The call's device outcome is read, after the work has
 * finished, by icgs_async_status on the same workspace. Stage timing is not recorded, and
 * icgs_last_stats reports the call only after icgs_async_status. */
ICGS_API icgs_status icgs_colorize_async(const icgs_scene* scene, const icgs_cameras* cams,
                                        const icgs_targets* targets, const icgs_options* opt, void* workspace,
                                        size_t workspace_bytes, float* coeffs_out, uint8_t* status_out,
                                        float* chol_out, void* stream);
ICGS_API icgs_status icgs_colorize_backward_async(const icgs_scene* scene, const icgs_cameras* cams,
                                                 const icgs_targets* targets, const icgs_options* opt,
                                                 const float* coeffs, const float* chol, const float* grad_coeffs,
                                                 void* workspace, size_t workspace_bytes, float* grad_targets,
                                                 float* grad_opacity, void* stream);
ICGS_API icgs_status icgs_colorize_refine_async(const icgs_scene* scene, const icgs_cameras* cams,
                                               const icgs_targets* targets, const icgs_options* opt, int32_t n_steps,
                                               const float* chol, void* workspace, size_t workspace_bytes,
                                               float* coeffs_inout, void* stream);
ICGS_API icgs_status icgs_render_async(const icgs_scene* scene, const icgs_cameras* cams, int32_t sh_degree,
                                      int32_t channels, const float* coeffs, int64_t instance_capacity,
                                      void* workspace, size_t workspace_bytes, float* images_out, void* stream);

/* The device outcome of the last *_async call that used `workspace` (DEVICE, the same pointer):
 * copies the status block back on `stream` and synchronises `stream`, so call it where the caller
 * joins the work (every earlier call on that workspace has then finished). Returns ICGS_OK,
 * ICGS_ERR_CAPACITY (icgs_last_required_instances() then gives the count to pass), or
 * ICGS_ERR_DEVICE_TIMEOUT / ICGS_ERR_NONFINITE_INPUT; updates icgs_last_stats (the kernel count
 * is not known here and reads 0). */
ICGS_API icgs_status icgs_async_status(const void* workspace, void* stream);

/* Size in bytes of the built-in scratch icgs_colorize_noalloc works in. */
ICGS_API size_t icgs_noalloc_scratch_bytes(void);

/* Diagnostic: D[128 x N] = A[128 x 256] * B[N x 256]^T through the tensor-core (tcgen05) operand
 * layout, MMA issue and TMEM read-back that the 16-bit accumulate walk uses. A and B are device,
 * row-major 16-bit (bf16 != 0: BF16, else FP16), D device float32 [128 x N]; N is 32 or 80;
 * workspace is device memory of at least 256 bytes. Synchronises `stream`. */
ICGS_API icgs_status icgs_selftest_tc(const void* A, const void* B, int32_t N, int32_t bf16, float* D,
                                      void* workspace, void* stream);

/* Diagnostic, as icgs_selftest_tc for an MMA of M = 64 or 128 rows: D[M x N] = A[M x 256] *
 * B[N x 256]^T, each row read back from the TMEM lane the walk reads it from. D_lanes (device float32
 * [128 x N], may be NULL) receives the raw contents of all 128 TMEM lanes, which shows where the
 * MMA placed each row. Invalid M or N: ICGS_ERR_INVALID_ARG. Synchronises `stream`. */
ICGS_API icgs_status icgs_selftest_tc_rows(const void* A, int32_t M, const void* B, int32_t N, int32_t bf16, float* D,
                                           float* D_lanes, void* workspace, void* stream);

/* Diagnostic, for testing the failure path: sets, for the calls of this host thread, the time limit
 * of the tensor-core walk's bounded mbarrier waits (limit_ns <= 0 restores the default, 1 s) and
 * whether the walk issues its MMAs (issue_mma = 0: it issues none, so each wait runs out with no
 * tensor-core work in flight, the kernel frees its TMEM and returns, and the call reports
 * ICGS_ERR_DEVICE_TIMEOUT). Call icgs_debug_tc_wait(0, 1) to restore normal operation. */
ICGS_API void icgs_debug_tc_wait(int64_t limit_ns, int32_t issue_mma);

/* Diagnostic: the depth sort of the tile lists (the "depth ordered list" of Eq. 2) as the colorize
 * calls run it. tile_off: device uint32 [ntiles + 1], non-decreasing from 0, delimits the lists in
 * keys; keys: device uint64 [nkeys], each (float32 depth bits << 32) | Gaussian index with a
 * positive finite depth, unique within its list. Every list is sorted ascending in place; keys
 * past nkeys are not touched (a list is cut at nkeys). workspace: device, 256-byte aligned, at
 * least icgs_sort_workspace_size(ntiles, nkeys) bytes (else ICGS_ERR_WORKSPACE_TOO_SMALL).
 * Synchronises `stream`. */
ICGS_API size_t icgs_sort_workspace_size(int32_t ntiles, int64_t nkeys);
ICGS_API icgs_status icgs_sort_tile_lists(const uint32_t* tile_off, uint64_t* keys, int32_t ntiles, int64_t nkeys,
                                          void* workspace, size_t workspace_bytes, void* stream);

/* Message of the last failed call on this host thread ("" if none). */
ICGS_API const char* icgs_last_error(void);

/* (Gaussian, tile) instances the last call on this host thread needed in its largest pass. */
ICGS_API int64_t icgs_last_required_instances(void);

/* Statistics of the last successful call on this host thread, for benchmarks:
 * out[0] = (Gaussian, tile) instances summed over passes, out[1] = (pixel, Gaussian) pairs with
 * nonzero blend weight, out[2] = Gaussians solved in FP64, out[3] = kernels launched,
 * out[4] = Gaussians re-folded exactly from the per-camera sums (MIXED, single pass). */
ICGS_API void icgs_last_stats(int64_t out[5]);

/* Stage timing for benchmarks (off by default, per host thread). When on, every call records CUDA
 * events on its stream at each stage boundary (no extra synchronisation) and
 * icgs_last_stage_ms(out, n) writes the milliseconds spent in stage i (summed over passes) to
 * out[i] for i < min(n, stage count) and returns the stage count. icgs_stage_name(i) names
 * stage i: project, scan, scatter, sort, blend, fold, solve, payload. */
ICGS_API void icgs_set_stage_timing(int enable);
ICGS_API int icgs_last_stage_ms(double* out, int n);
ICGS_API const char* icgs_stage_name(int i);

#ifdef __cplusplus
}
#endif

#endif /* ICGS_H */
