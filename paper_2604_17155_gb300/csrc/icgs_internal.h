// icgs_internal.h -- types shared by the CUDA translation units of libicgs.so (not public).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/icgs.h"

namespace icgs {

constexpr int kTile = 16;            // screen tiles are 16x16 pixels; one CTA of 256 threads each
constexpr int kTilePixels = kTile * kTile;
constexpr int kMaxSH = 16;           // (L+1)^2 for L = 3
// A payload CTA stages at least one Gaussian's (L+1)^2 x K coefficients in 48 KB of shared memory.
constexpr int kMaxPayloadRow = 12287;
constexpr int kSortCap = 4096;       // tile lists up to this length are sorted in shared memory at once
constexpr uint32_t kMaxCapacity = 0x7FFFFFF0u;
constexpr uint8_t kGaussOk = 0, kGaussUnseen = 1, kGaussFp64 = 2;  // icgs.h ICGS_GAUSSIAN_*

// The per-Gaussian solve record the colorize calls write (chol_out) and the adjoint and refinement
// read: P = B (B + 1) / 2 floats each of the row-packed lower Cholesky factor L of A = G + w Lambda,
// then A itself in float-float, row-packed lower triangle, hi parts then lo parts.
__host__ __device__ constexpr int solve_record_floats(int B) { return 3 * (B * (B + 1) / 2); }

// Device status block at the start of every workspace; read back at the end of each call.
struct DevStatus {
  uint32_t flags;             // kFlag* bits
  uint32_t big_tiles;         // tiles of 1025..2048 keys queued (from the front of the queue) in the current pass
  uint32_t sort_next;         // next tile of the persistent tile sort (work counter)
  uint32_t long_tiles;        // tiles of more than 2048 keys queued (from the end of the queue)
  uint64_t instances_needed;  // max over passes of (Gaussian, tile) instances
  uint64_t instances_total;   // sum over passes
  uint64_t contrib_pairs;     // pixel-Gaussian pairs with nonzero weight (sum over passes)
  uint32_t fp64_count;        // Gaussians solved in FP64
  uint32_t refold_count;      // Gaussians re-folded exactly from the per-camera sums
};
constexpr uint32_t kFlagOverflow = 1u;
constexpr uint32_t kFlagTimeout = 2u;    // a bounded device-side wait gave up
constexpr uint32_t kFlagNonfinite = 4u;  // a walk read a NaN or infinite target value
constexpr uint32_t kFlagLayout = 8u;     // a kernel found its shared memory base misaligned and did nothing

// One camera as the kernels see it (built on the host from icgs_cameras).
struct DevCam {
  float fx, fy, cx, cy;
  float w[12];        // world_to_cam, row-major [R|t]
  float centre[3];    // -R^T t (host double, rounded)
  float limx, limy;   // 1.3 * tan(fov/2) in x and y
  float rnorm2;       // >= squared spectral norm of R (the early frustum cull of the projection)
  double centre_d[3]; // -R^T t in double (the FP64 re-fold of ill-conditioned Gaussians)
};

// Projected Gaussian as the blend kernels read it: 32 bytes, one sector.
//   box.x, box.y = hi parts of the projected mean (float-float: mean = hi + lo),
//   box.z = fp16 pair (lo_x, lo_y) * kMeanLoScale (|lo| <= half an ulp of hi),
//   box.w = fp16 pair (half-width, half-height) of the padded support box {q <= 2 ln(255 o)},
//           rounded up so the box stays a superset,
//   par = (conic_a, conic_b, conic_c, opacity) with q = a dx^2 + 2 b dx dy + c dy^2.
struct ProjRec {
  float4 box;
  float4 par;
};

// Sub-allocation of a caller workspace (every region 256-byte aligned).
struct Workspace {
  char* base = nullptr;
  size_t bytes = 0;
  DevStatus* status = nullptr;
  DevCam* cams = nullptr;
  ProjRec* rec = nullptr;          // [cb * n]
  uint4* rect = nullptr;           // [cb * n] by processing position: (tx0|ty0<<16, tx1|ty1<<16, depth key bits, 0)
  uint32_t* tile_off = nullptr;    // [cb * T + 1] counts, then exclusive offsets
  uint32_t* tile_cur = nullptr;    // [cb * T]
  uint32_t* scan_tmp = nullptr;    // [scan blocks + 1]
  uint32_t* big_list = nullptr;    // [cb * T]
  uint64_t* entries = nullptr;     // [capacity] (depth key << 32 | index)
  uint64_t* entries_tmp = nullptr; // [capacity] merge buffer for long tiles
  uint32_t* order = nullptr;       // [n] Gaussians in processing order (Morton cells of the scene box)
  uint32_t* cell_off = nullptr;    // [cells + 1] counts, then offsets of the cells in order
  uint32_t* cell_cur = nullptr;    // [cells]
  uint32_t* cell_tmp = nullptr;    // [cells / 1024 + 2] scan block sums
  uint32_t* cell_box = nullptr;    // [6] order keys of the scene box (min xyz, max xyz)
  float4* packed = nullptr;        // [3 n] parameters by processing position (mean, o), (scale, qw), (qxyz, 0)
  float* payload = nullptr;        // [cb * n * (K+1)] per (camera, Gaussian) colour / adjoint terms
  float* acc = nullptr;            // [cb * n * RS] (L>0) or [n * RS] (L=0), RS = acc_stride
  float* G = nullptr;              // [n * B * B] Gram rows, hi
  float* Glo = nullptr;            // [n * B * B] compensation
  float* bvec = nullptr;           // [n * B * K]
  float* blo = nullptr;            // [n * B * K]
  float* wsum = nullptr;           // [n]
  float* wlo = nullptr;            // [n]
  float* u = nullptr;              // [n * B * K] backward: A^-1 dL/dc, hi part
  float* u_lo = nullptr;           // [n * B * K] backward: its lo part (float-float)
  float* reg = nullptr;            // [n] backward: sum_mk lambda_m u_mk c_mk
  float* grad_o_acc = nullptr;     // [n]
  float* lam = nullptr;            // [B] Tikhonov weights
  float* img = nullptr;            // [cb * H * W * K] refinement: renders of the pass's cameras
  size_t total = 0;
};

struct Problem {
  int64_t n = 0;
  int n_cams = 0, width = 0, height = 0;
  float near_z = 0.2f;
  int tiles_x = 0, tiles_y = 0, tiles = 0;
  int K = 0, L = 0, B = 1;
  int acc_stride = 4;               // floats per accumulator row (V, S_0..S_{K-1}), padded to 4
  int cam_batch = 0;
  uint32_t capacity = 0;
  int precision = 0;
  float cond_tau = 1e-3f;       // MIXED: FP64 solve below this pivot ratio
  float refold_tau = 0.0f;      // MIXED, single pass: exact re-fold below this pivot ratio (0: none)
  int mode = 0;                     // 0 colorize, 1 backward, 2 render
};

// Kernel launches of the current call on this host thread (for the benchmark's launch count).
void note_launches(int count);

// Bytes of workspace icgs_colorize itself needs (icgs_workspace_size also covers the adjoint).
size_t colorize_workspace_bytes(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                                const icgs_options* opt);

// Replaces the message icgs_last_error() returns on this host thread (printf-style).
void set_error_message(const char* fmt, ...);

// ---- launchers (each .cu file exposes host functions that enqueue its kernels) ----
void launch_project(const Problem& p, const float* means, const float* scales, const float* quats,
                    const float* opac, int cb, const Workspace& ws, cudaStream_t s);
void launch_scan(const Problem& p, int cb, const Workspace& ws, cudaStream_t s);
// Cells of the processing order, and the order itself (ws.order; once per call, before the passes).
int spatial_cells();
void launch_spatial_order(const Problem& p, const float* means, const float* scales, const float* quats,
                          const float* opac, const Workspace& ws, cudaStream_t s);
void launch_scatter(const Problem& p, int cb, const Workspace& ws, cudaStream_t s);
void launch_tile_sort(const Problem& p, int cb, const Workspace& ws, cudaStream_t s);
// sub_img (nullable, float32 [cb,H,W,K] of this pass's cameras): accumulate t - img instead of t
// (refinement); forces the CUDA-core walk.
bool launch_blend_refine(const Problem& p, int cb, int cam0, const void* targets, int dtype, const Workspace& ws,
                         cudaStream_t s);
void launch_blend_accumulate(const Problem& p, int cb, int cam0, const void* targets, int dtype,
                             const float* sub_img, const Workspace& ws, cudaStream_t s);
// Tensor-core contraction of the accumulate walk (MIXED precision, 16-bit targets, 16..64 channels).
bool tc_accumulate_applies(const Problem& p, int dtype);
void launch_blend_accumulate_tc(const Problem& p, int cb, int cam0, const void* targets, int dtype,
                                const Workspace& ws, cudaStream_t s);
// Diagnostic (this host thread): the tensor-core walk's wait limit (<= 0: the default 1 s) and
// whether it issues its MMAs (false: every wait runs out, with nothing in flight).
void set_tc_wait_diagnostic(int64_t limit_ns, bool issue_mma);
cudaError_t launch_tc_selftest(const uint16_t* A, int M, const uint16_t* B, int N, bool bf16, float* D, float* D_lanes,
                               DevStatus* status, cudaStream_t s);
void launch_fold(const Problem& p, const float* means, int cb, bool first, bool want_gram, const Workspace& ws,
                 cudaStream_t s);
// c += A^-1 (b - w Lambda c) from the stored factor (refinement, Alg. 1 line 10).
void launch_refine_update(const Problem& p, const float* lam_dev, const float* lam_host, const float* chol,
                          const Workspace& ws, float* coeffs, cudaStream_t s);
// means/cams/n_acc_cams: when every camera was accumulated in one pass (n_acc_cams > 0), a MIXED
// solve re-folds each Gaussian it flags in FP64 from the per-camera sums still in ws.acc.
// keep (nullable, L = 0 only): per Gaussian and channel, 1 where the colour c Y_0 reaches tau.
void launch_solve(const Problem& p, const float* lam_dev, const float* lam_host, const Workspace& ws,
                  float* coeffs, uint8_t* status, float* chol, const float* means, int n_acc_cams,
                  cudaStream_t s, float tau = 0.0f, uint8_t* keep = nullptr);
// Copies one target set's accumulator rows (V, S_0..S_{Ks-1}, row stride RSs) into the combined
// rows (stride RS): S to columns 1 + col0.., V only for the first set (col0 == 0).
void launch_merge_set(int64_t rows, int Ks, int RSs, const float* src, int RS, int col0, float* dst, cudaStream_t s);
// The normal equations of the current workspace as packed doubles (hi + lo; per Gaussian the upper
// triangle of G row by row, then b [B,K], then w), and back (camera sharding).
void launch_export_normal(const Problem& p, const Workspace& ws, double* sums, cudaStream_t s);
void launch_import_normal(const Problem& p, const Workspace& ws, const double* sums, cudaStream_t s);
void launch_payload_render(const Problem& p, const float* means, const float* coeffs, int cb,
                           const Workspace& ws, cudaStream_t s);
void launch_blend_render(const Problem& p, int cb, int cam0, const Workspace& ws, float* images,
                         cudaStream_t s);
void launch_adjoint_prepare(const Problem& p, const float* lam_dev, const float* lam_host,
                            const float* coeffs, const float* chol, const float* grad_coeffs,
                            const Workspace& ws, cudaStream_t s);
void launch_payload_adjoint(const Problem& p, const float* means, const float* coeffs, int cb,
                            const Workspace& ws, cudaStream_t s);
void launch_blend_adjoint(const Problem& p, int cb, int cam0, const void* targets, int dtype,
                          const Workspace& ws, float* grad_targets, bool want_grad_o,
                          cudaStream_t s);

}  // namespace icgs
