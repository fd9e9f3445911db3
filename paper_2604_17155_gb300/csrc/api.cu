// api.cu -- the C ABI declared in include/icgs.h: argument checks, workspace layout and the
// sequence of kernel launches for colorize (Alg. 1 lines 1-6), its adjoint, and render.
//
// One call processes the cameras in passes of cam_batch cameras. Per pass: project + count
// (k_project), exclusive scan of tile counts, scatter of (depth key, index) into tile slots, per-tile
// depth sort, then the walk (accumulate / render / adjoint). For L > 0 a fold turns the pass's
// per-(camera, Gaussian) sums V and S into the normal equations; for L = 0 the walk accumulates
// straight into one [n, 1+K] array. The call ends with one device->host copy of the status block
// and a stream synchronisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/icgs.h"
#include "icgs_internal.h"

using namespace icgs;

namespace {

thread_local char g_err[1024] = "";
thread_local int64_t g_required = 0;
thread_local int64_t g_stats[5] = {0, 0, 0, 0, 0};
thread_local int64_t g_launches = 0;

// ---- stage timing: one CUDA event per stage boundary, elapsed times read after the final sync ----
enum Stage { kProject = 0, kScan, kScatter, kSort, kBlend, kFold, kSolve, kPayload, kStageCount };
const char* const kStageNames[kStageCount] = {"project", "scan", "scatter", "sort", "blend", "fold", "solve", "payload"};

struct StageTimer {
  bool on = false;
  std::vector<cudaEvent_t> events;  // created on first use, reused by later calls of this thread
  std::vector<int> stage_of;        // stage_of[k] = stage between event k and event k+1
  int used = 0;
  double ms[kStageCount] = {};
  void begin(cudaStream_t s) {
    used = 0;
    stage_of.clear();
    for (double& m : ms) m = 0.0;
    if (on) record(s);
  }
  void record(cudaStream_t s) {
    if (used == (int)events.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
      events.push_back(e);
    }
    cudaEventRecord(events[(size_t)used++], s);
  }
  // marks the end of `stage` (which started at the previous mark)
  void mark(int stage, cudaStream_t s) {
    if (!on) return;
    stage_of.push_back(stage);
    record(s);
  }
  void collect() {
    if (!on) return;
    for (int k = 0; k + 1 < used && k < (int)stage_of.size(); ++k) {
      float m = 0.0f;
      if (cudaEventElapsedTime(&m, events[(size_t)k], events[(size_t)k + 1]) == cudaSuccess) ms[stage_of[(size_t)k]] += m;
    }
  }
};
thread_local StageTimer g_timer;

icgs_status fail(icgs_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

#define ICGS_TRY_CUDA(expr)                                                                  \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return fail(ICGS_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

constexpr int kNeedAccumulate = 1, kNeedBackward = 2, kNeedRender = 4, kNeedRefine = 8;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Lays the regions out from `base` (or only sizes them when base is null).
Workspace carve(char* base, const Problem& p, int need) {
  Workspace ws;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* ptr = base ? base + off : nullptr;
    off += align256(bytes);
    return ptr;
  };
  const int64_t cbn = (int64_t)p.cam_batch * p.n;
  const int64_t ct = (int64_t)p.cam_batch * p.tiles;
  ws.base = base;
  ws.status = reinterpret_cast<DevStatus*>(take(sizeof(DevStatus)));
  ws.cams = reinterpret_cast<DevCam*>(take(sizeof(DevCam) * (size_t)p.n_cams));
  ws.lam = reinterpret_cast<float*>(take(sizeof(float) * kMaxSH));
  ws.rec = reinterpret_cast<ProjRec*>(take(sizeof(ProjRec) * (size_t)cbn));
  ws.rect = reinterpret_cast<uint4*>(take(sizeof(uint4) * (size_t)cbn));
  ws.tile_off = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)(ct + 1)));
  ws.tile_cur = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)ct));
  ws.scan_tmp = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)(ct / 1024 + 2)));
  ws.big_list = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)ct));
  ws.entries = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * (size_t)p.capacity));
  ws.entries_tmp = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * (size_t)p.capacity));
  const size_t cells = (size_t)spatial_cells();
  ws.order = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)p.n));
  ws.cell_off = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (cells + 1)));
  ws.cell_cur = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * cells));
  ws.cell_tmp = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (cells / 1024 + 2)));
  ws.cell_box = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * 8));
  ws.packed = reinterpret_cast<float4*>(take(sizeof(float4) * 3 * (size_t)p.n));
  const size_t B = (size_t)p.B, K = (size_t)p.K, n = (size_t)p.n;
  if (need & kNeedAccumulate) {
    ws.acc = reinterpret_cast<float*>(take(sizeof(float) * (p.L == 0 ? n : (size_t)cbn) * (size_t)p.acc_stride));
    if (p.L > 0) {
      const bool mixed = p.precision == ICGS_PRECISION_MIXED;
      ws.G = reinterpret_cast<float*>(take(sizeof(float) * n * B * B));
      ws.bvec = reinterpret_cast<float*>(take(sizeof(float) * n * B * K));
      ws.wsum = reinterpret_cast<float*>(take(sizeof(float) * n));
      if (mixed) {
        ws.Glo = reinterpret_cast<float*>(take(sizeof(float) * n * B * B));
        ws.blo = reinterpret_cast<float*>(take(sizeof(float) * n * B * K));
        ws.wlo = reinterpret_cast<float*>(take(sizeof(float) * n));
      }
    }
  }
  if (need & kNeedRefine) {  // residual sums, b and w (the Gram is fixed), colours and renders
    const bool mixed = p.precision == ICGS_PRECISION_MIXED;
    ws.acc = reinterpret_cast<float*>(take(sizeof(float) * (p.L == 0 ? n : (size_t)cbn) * (size_t)p.acc_stride));
    if (p.L > 0) {
      ws.bvec = reinterpret_cast<float*>(take(sizeof(float) * n * B * K));
      ws.wsum = reinterpret_cast<float*>(take(sizeof(float) * n));
      if (mixed) {
        ws.blo = reinterpret_cast<float*>(take(sizeof(float) * n * B * K));
        ws.wlo = reinterpret_cast<float*>(take(sizeof(float) * n));
      }
    }
    ws.payload = reinterpret_cast<float*>(take(sizeof(float) * (size_t)cbn * K));
    ws.img = reinterpret_cast<float*>(take(sizeof(float) * (size_t)p.cam_batch * p.width * p.height * K));
  }
  if (need & kNeedBackward) {
    ws.payload = reinterpret_cast<float*>(take(sizeof(float) * (size_t)cbn * (K + 1)));
    ws.u = reinterpret_cast<float*>(take(sizeof(float) * n * B * K));
    ws.u_lo = reinterpret_cast<float*>(take(sizeof(float) * n * B * K));
    ws.reg = reinterpret_cast<float*>(take(sizeof(float) * n));
  } else if (need & kNeedRender) {
    ws.payload = reinterpret_cast<float*>(take(sizeof(float) * (size_t)cbn * K));
  }
  ws.total = off;
  ws.bytes = off;
  return ws;
}

bool finite_all(const float* v, size_t m) {
  for (size_t i = 0; i < m; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

icgs_status setup(const icgs_scene* sc, const icgs_cameras* cams, int K, int L, int precision,
                  float cond_tau, float refold_tau, int cam_batch, int64_t capacity, Problem& p) {
  if (!sc || !cams) return fail(ICGS_ERR_INVALID_ARG, "scene and cameras must not be NULL");
  if (sc->n < 0 || sc->n > 0x7FFFFFFF) return fail(ICGS_ERR_INVALID_ARG, "scene.n = %lld out of range", (long long)sc->n);
  if (sc->n > 0 && (!sc->means || !sc->scales || !sc->quats || !sc->opacity))
    return fail(ICGS_ERR_INVALID_ARG, "scene arrays must not be NULL");
  if (cams->n_cams < 1) return fail(ICGS_ERR_INVALID_ARG, "n_cams = %d must be >= 1", cams->n_cams);
  if (cams->width < 1 || cams->height < 1 || cams->width > 65535 * kTile || cams->height > 65535 * kTile)
    return fail(ICGS_ERR_INVALID_ARG, "image size %dx%d out of range", cams->width, cams->height);
  if (!cams->intrinsics || !cams->world_to_cam) return fail(ICGS_ERR_INVALID_ARG, "camera arrays must not be NULL");
  if (!finite_all(cams->intrinsics, 4 * (size_t)cams->n_cams) || !finite_all(cams->world_to_cam, 12 * (size_t)cams->n_cams))
    return fail(ICGS_ERR_INVALID_ARG, "camera parameters must be finite");
  for (int j = 0; j < cams->n_cams; ++j)
    if (!(cams->intrinsics[4 * j] > 0.0f) || !(cams->intrinsics[4 * j + 1] > 0.0f))
      return fail(ICGS_ERR_INVALID_ARG, "camera %d: focal lengths must be > 0", j);
  if (K < 1) return fail(ICGS_ERR_INVALID_ARG, "channels = %d must be >= 1", K);
  if (L < 0 || L > 3) return fail(ICGS_ERR_INVALID_ARG, "sh_degree = %d must be in 0..3", L);
  if (precision != ICGS_PRECISION_PLAIN && precision != ICGS_PRECISION_MIXED)
    return fail(ICGS_ERR_INVALID_ARG, "precision = %d is not an icgs_precision", precision);
  p.n = sc->n;
  p.n_cams = cams->n_cams;
  p.width = cams->width;
  p.height = cams->height;
  p.near_z = cams->near_z > 0.0f ? cams->near_z : 0.2f;
  p.tiles_x = (p.width + kTile - 1) / kTile;
  p.tiles_y = (p.height + kTile - 1) / kTile;
  p.tiles = p.tiles_x * p.tiles_y;
  p.K = K;
  p.acc_stride = (1 + K + 3) & ~3;
  p.L = L;
  p.B = (L + 1) * (L + 1);
  p.precision = precision;
  p.cond_tau = cond_tau > 0.0f ? cond_tau : 1e-3f;
  p.refold_tau = refold_tau > 0.0f ? refold_tau : 0.0f;
  p.cam_batch = cam_batch > 0 ? std::min(cam_batch, p.n_cams) : std::min(p.n_cams, 128);
  p.cam_batch = std::min(p.cam_batch, 65535);  // grid y dimension of the per-pair kernels
  if ((int64_t)p.cam_batch * p.tiles > 0x7FFFFFFFll)
    return fail(ICGS_ERR_INVALID_ARG, "cam_batch x tiles too large; lower cam_batch");
  int64_t cap = capacity > 0 ? capacity : 6 * (int64_t)p.n * p.cam_batch + (1 << 16);
  p.capacity = (uint32_t)std::min<int64_t>(cap, kMaxCapacity);
  return ICGS_OK;
}

std::vector<DevCam> build_cams(const icgs_cameras* cams) {
  std::vector<DevCam> out((size_t)cams->n_cams);
  for (int j = 0; j < cams->n_cams; ++j) {
    DevCam& c = out[(size_t)j];
    std::memset(&c, 0, sizeof c);
    const float* in = cams->intrinsics + 4 * j;
    const float* w = cams->world_to_cam + 12 * j;
    c.fx = in[0]; c.fy = in[1]; c.cx = in[2]; c.cy = in[3];
    for (int k = 0; k < 12; ++k) c.w[k] = w[k];
    for (int a = 0; a < 3; ++a) {  // centre = -R^T t
      double s = 0.0;
      for (int r = 0; r < 3; ++r) s -= (double)w[4 * r + a] * (double)w[4 * r + 3];
      c.centre[a] = (float)s;
      c.centre_d[a] = s;
    }
    c.limx = (float)(1.3 * ((double)cams->width / (2.0 * (double)in[0])));
    c.limy = (float)(1.3 * ((double)cams->height / (2.0 * (double)in[1])));
    // upper bound on the squared spectral norm of R: the largest absolute row sum of R^T R
    // (Gershgorin; exactly 1 for a rotation)
    double bound = 0.0;
    for (int a = 0; a < 3; ++a) {
      double row = 0.0;
      for (int b = 0; b < 3; ++b) {
        double g = 0.0;
        for (int r = 0; r < 3; ++r) g += (double)w[4 * r + a] * (double)w[4 * r + b];
        row += std::fabs(g);
      }
      bound = std::max(bound, row);
    }
    c.rnorm2 = (float)(bound * (1.0 + 1e-6));
  }
  return out;
}

void default_lambda(int L, float* lam) {
  const float band[4] = {1e-5f, 1e-4f, 1e-3f, 1e-2f};  // Sec. 4, Implementation Details
  for (int l = 0; l <= L; ++l)
    for (int m = -l; m <= l; ++m) lam[l * l + l + m] = band[l];
}

// The camera table and lambda travel to the workspace as kernel parameters (copied at launch, up to
// 32 KB on sm_70 and later), so no call waits on, or keeps alive, pageable host memory.
constexpr int kUploadCams = 128;
struct UploadBatch {
  DevCam cams[kUploadCams];
  float lam[kMaxSH];
  int count;  // cameras in this batch
  int n_lam;  // lambda entries (first batch only)
};
static_assert(sizeof(UploadBatch) + 2 * sizeof(void*) <= 32000, "kernel parameter space");

__global__ void k_upload(const UploadBatch batch, DevCam* __restrict__ dst, float* __restrict__ lam_dst) {
  const int t = threadIdx.x;
  if (t < batch.count) dst[t] = batch.cams[t];
  if (t < batch.n_lam) lam_dst[t] = batch.lam[t];
}

icgs_status upload_common(const Problem& p, const icgs_cameras* cams, const float* lam_host,
                          const Workspace& ws, cudaStream_t s) {
  const std::vector<DevCam> dc = build_cams(cams);
  g_launches = 0;
  ICGS_TRY_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(DevStatus), s));
  UploadBatch batch;
  for (size_t j0 = 0; j0 < dc.size(); j0 += kUploadCams) {
    std::memset(&batch, 0, sizeof batch);
    batch.count = (int)std::min(dc.size() - j0, (size_t)kUploadCams);
    std::memcpy(batch.cams, dc.data() + j0, sizeof(DevCam) * (size_t)batch.count);
    if (j0 == 0 && lam_host) {
      batch.n_lam = p.B;
      std::memcpy(batch.lam, lam_host, sizeof(float) * (size_t)p.B);
    }
    k_upload<<<1, kUploadCams, 0, s>>>(batch, ws.cams + j0, ws.lam);
    ICGS_TRY_CUDA(cudaGetLastError());
    icgs::note_launches(1);
  }
  g_timer.begin(s);
  return ICGS_OK;
}

// Projection, binning and the depth sort of every tile list (the walks read the sorted lists from
// global memory). first: the call's first pass, which also computes the Gaussians' processing order.
icgs_status bin_pass(const Problem& p, const icgs_scene* sc, int cb, bool first, const Workspace& wp, cudaStream_t s) {
  const int64_t ct = (int64_t)cb * p.tiles;
  if (first) launch_spatial_order(p, sc->means, sc->scales, sc->quats, sc->opacity, wp, s);
  ICGS_TRY_CUDA(cudaMemsetAsync(wp.tile_off, 0, sizeof(uint32_t) * (size_t)(ct + 1), s));
  ICGS_TRY_CUDA(cudaMemsetAsync(wp.tile_cur, 0, sizeof(uint32_t) * (size_t)ct, s));
  launch_project(p, sc->means, sc->scales, sc->quats, sc->opacity, cb, wp, s);
  g_timer.mark(kProject, s);
  launch_scan(p, cb, wp, s);
  g_timer.mark(kScan, s);
  launch_scatter(p, cb, wp, s);
  g_timer.mark(kScatter, s);
  launch_tile_sort(p, cb, wp, s);
  g_timer.mark(kSort, s);
  return ICGS_OK;
}

// The outcome a call's device status block reports (read back after the work has finished).
icgs_status status_of(const DevStatus& st) {
  g_required = (int64_t)st.instances_needed;
  if (st.flags & kFlagTimeout)
    return fail(ICGS_ERR_DEVICE_TIMEOUT, "a bounded wait for the tensor-core MMAs gave up");
  if (st.flags & kFlagLayout)
    return fail(ICGS_ERR_UNSUPPORTED, "the tensor-core walk needs a 128-byte aligned dynamic shared memory base");
  if (st.flags & kFlagOverflow)
    return fail(ICGS_ERR_CAPACITY, "a pass needed %lld (Gaussian, tile) instances; pass at least that as "
                "icgs_options.instance_capacity", (long long)st.instances_needed);
  if (st.flags & kFlagNonfinite)
    return fail(ICGS_ERR_NONFINITE_INPUT, "a target value read by the walk is NaN or infinite");
  g_stats[0] = (int64_t)st.instances_total;
  g_stats[1] = (int64_t)st.contrib_pairs;
  g_stats[2] = (int64_t)st.fp64_count;
  g_stats[3] = g_launches;
  g_stats[4] = (int64_t)st.refold_count;
  return ICGS_OK;
}

// End of a call: synchronous calls copy the status block back and synchronise `s`; enqueue-only
// calls (sync false) only check that every launch was accepted.
icgs_status finish(const Workspace& ws, cudaStream_t s, bool sync = true) {
  ICGS_TRY_CUDA(cudaGetLastError());
  if (!sync) return ICGS_OK;
  DevStatus st;
  ICGS_TRY_CUDA(cudaMemcpyAsync(&st, ws.status, sizeof st, cudaMemcpyDeviceToHost, s));
  ICGS_TRY_CUDA(cudaStreamSynchronize(s));
  g_timer.collect();
  return status_of(st);
}

// Enqueue-only calls record no stage events (reading them back needs a synchronisation).
struct TimerPause {
  bool was;
  explicit TimerPause(bool pause) : was(g_timer.on) {
    if (pause) g_timer.on = false;
  }
  ~TimerPause() { g_timer.on = was; }
};

icgs_status check_targets(const icgs_targets* t) {
  if (!t || !t->data) return fail(ICGS_ERR_INVALID_ARG, "targets must not be NULL");
  if (t->dtype != ICGS_F32 && t->dtype != ICGS_BF16 && t->dtype != ICGS_F16)
    return fail(ICGS_ERR_INVALID_ARG, "targets.dtype = %d is not an icgs_dtype", (int)t->dtype);
  if (t->channels < 1) return fail(ICGS_ERR_INVALID_ARG, "targets.channels = %d must be >= 1", t->channels);
  return ICGS_OK;
}

icgs_status lambda_of(const icgs_options* opt, int L, float* lam) {
  const int B = (L + 1) * (L + 1);
  if (opt && opt->lambda) {
    for (int m = 0; m < B; ++m) {
      lam[m] = opt->lambda[m];
      if (!(lam[m] >= 0.0f) || !std::isfinite(lam[m]))
        return fail(ICGS_ERR_INVALID_ARG, "lambda[%d] must be finite and >= 0", m);
    }
  } else {
    default_lambda(L, lam);
  }
  return ICGS_OK;
}

}  // namespace

void icgs::note_launches(int count) { g_launches += count; }

size_t icgs::colorize_workspace_bytes(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                                      const icgs_options* opt) {
  if (!targets || !opt) return 0;
  Problem p;
  if (setup(scene, cams, targets->channels, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau, opt->cam_batch,
            opt->instance_capacity, p) != ICGS_OK)
    return 0;
  return carve(nullptr, p, kNeedAccumulate).total;
}

void icgs::set_error_message(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

extern "C" {

size_t icgs_workspace_size(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                           const icgs_options* opt) {
  if (!targets || !opt) return 0;
  Problem p;
  if (setup(scene, cams, targets->channels, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau, opt->cam_batch,
            opt->instance_capacity, p) != ICGS_OK)
    return 0;
  return carve(nullptr, p, kNeedAccumulate | kNeedBackward).total;
}

static icgs_status colorize_impl(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                                 const icgs_options* opt, void* workspace, size_t workspace_bytes, float* coeffs_out,
                                 uint8_t* status_out, float* chol_out, void* stream, bool sync) {
  TimerPause pause(!sync);
  g_err[0] = '\0';
  if (!opt) return fail(ICGS_ERR_INVALID_ARG, "options must not be NULL");
  icgs_status st = check_targets(targets);
  if (st != ICGS_OK) return st;
  Problem p;
  st = setup(scene, cams, targets->channels, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau, opt->cam_batch,
             opt->instance_capacity, p);
  if (st != ICGS_OK) return st;
  if (!coeffs_out && p.n > 0) return fail(ICGS_ERR_INVALID_ARG, "coeffs_out must not be NULL");
  float lam[kMaxSH];
  if ((st = lambda_of(opt, p.L, lam)) != ICGS_OK) return st;
  const Workspace need = carve(nullptr, p, kNeedAccumulate);
  if (!workspace || workspace_bytes < need.total)
    return fail(ICGS_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", workspace_bytes, need.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Workspace ws = carve(static_cast<char*>(workspace), p, kNeedAccumulate);
  if (p.n == 0) return ICGS_OK;
  if ((st = upload_common(p, cams, lam, ws, s)) != ICGS_OK) return st;
  if (p.L == 0)
    ICGS_TRY_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(float) * (size_t)p.n * p.acc_stride, s));
  for (int cam0 = 0; cam0 < p.n_cams; cam0 += p.cam_batch) {
    const int cb = std::min(p.cam_batch, p.n_cams - cam0);
    Workspace wp = ws;
    wp.cams = ws.cams + cam0;
    if (p.L > 0)
      ICGS_TRY_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(float) * (size_t)cb * (size_t)p.n * p.acc_stride, s));
    if ((st = bin_pass(p, scene, cb, cam0 == 0, wp, s)) != ICGS_OK) return st;
    launch_blend_accumulate(p, cb, cam0, targets->data, (int)targets->dtype, nullptr, wp, s);
    g_timer.mark(kBlend, s);
    if (p.L > 0) {
      launch_fold(p, scene->means, cb, cam0 == 0, true, wp, s);
      g_timer.mark(kFold, s);
    }
  }
  launch_solve(p, ws.lam, lam, ws, coeffs_out, status_out, chol_out, scene->means,
               p.cam_batch >= p.n_cams ? p.n_cams : 0, s);
  g_timer.mark(kSolve, s);
  return finish(ws, s, sync);
}

namespace {

// ---- target sets: several target images on one geometry ----
constexpr int kMaxSets = 64;

icgs_status check_sets(int32_t n_sets, const icgs_targets* sets, int& K_total) {
  if (n_sets < 1 || n_sets > kMaxSets || !sets)
    return fail(ICGS_ERR_INVALID_ARG, "n_sets = %d must be in 1..%d with a sets array", n_sets, kMaxSets);
  K_total = 0;
  for (int k = 0; k < n_sets; ++k) {
    icgs_status st = check_targets(&sets[k]);
    if (st != ICGS_OK) return st;
    K_total += sets[k].channels;
  }
  return ICGS_OK;
}

int acc_stride_of(int K) { return (1 + K + 3) & ~3; }

// Rows of an accumulator: one per Gaussian (L = 0, summed over every pass) or per (camera of the
// pass, Gaussian) (L > 0, folded after each pass).
int64_t acc_rows(const Problem& p) { return p.L == 0 ? p.n : (int64_t)p.cam_batch * p.n; }

// Bytes of the per-set accumulator regions that follow the colorize workspace of the combined
// channels; offs (nullable) receives each region's offset from the end of that workspace.
size_t set_regions(const Problem& p, int32_t n_sets, const icgs_targets* sets, size_t* offs) {
  size_t off = 0;
  for (int k = 0; k < n_sets; ++k) {
    if (offs) offs[k] = off;
    off += align256(sizeof(float) * (size_t)acc_rows(p) * (size_t)acc_stride_of(sets[k].channels));
  }
  return off;
}

}  // namespace

size_t icgs_sets_workspace_size(const icgs_scene* scene, const icgs_cameras* cams, int32_t n_sets,
                                const icgs_targets* sets, const icgs_options* opt) {
  int K = 0;
  if (!opt || check_sets(n_sets, sets, K) != ICGS_OK) return 0;
  Problem p;
  if (setup(scene, cams, K, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau, opt->cam_batch,
            opt->instance_capacity, p) != ICGS_OK)
    return 0;
  return carve(nullptr, p, kNeedAccumulate).total + set_regions(p, n_sets, sets, nullptr);
}

icgs_status icgs_colorize_sets(const icgs_scene* scene, const icgs_cameras* cams, int32_t n_sets,
                               const icgs_targets* sets, const icgs_options* opt, void* workspace,
                               size_t workspace_bytes, float* coeffs_out, uint8_t* status_out, float* chol_out,
                               float threshold, uint8_t* keep_out, void* stream) {
  g_err[0] = '\0';
  if (!opt) return fail(ICGS_ERR_INVALID_ARG, "options must not be NULL");
  int K = 0;
  icgs_status st = check_sets(n_sets, sets, K);
  if (st != ICGS_OK) return st;
  Problem p;
  st = setup(scene, cams, K, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau, opt->cam_batch,
             opt->instance_capacity, p);
  if (st != ICGS_OK) return st;
  if (!coeffs_out && p.n > 0) return fail(ICGS_ERR_INVALID_ARG, "coeffs_out must not be NULL");
  if (keep_out && p.L != 0)
    return fail(ICGS_ERR_UNSUPPORTED, "the threshold epilogue needs sh_degree 0 (view-independent values)");
  if (!std::isfinite(threshold)) return fail(ICGS_ERR_INVALID_ARG, "threshold must be finite");
  float lam[kMaxSH];
  if ((st = lambda_of(opt, p.L, lam)) != ICGS_OK) return st;
  size_t offs[kMaxSets];
  const size_t base_bytes = carve(nullptr, p, kNeedAccumulate).total;
  const size_t need = base_bytes + set_regions(p, n_sets, sets, offs);
  if (!workspace || workspace_bytes < need)
    return fail(ICGS_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", workspace_bytes, need);
  if (reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(workspace);
  const Workspace ws = carve(base, p, kNeedAccumulate);
  float* set_acc[kMaxSets];
  Problem ps[kMaxSets];
  for (int k = 0, col0 = 0; k < n_sets; col0 += sets[k].channels, ++k) {
    set_acc[k] = reinterpret_cast<float*>(base + base_bytes + offs[k]);
    ps[k] = p;
    ps[k].K = sets[k].channels;
    ps[k].acc_stride = acc_stride_of(sets[k].channels);
  }
  if (p.n == 0) return ICGS_OK;
  if ((st = upload_common(p, cams, lam, ws, s)) != ICGS_OK) return st;
  auto zero_accs = [&](int64_t rows) -> icgs_status {
    ICGS_TRY_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(float) * (size_t)rows * p.acc_stride, s));
    for (int k = 0; k < n_sets; ++k)
      ICGS_TRY_CUDA(cudaMemsetAsync(set_acc[k], 0, sizeof(float) * (size_t)rows * ps[k].acc_stride, s));
    return ICGS_OK;
  };
  auto merge_all = [&](int64_t rows) {
    for (int k = 0, col0 = 0; k < n_sets; col0 += sets[k].channels, ++k)
      launch_merge_set(rows, ps[k].K, ps[k].acc_stride, set_acc[k], p.acc_stride, col0, ws.acc, s);
  };
  if (p.L == 0 && (st = zero_accs(p.n)) != ICGS_OK) return st;
  for (int cam0 = 0; cam0 < p.n_cams; cam0 += p.cam_batch) {
    const int cb = std::min(p.cam_batch, p.n_cams - cam0);
    Workspace wp = ws;
    wp.cams = ws.cams + cam0;
    if (p.L > 0 && (st = zero_accs((int64_t)cb * p.n)) != ICGS_OK) return st;
    if ((st = bin_pass(p, scene, cb, cam0 == 0, wp, s)) != ICGS_OK) return st;  // one binning for every set
    for (int k = 0; k < n_sets; ++k) {
      Workspace wk = wp;
      wk.acc = set_acc[k];
      launch_blend_accumulate(ps[k], cb, cam0, sets[k].data, (int)sets[k].dtype, nullptr, wk, s);
    }
    g_timer.mark(kBlend, s);
    if (p.L > 0) {
      merge_all((int64_t)cb * p.n);
      launch_fold(p, scene->means, cb, cam0 == 0, true, wp, s);
      g_timer.mark(kFold, s);
    }
  }
  if (p.L == 0) merge_all(p.n);
  launch_solve(p, ws.lam, lam, ws, coeffs_out, status_out, chol_out, scene->means,
               p.cam_batch >= p.n_cams ? p.n_cams : 0, s, threshold, keep_out);
  g_timer.mark(kSolve, s);
  return finish(ws, s);
}

namespace {

// Copy streams and event pool of icgs_colorize_host, one set per host thread and device.
struct HostPipe {
  int device = -1;
  cudaStream_t copy[2] = {nullptr, nullptr};  // chunks alternate between two copy streams
  cudaEvent_t start = nullptr;
  std::vector<cudaEvent_t> ready;
};
thread_local HostPipe g_pipe;

constexpr int kHostChunks = 8;  // camera chunks per pass: copy of chunk c+1 overlaps the walk of c

icgs_status host_pipe(int n_events, HostPipe*& out) {
  int dev = 0;
  ICGS_TRY_CUDA(cudaGetDevice(&dev));
  HostPipe& hp = g_pipe;
  if (hp.device != dev) {  // first use on this thread, or another device: a fresh stream and pool
    hp = HostPipe();
    for (int k = 0; k < 2; ++k) ICGS_TRY_CUDA(cudaStreamCreateWithFlags(&hp.copy[k], cudaStreamNonBlocking));
    ICGS_TRY_CUDA(cudaEventCreateWithFlags(&hp.start, cudaEventDisableTiming));
    hp.device = dev;
  }
  while ((int)hp.ready.size() < n_events) {
    cudaEvent_t e;
    ICGS_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    hp.ready.push_back(e);
  }
  out = &hp;
  return ICGS_OK;
}

size_t target_elem_bytes(int dtype) { return dtype == ICGS_F32 ? 4 : 2; }

// Sizes of the regions icgs_colorize_host adds after the colorize workspace: the staged targets,
// the coefficients and the status bytes.
void host_regions(const Problem& p, int dtype, size_t& t_bytes, size_t& c_bytes, size_t& s_bytes) {
  t_bytes = align256((size_t)p.n_cams * p.height * p.width * p.K * target_elem_bytes(dtype));
  c_bytes = align256((size_t)p.n * p.B * p.K * sizeof(float));
  s_bytes = align256((size_t)p.n);
}

}  // namespace

size_t icgs_colorize_host_workspace_size(const icgs_scene* scene, const icgs_cameras* cams,
                                         const icgs_targets* targets, const icgs_options* opt) {
  if (!targets || !opt) return 0;
  Problem p;
  if (setup(scene, cams, targets->channels, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau,
            opt->cam_batch, opt->instance_capacity, p) != ICGS_OK)
    return 0;
  size_t t_bytes, c_bytes, s_bytes;
  host_regions(p, (int)targets->dtype, t_bytes, c_bytes, s_bytes);
  return carve(nullptr, p, kNeedAccumulate).total + t_bytes + c_bytes + s_bytes;
}

icgs_status icgs_colorize_host(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                               const icgs_options* opt, void* workspace, size_t workspace_bytes, float* coeffs_host,
                               uint8_t* status_host, float* chol_out, void* stream) {
  g_err[0] = '\0';
  if (!opt) return fail(ICGS_ERR_INVALID_ARG, "options must not be NULL");
  icgs_status st = check_targets(targets);
  if (st != ICGS_OK) return st;
  Problem p;
  st = setup(scene, cams, targets->channels, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau,
             opt->cam_batch, opt->instance_capacity, p);
  if (st != ICGS_OK) return st;
  if (!coeffs_host && p.n > 0) return fail(ICGS_ERR_INVALID_ARG, "coeffs_host must not be NULL");
  float lam[kMaxSH];
  if ((st = lambda_of(opt, p.L, lam)) != ICGS_OK) return st;
  const Workspace need = carve(nullptr, p, kNeedAccumulate);
  size_t t_bytes, c_bytes, s_bytes;
  const int dtype = (int)targets->dtype;
  host_regions(p, dtype, t_bytes, c_bytes, s_bytes);
  const size_t total = need.total + t_bytes + c_bytes + s_bytes;
  if (!workspace || workspace_bytes < total)
    return fail(ICGS_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", workspace_bytes, total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(workspace);
  const Workspace ws = carve(base, p, kNeedAccumulate);
  char* t_dev = base + need.total;
  float* c_dev = reinterpret_cast<float*>(t_dev + t_bytes);
  uint8_t* st_dev = reinterpret_cast<uint8_t*>(t_dev + t_bytes + c_bytes);
  if (p.n == 0) return ICGS_OK;
  const size_t cam_bytes = (size_t)p.height * p.width * p.K * target_elem_bytes(dtype);
  const char* t_host = static_cast<const char*>(targets->data);

  // camera chunks of every pass, in order; chunk c of the whole call waits on ready[c]
  std::vector<int> chunk_cam0, chunk_n;
  for (int cam0 = 0; cam0 < p.n_cams; cam0 += p.cam_batch) {
    const int cb = std::min(p.cam_batch, p.n_cams - cam0);
    const int per = std::max(1, (cb + kHostChunks - 1) / kHostChunks);
    for (int j0 = 0; j0 < cb; j0 += per) {
      chunk_cam0.push_back(cam0 + j0);
      chunk_n.push_back(std::min(per, cb - j0));
    }
  }
  HostPipe* hp = nullptr;
  if ((st = host_pipe((int)chunk_cam0.size(), hp)) != ICGS_OK) return st;
  // the staging buffer is overwritten only after the work already queued on `stream` (which may
  // read it) has finished
  ICGS_TRY_CUDA(cudaEventRecord(hp->start, s));
  for (int k = 0; k < 2; ++k) ICGS_TRY_CUDA(cudaStreamWaitEvent(hp->copy[k], hp->start, 0));
  // Copies are enqueued kCopyAhead chunks ahead of the walk that reads them, interleaved with the
  // compute launches: from page-locked memory every call returns at once and the copies run
  // behind the binning and the walks; from pageable memory, where each copy holds the host until
  // it is done, the walks already enqueued still run while the next chunk is copied.
  constexpr size_t kCopyAhead = 2;
  size_t copied = 0;
  auto enqueue_copy = [&]() -> icgs_status {
    if (copied >= chunk_cam0.size()) return ICGS_OK;
    const size_t off = (size_t)chunk_cam0[copied] * cam_bytes;
    cudaStream_t cs = hp->copy[copied & 1];
    ICGS_TRY_CUDA(cudaMemcpyAsync(t_dev + off, t_host + off, (size_t)chunk_n[copied] * cam_bytes,
                                  cudaMemcpyHostToDevice, cs));
    ICGS_TRY_CUDA(cudaEventRecord(hp->ready[copied], cs));
    ++copied;
    return ICGS_OK;
  };
  for (size_t k = 0; k < kCopyAhead; ++k)
    if ((st = enqueue_copy()) != ICGS_OK) return st;

  if ((st = upload_common(p, cams, lam, ws, s)) != ICGS_OK) return st;
  if (p.L == 0)
    ICGS_TRY_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(float) * (size_t)p.n * p.acc_stride, s));
  size_t chunk = 0;
  for (int cam0 = 0; cam0 < p.n_cams; cam0 += p.cam_batch) {
    const int cb = std::min(p.cam_batch, p.n_cams - cam0);
    Workspace wp = ws;
    wp.cams = ws.cams + cam0;
    if (p.L > 0)
      ICGS_TRY_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(float) * (size_t)cb * (size_t)p.n * p.acc_stride, s));
    // projection, binning and sorting need no targets: they run while the first chunks arrive
    if ((st = bin_pass(p, scene, cb, cam0 == 0, wp, s)) != ICGS_OK) return st;
    for (; chunk < chunk_cam0.size() && chunk_cam0[chunk] < cam0 + cb; ++chunk) {
      const int j0 = chunk_cam0[chunk] - cam0, jc = chunk_n[chunk];
      while (copied < chunk_cam0.size() && copied < chunk + 1 + kCopyAhead)
        if ((st = enqueue_copy()) != ICGS_OK) return st;
      ICGS_TRY_CUDA(cudaStreamWaitEvent(s, hp->ready[chunk], 0));
      Workspace wc = wp;  // the chunk's cameras are a contiguous slice of the pass
      wc.tile_off = wp.tile_off + (size_t)j0 * p.tiles;
      wc.rec = wp.rec + (size_t)j0 * p.n;
      if (p.L > 0) wc.acc = wp.acc + (size_t)j0 * p.n * p.acc_stride;
      launch_blend_accumulate(p, jc, cam0 + j0, t_dev, dtype, nullptr, wc, s);
    }
    g_timer.mark(kBlend, s);
    if (p.L > 0) {
      launch_fold(p, scene->means, cb, cam0 == 0, true, wp, s);
      g_timer.mark(kFold, s);
    }
  }
  launch_solve(p, ws.lam, lam, ws, c_dev, st_dev, chol_out, scene->means, p.cam_batch >= p.n_cams ? p.n_cams : 0,
               s);
  g_timer.mark(kSolve, s);
  ICGS_TRY_CUDA(cudaMemcpyAsync(coeffs_host, c_dev, (size_t)p.n * p.B * p.K * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (status_host) ICGS_TRY_CUDA(cudaMemcpyAsync(status_host, st_dev, (size_t)p.n, cudaMemcpyDeviceToHost, s));
  return finish(ws, s);
}

int64_t icgs_normal_size(int32_t sh_degree, int32_t channels) {
  if (sh_degree < 0 || sh_degree > 3 || channels < 1) return 0;
  const int64_t B = (int64_t)(sh_degree + 1) * (sh_degree + 1);
  return B * (B + 1) / 2 + B * channels + 1;
}

icgs_status icgs_accumulate(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                            const icgs_options* opt, void* workspace, size_t workspace_bytes, double* sums_out,
                            void* stream) {
  g_err[0] = '\0';
  if (!opt) return fail(ICGS_ERR_INVALID_ARG, "options must not be NULL");
  icgs_status st = check_targets(targets);
  if (st != ICGS_OK) return st;
  Problem p;
  st = setup(scene, cams, targets->channels, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau,
             opt->cam_batch, opt->instance_capacity, p);
  if (st != ICGS_OK) return st;
  if (!sums_out && p.n > 0) return fail(ICGS_ERR_INVALID_ARG, "sums_out is required");
  const Workspace need = carve(nullptr, p, kNeedAccumulate);
  if (!workspace || workspace_bytes < need.total)
    return fail(ICGS_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", workspace_bytes, need.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Workspace ws = carve(static_cast<char*>(workspace), p, kNeedAccumulate);
  if (p.n == 0) return ICGS_OK;
  if ((st = upload_common(p, cams, nullptr, ws, s)) != ICGS_OK) return st;
  if (p.L == 0)
    ICGS_TRY_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(float) * (size_t)p.n * p.acc_stride, s));
  for (int cam0 = 0; cam0 < p.n_cams; cam0 += p.cam_batch) {
    const int cb = std::min(p.cam_batch, p.n_cams - cam0);
    Workspace wp = ws;
    wp.cams = ws.cams + cam0;
    if (p.L > 0)
      ICGS_TRY_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(float) * (size_t)cb * (size_t)p.n * p.acc_stride, s));
    if ((st = bin_pass(p, scene, cb, cam0 == 0, wp, s)) != ICGS_OK) return st;
    launch_blend_accumulate(p, cb, cam0, targets->data, (int)targets->dtype, nullptr, wp, s);
    g_timer.mark(kBlend, s);
    if (p.L > 0) {
      launch_fold(p, scene->means, cb, cam0 == 0, true, wp, s);
      g_timer.mark(kFold, s);
    }
  }
  launch_export_normal(p, ws, sums_out, s);
  return finish(ws, s);
}

namespace {

// Workspace of icgs_solve: the status block, lambda and the normal equations in the layout the
// solve kernels read (hi, lo for MIXED; for L = 0 one accumulator row per Gaussian).
Workspace carve_solve(char* base, const Problem& p) {
  Workspace ws;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* ptr = base ? base + off : nullptr;
    off += align256(bytes);
    return ptr;
  };
  const size_t B = (size_t)p.B, K = (size_t)p.K, n = (size_t)p.n;
  ws.base = base;
  ws.status = reinterpret_cast<DevStatus*>(take(sizeof(DevStatus)));
  ws.lam = reinterpret_cast<float*>(take(sizeof(float) * kMaxSH));
  if (p.L == 0) {
    ws.acc = reinterpret_cast<float*>(take(sizeof(float) * n * (size_t)p.acc_stride));
  } else {
    const bool mixed = p.precision == ICGS_PRECISION_MIXED;
    ws.G = reinterpret_cast<float*>(take(sizeof(float) * n * B * B));
    ws.bvec = reinterpret_cast<float*>(take(sizeof(float) * n * B * K));
    ws.wsum = reinterpret_cast<float*>(take(sizeof(float) * n));
    if (mixed) {
      ws.Glo = reinterpret_cast<float*>(take(sizeof(float) * n * B * B));
      ws.blo = reinterpret_cast<float*>(take(sizeof(float) * n * B * K));
      ws.wlo = reinterpret_cast<float*>(take(sizeof(float) * n));
    }
  }
  ws.total = off;
  ws.bytes = off;
  return ws;
}

icgs_status setup_solve(int64_t n, int32_t sh_degree, int32_t channels, const icgs_options* opt, Problem& p) {
  if (!opt) return fail(ICGS_ERR_INVALID_ARG, "options must not be NULL");
  if (n < 0) return fail(ICGS_ERR_INVALID_ARG, "n = %lld must be >= 0", (long long)n);
  if (sh_degree < 0 || sh_degree > 3) return fail(ICGS_ERR_INVALID_ARG, "sh_degree = %d must be in 0..3", sh_degree);
  if (channels < 1) return fail(ICGS_ERR_INVALID_ARG, "channels = %d must be >= 1", channels);
  if (opt->precision != ICGS_PRECISION_PLAIN && opt->precision != ICGS_PRECISION_MIXED)
    return fail(ICGS_ERR_INVALID_ARG, "precision = %d is not an icgs_precision", opt->precision);
  p = Problem();
  p.n = n;
  p.L = sh_degree;
  p.B = (sh_degree + 1) * (sh_degree + 1);
  p.K = channels;
  p.acc_stride = (1 + channels + 3) & ~3;
  p.precision = opt->precision;
  p.cond_tau = opt->cond_tau > 0.0f ? opt->cond_tau : 1e-3f;
  return ICGS_OK;
}

}  // namespace

size_t icgs_solve_workspace_size(int64_t n, int32_t sh_degree, int32_t channels, const icgs_options* opt) {
  Problem p;
  if (setup_solve(n, sh_degree, channels, opt, p) != ICGS_OK) return 0;
  return carve_solve(nullptr, p).total;
}

icgs_status icgs_solve(int64_t n, int32_t sh_degree, int32_t channels, const double* sums, const icgs_options* opt,
                       void* workspace, size_t workspace_bytes, float* coeffs_out, uint8_t* status_out,
                       float* chol_out, void* stream) {
  g_err[0] = '\0';
  Problem p;
  icgs_status st = setup_solve(n, sh_degree, channels, opt, p);
  if (st != ICGS_OK) return st;
  if (p.n > 0 && (!sums || !coeffs_out)) return fail(ICGS_ERR_INVALID_ARG, "sums and coeffs_out are required");
  float lam[kMaxSH];
  if ((st = lambda_of(opt, p.L, lam)) != ICGS_OK) return st;
  const Workspace need = carve_solve(nullptr, p);
  if (!workspace || workspace_bytes < need.total)
    return fail(ICGS_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", workspace_bytes, need.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Workspace ws = carve_solve(static_cast<char*>(workspace), p);
  if (p.n == 0) return ICGS_OK;
  g_launches = 0;
  ICGS_TRY_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(DevStatus), s));
  ICGS_TRY_CUDA(cudaMemcpyAsync(ws.lam, lam, sizeof(float) * p.B, cudaMemcpyHostToDevice, s));
  g_timer.begin(s);
  launch_import_normal(p, ws, sums, s);
  // the per-camera sums are not available here: no exact re-fold, FP64 below cond_tau
  launch_solve(p, ws.lam, lam, ws, coeffs_out, status_out, chol_out, nullptr, 0, s);
  g_timer.mark(kSolve, s);
  return finish(ws, s);
}

static icgs_status backward_impl(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                                 const icgs_options* opt, const float* coeffs, const float* chol,
                                 const float* grad_coeffs, void* workspace, size_t workspace_bytes,
                                 float* grad_targets, float* grad_opacity, void* stream, bool sync) {
  TimerPause pause(!sync);
  g_err[0] = '\0';
  if (!opt) return fail(ICGS_ERR_INVALID_ARG, "options must not be NULL");
  icgs_status st = check_targets(targets);
  if (st != ICGS_OK) return st;
  Problem p;
  st = setup(scene, cams, targets->channels, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau, opt->cam_batch,
             opt->instance_capacity, p);
  if (st != ICGS_OK) return st;
  if (p.K > 64) return fail(ICGS_ERR_UNSUPPORTED, "the adjoint supports up to 64 channels, got %d", p.K);
  if ((!coeffs || !chol || !grad_coeffs) && p.n > 0)
    return fail(ICGS_ERR_INVALID_ARG, "coeffs, chol and grad_coeffs are required");
  float lam[kMaxSH];
  if ((st = lambda_of(opt, p.L, lam)) != ICGS_OK) return st;
  const Workspace need = carve(nullptr, p, kNeedBackward);
  if (!workspace || workspace_bytes < need.total)
    return fail(ICGS_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", workspace_bytes, need.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace ws = carve(static_cast<char*>(workspace), p, kNeedBackward);
  if (p.n == 0) {
    if (grad_targets)
      ICGS_TRY_CUDA(cudaMemsetAsync(grad_targets, 0, sizeof(float) * (size_t)p.n_cams * p.width * p.height * p.K, s));
    if (sync) ICGS_TRY_CUDA(cudaStreamSynchronize(s));
    return ICGS_OK;
  }
  if ((st = upload_common(p, cams, lam, ws, s)) != ICGS_OK) return st;
  ws.grad_o_acc = grad_opacity;
  if (grad_opacity) ICGS_TRY_CUDA(cudaMemsetAsync(grad_opacity, 0, sizeof(float) * (size_t)p.n, s));
  launch_adjoint_prepare(p, ws.lam, lam, coeffs, chol, grad_coeffs, ws, s);
  g_timer.mark(kSolve, s);
  for (int cam0 = 0; cam0 < p.n_cams; cam0 += p.cam_batch) {
    const int cb = std::min(p.cam_batch, p.n_cams - cam0);
    Workspace wp = ws;
    wp.cams = ws.cams + cam0;
    if ((st = bin_pass(p, scene, cb, cam0 == 0, wp, s)) != ICGS_OK) return st;
    launch_payload_adjoint(p, scene->means, coeffs, cb, wp, s);
    g_timer.mark(kPayload, s);
    launch_blend_adjoint(p, cb, cam0, targets->data, (int)targets->dtype, wp, grad_targets, grad_opacity != nullptr, s);
    g_timer.mark(kBlend, s);
  }
  return finish(ws, s, sync);
}

size_t icgs_refine_workspace_size(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                                  const icgs_options* opt) {
  if (!targets || !opt) return 0;
  Problem p;
  if (setup(scene, cams, targets->channels, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau, opt->cam_batch,
            opt->instance_capacity, p) != ICGS_OK)
    return 0;
  return carve(nullptr, p, kNeedRefine).total;
}

static icgs_status refine_impl(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                               const icgs_options* opt, int32_t n_steps, const float* chol, void* workspace,
                               size_t workspace_bytes, float* coeffs_inout, void* stream, bool sync) {
  TimerPause pause(!sync);
  g_err[0] = '\0';
  if (!opt) return fail(ICGS_ERR_INVALID_ARG, "options must not be NULL");
  icgs_status st = check_targets(targets);
  if (st != ICGS_OK) return st;
  Problem p;
  st = setup(scene, cams, targets->channels, opt->sh_degree, opt->precision, opt->cond_tau, opt->refold_tau, opt->cam_batch,
             opt->instance_capacity, p);
  if (st != ICGS_OK) return st;
  if (n_steps < 0) return fail(ICGS_ERR_INVALID_ARG, "n_steps = %d must be >= 0", n_steps);
  if (p.B * p.K > kMaxPayloadRow)
    return fail(ICGS_ERR_UNSUPPORTED, "(L+1)^2 x channels = %d exceeds %d for the render", p.B * p.K, kMaxPayloadRow);
  if ((!chol || !coeffs_inout) && p.n > 0) return fail(ICGS_ERR_INVALID_ARG, "chol and coeffs_inout are required");
  float lam[kMaxSH];
  if ((st = lambda_of(opt, p.L, lam)) != ICGS_OK) return st;
  const Workspace need = carve(nullptr, p, kNeedRefine);
  if (!workspace || workspace_bytes < need.total)
    return fail(ICGS_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", workspace_bytes, need.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Workspace ws = carve(static_cast<char*>(workspace), p, kNeedRefine);
  if (p.n == 0 || n_steps == 0) return ICGS_OK;
  if ((st = upload_common(p, cams, lam, ws, s)) != ICGS_OK) return st;
  const bool one_pass = p.cam_batch >= p.n_cams;  // the binning of one pass is reused across steps
  for (int step = 0; step < n_steps; ++step) {
    if (p.L == 0) ICGS_TRY_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(float) * (size_t)p.n * p.acc_stride, s));
    for (int cam0 = 0; cam0 < p.n_cams; cam0 += p.cam_batch) {
      const int cb = std::min(p.cam_batch, p.n_cams - cam0);
      Workspace wp = ws;
      wp.cams = ws.cams + cam0;
      if (p.L > 0)
        ICGS_TRY_CUDA(cudaMemsetAsync(ws.acc, 0, sizeof(float) * (size_t)cb * (size_t)p.n * p.acc_stride, s));
      if (!(one_pass && step > 0))
        if ((st = bin_pass(p, scene, cb, step == 0 && cam0 == 0, wp, s)) != ICGS_OK) return st;
      launch_payload_render(p, scene->means, coeffs_inout, cb, wp, s);  // Alg. 1 line 8: render
      if (launch_blend_refine(p, cb, cam0, targets->data, (int)targets->dtype, wp, s)) {  // lines 8-9, one walk
        g_timer.mark(kPayload, s);
      } else {
        launch_blend_render(p, cb, 0, wp, ws.img, s);
        g_timer.mark(kPayload, s);
        launch_blend_accumulate(p, cb, cam0, targets->data, (int)targets->dtype, ws.img, wp, s);  // line 9
      }
      g_timer.mark(kBlend, s);
      if (p.L > 0) {
        launch_fold(p, scene->means, cb, cam0 == 0, false, wp, s);
        g_timer.mark(kFold, s);
      }
    }
    launch_refine_update(p, ws.lam, lam, chol, ws, coeffs_inout, s);  // line 10
    g_timer.mark(kSolve, s);
  }
  return finish(ws, s, sync);
}

size_t icgs_render_workspace_size(const icgs_scene* scene, const icgs_cameras* cams, int32_t sh_degree,
                                  int32_t channels, int64_t instance_capacity) {
  Problem p;
  if (setup(scene, cams, channels, sh_degree, ICGS_PRECISION_PLAIN, 0.0f, 0.0f, 0, instance_capacity, p) != ICGS_OK) return 0;
  return carve(nullptr, p, kNeedRender).total;
}

static icgs_status render_impl(const icgs_scene* scene, const icgs_cameras* cams, int32_t sh_degree,
                               int32_t channels, const float* coeffs, int64_t instance_capacity, void* workspace,
                               size_t workspace_bytes, float* images_out, void* stream, bool sync) {
  TimerPause pause(!sync);
  g_err[0] = '\0';
  Problem p;
  icgs_status st = setup(scene, cams, channels, sh_degree, ICGS_PRECISION_PLAIN, 0.0f, 0.0f, 0, instance_capacity, p);
  if (st != ICGS_OK) return st;
  if (!images_out || (!coeffs && p.n > 0)) return fail(ICGS_ERR_INVALID_ARG, "coeffs and images_out are required");
  if (p.B * p.K > kMaxPayloadRow)
    return fail(ICGS_ERR_UNSUPPORTED, "(L+1)^2 x channels = %d exceeds %d for the render", p.B * p.K, kMaxPayloadRow);
  const Workspace need = carve(nullptr, p, kNeedRender);
  if (!workspace || workspace_bytes < need.total)
    return fail(ICGS_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", workspace_bytes, need.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Workspace ws = carve(static_cast<char*>(workspace), p, kNeedRender);
  if (p.n == 0) {
    ICGS_TRY_CUDA(cudaMemsetAsync(images_out, 0, sizeof(float) * (size_t)p.n_cams * p.width * p.height * p.K, s));
    if (sync) ICGS_TRY_CUDA(cudaStreamSynchronize(s));
    return ICGS_OK;
  }
  if ((st = upload_common(p, cams, nullptr, ws, s)) != ICGS_OK) return st;
  for (int cam0 = 0; cam0 < p.n_cams; cam0 += p.cam_batch) {
    const int cb = std::min(p.cam_batch, p.n_cams - cam0);
    Workspace wp = ws;
    wp.cams = ws.cams + cam0;
    if ((st = bin_pass(p, scene, cb, cam0 == 0, wp, s)) != ICGS_OK) return st;
    launch_payload_render(p, scene->means, coeffs, cb, wp, s);
    g_timer.mark(kPayload, s);
    launch_blend_render(p, cb, cam0, wp, images_out, s);
    g_timer.mark(kBlend, s);
  }
  return finish(ws, s, sync);
}

icgs_status icgs_colorize(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                          const icgs_options* opt, void* workspace, size_t workspace_bytes, float* coeffs_out,
                          uint8_t* status_out, float* chol_out, void* stream) {
  return colorize_impl(scene, cams, targets, opt, workspace, workspace_bytes, coeffs_out, status_out, chol_out, stream,
                       true);
}

icgs_status icgs_colorize_async(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                                const icgs_options* opt, void* workspace, size_t workspace_bytes, float* coeffs_out,
                                uint8_t* status_out, float* chol_out, void* stream) {
  return colorize_impl(scene, cams, targets, opt, workspace, workspace_bytes, coeffs_out, status_out, chol_out, stream,
                       false);
}

icgs_status icgs_colorize_backward(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                                   const icgs_options* opt, const float* coeffs, const float* chol,
                                   const float* grad_coeffs, void* workspace, size_t workspace_bytes,
                                   float* grad_targets, float* grad_opacity, void* stream) {
  return backward_impl(scene, cams, targets, opt, coeffs, chol, grad_coeffs, workspace, workspace_bytes, grad_targets,
                       grad_opacity, stream, true);
}

icgs_status icgs_colorize_backward_async(const icgs_scene* scene, const icgs_cameras* cams,
                                         const icgs_targets* targets, const icgs_options* opt, const float* coeffs,
                                         const float* chol, const float* grad_coeffs, void* workspace,
                                         size_t workspace_bytes, float* grad_targets, float* grad_opacity,
                                         void* stream) {
  return backward_impl(scene, cams, targets, opt, coeffs, chol, grad_coeffs, workspace, workspace_bytes, grad_targets,
                       grad_opacity, stream, false);
}

icgs_status icgs_colorize_refine(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                                 const icgs_options* opt, int32_t n_steps, const float* chol, void* workspace,
                                 size_t workspace_bytes, float* coeffs_inout, void* stream) {
  return refine_impl(scene, cams, targets, opt, n_steps, chol, workspace, workspace_bytes, coeffs_inout, stream, true);
}

icgs_status icgs_colorize_refine_async(const icgs_scene* scene, const icgs_cameras* cams,
                                       const icgs_targets* targets, const icgs_options* opt, int32_t n_steps,
                                       const float* chol, void* workspace, size_t workspace_bytes,
                                       float* coeffs_inout, void* stream) {
  return refine_impl(scene, cams, targets, opt, n_steps, chol, workspace, workspace_bytes, coeffs_inout, stream, false);
}

icgs_status icgs_render(const icgs_scene* scene, const icgs_cameras* cams, int32_t sh_degree, int32_t channels,
                        const float* coeffs, int64_t instance_capacity, void* workspace, size_t workspace_bytes,
                        float* images_out, void* stream) {
  return render_impl(scene, cams, sh_degree, channels, coeffs, instance_capacity, workspace, workspace_bytes,
                     images_out, stream, true);
}

icgs_status icgs_render_async(const icgs_scene* scene, const icgs_cameras* cams, int32_t sh_degree,
                              int32_t channels, const float* coeffs, int64_t instance_capacity, void* workspace,
                              size_t workspace_bytes, float* images_out, void* stream) {
  return render_impl(scene, cams, sh_degree, channels, coeffs, instance_capacity, workspace, workspace_bytes,
                     images_out, stream, false);
}

icgs_status icgs_async_status(const void* workspace, void* stream) {
  g_err[0] = '\0';
  if (!workspace) return fail(ICGS_ERR_INVALID_ARG, "workspace must not be NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevStatus st;
  ICGS_TRY_CUDA(cudaMemcpyAsync(&st, workspace, sizeof st, cudaMemcpyDeviceToHost, s));
  ICGS_TRY_CUDA(cudaStreamSynchronize(s));
  g_launches = 0;
  return status_of(st);
}

icgs_status icgs_selftest_tc_rows(const void* A, int32_t M, const void* B, int32_t N, int32_t bf16, float* D,
                                  float* D_lanes, void* workspace, void* stream) {
  g_err[0] = '\0';
  if (!A || !B || !D || !workspace) return fail(ICGS_ERR_INVALID_ARG, "A, B, D and workspace are required");
  if (M != 64 && M != 128) return fail(ICGS_ERR_INVALID_ARG, "M = %d must be 64 or 128", M);
  if (N != 32 && N != 80) return fail(ICGS_ERR_INVALID_ARG, "N = %d must be 32 or 80", N);
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace ws;
  ws.status = static_cast<DevStatus*>(workspace);
  ICGS_TRY_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(DevStatus), s));
  ICGS_TRY_CUDA(launch_tc_selftest(static_cast<const uint16_t*>(A), M, static_cast<const uint16_t*>(B), N, bf16 != 0, D,
                                   D_lanes, ws.status, s));
  return finish(ws, s);
}

void icgs_debug_tc_wait(int64_t limit_ns, int32_t issue_mma) { set_tc_wait_diagnostic(limit_ns, issue_mma != 0); }

size_t icgs_sort_workspace_size(int32_t ntiles, int64_t nkeys) {
  if (ntiles < 0 || nkeys < 0) return 0;
  return align256(sizeof(DevStatus)) + align256(sizeof(uint32_t) * (size_t)ntiles) +
         align256(sizeof(uint64_t) * (size_t)nkeys);
}

icgs_status icgs_sort_tile_lists(const uint32_t* tile_off, uint64_t* keys, int32_t ntiles, int64_t nkeys,
                                 void* workspace, size_t workspace_bytes, void* stream) {
  g_err[0] = '\0';
  if (ntiles < 0 || nkeys < 0) return fail(ICGS_ERR_INVALID_ARG, "ntiles = %d and nkeys = %lld must be >= 0", ntiles, (long long)nkeys);
  if (nkeys > (int64_t)kMaxCapacity) return fail(ICGS_ERR_INVALID_ARG, "nkeys = %lld exceeds %u", (long long)nkeys, kMaxCapacity);
  if (!tile_off || !workspace || (nkeys > 0 && !keys)) return fail(ICGS_ERR_INVALID_ARG, "tile_off, keys and workspace are required");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(ICGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  const size_t need = icgs_sort_workspace_size(ntiles, nkeys);
  if (workspace_bytes < need)
    return fail(ICGS_ERR_WORKSPACE_TOO_SMALL, "workspace holds %zu bytes, the sort needs %zu", workspace_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(workspace);
  Workspace ws;
  ws.status = reinterpret_cast<DevStatus*>(base);
  ws.big_list = reinterpret_cast<uint32_t*>(base + align256(sizeof(DevStatus)));
  ws.entries_tmp = reinterpret_cast<uint64_t*>(base + align256(sizeof(DevStatus)) + align256(sizeof(uint32_t) * (size_t)ntiles));
  ws.tile_off = const_cast<uint32_t*>(tile_off);
  ws.entries = keys;
  Problem p;
  p.tiles = ntiles;
  p.capacity = (uint32_t)nkeys;
  ICGS_TRY_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(DevStatus), s));
  g_launches = 0;
  if (ntiles > 0) launch_tile_sort(p, 1, ws, s);
  return finish(ws, s);
}

icgs_status icgs_selftest_tc(const void* A, const void* B, int32_t N, int32_t bf16, float* D, void* workspace,
                             void* stream) {
  return icgs_selftest_tc_rows(A, 128, B, N, bf16, D, nullptr, workspace, stream);
}

const char* icgs_last_error(void) { return g_err; }

int64_t icgs_last_required_instances(void) { return g_required; }

void icgs_last_stats(int64_t out[4]) {
  if (!out) return;
  for (int k = 0; k < 5; ++k) out[k] = g_stats[k];
}

void icgs_set_stage_timing(int enable) { g_timer.on = enable != 0; }

int icgs_last_stage_ms(double* out, int n) {
  for (int k = 0; k < n && k < kStageCount; ++k) out[k] = g_timer.ms[k];
  return kStageCount;
}

const char* icgs_stage_name(int i) { return (i >= 0 && i < kStageCount) ? kStageNames[i] : ""; }

}  // extern "C"
