// noalloc.cu -- icgs_colorize_noalloc: colorize using scratch memory that is built into the
// library, for callers that cannot allocate device memory themselves.
//
// Who needs this: code that runs where no device allocation is possible or allowed -- a plugin
// loaded into a host application that owns every byte of device memory through its own
// allocator, or a latency-critical loop whose rules forbid allocating (or failing to allocate)
// after start-up. Such a caller cannot provide the workspace icgs_colorize asks for, so this
// entry point takes the workspace from a fixed array that exists on every GPU that loads the
// library, for as long as the process lives.
//
// Limits: the array holds kScratchBytes (64 MiB); problems whose workspace does not fit are
// rejected with ICGS_ERR_WORKSPACE_TOO_SMALL (too many Gaussians x cameras) or ICGS_ERR_CAPACITY
// (too many Gaussian-tile instances for what is left). All calls on a device share the one
// array: calls that overlap on the GPU (on different streams, or from different host threads)
// overwrite each other's scratch and must not be issued. Each call clears what has to start at
// zero; the array otherwise keeps the contents of the last call.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/icgs.h"
#include "icgs_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

// The scratch itself. Host code must not pass this symbol to a kernel: on the host it only names
// a stand-in, and the device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, resolved on the first call per device
// (that first call should therefore come before any stream capture).
icgs_status scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    icgs::set_error_message("cudaGetDevice: %s", cudaGetErrorString(e));
    return ICGS_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    icgs::set_error_message("device ordinal %d beyond the %d devices icgs_colorize_noalloc supports", dev, kMaxDevices);
    return ICGS_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      icgs::set_error_message("cudaGetSymbolAddress of the built-in scratch failed on device %d: %s", dev,
                              cudaGetErrorString(e));
      return ICGS_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return ICGS_OK;
}

}  // namespace

extern "C" {

size_t icgs_noalloc_scratch_bytes(void) { return kScratchBytes; }

icgs_status icgs_colorize_noalloc(const icgs_scene* scene, const icgs_cameras* cams, const icgs_targets* targets,
                                  const icgs_options* opt, float* coeffs_out, uint8_t* status_out,
                                  float* chol_out, void* stream) {
  if (!opt) {
    icgs::set_error_message("options must not be NULL");
    return ICGS_ERR_INVALID_ARG;
  }
  void* scratch = nullptr;
  icgs_status st = scratch_address(&scratch);
  if (st != ICGS_OK) return st;
  icgs_options o = *opt;
  if (o.instance_capacity <= 0) {
    // give the (Gaussian, tile) instance buffers whatever colorize's fixed regions leave free
    o.instance_capacity = 1;
    const size_t fixed = icgs::colorize_workspace_bytes(scene, cams, targets, &o);
    if (fixed == 0) return icgs_colorize(scene, cams, targets, &o, scratch, kScratchBytes, coeffs_out, status_out,
                                         chol_out, stream);  // invalid arguments: let colorize report them
    if (fixed + 2 * 256 + 16 > kScratchBytes) {
      icgs::set_error_message("icgs_colorize_noalloc: this problem needs more than the %zu bytes of built-in "
                              "scratch before any instance buffer (%zu bytes); use icgs_colorize with a "
                              "caller workspace", kScratchBytes, fixed);
      return ICGS_ERR_WORKSPACE_TOO_SMALL;
    }
    o.instance_capacity = (int64_t)((kScratchBytes - fixed - 2 * 256) / (2 * sizeof(uint64_t)));
  }
  st = icgs_colorize(scene, cams, targets, &o, scratch, kScratchBytes, coeffs_out, status_out, chol_out, stream);
  if (st == ICGS_ERR_CAPACITY)
    icgs::set_error_message("icgs_colorize_noalloc: the scene needs %lld (Gaussian, tile) instances in one pass, "
                            "more than the %lld that fit in the %zu bytes of built-in scratch; lower "
                            "cam_batch or use icgs_colorize with a caller workspace",
                            (long long)icgs_last_required_instances(), (long long)o.instance_capacity,
                            kScratchBytes);
  else if (st == ICGS_ERR_WORKSPACE_TOO_SMALL)
    icgs::set_error_message("icgs_colorize_noalloc: the problem does not fit in the %zu bytes of built-in "
                            "scratch; use icgs_colorize with a caller workspace", kScratchBytes);
  return st;
}

}  // extern "C"
