// Allocation-free variant of the LSC forward (declaration and contract in
// include/delimit.h, delimit_lsc_forward_noalloc).
//
// Some callers cannot allocate device memory at the point where they run the
// layer: code that runs inside a region where the CUDA allocator must not be
// touched (a host callback, a stream being captured by another component, an
// allocator-owning host framework that forbids side allocations), or
// deployments with a fixed, pre-budgeted memory footprint.  For them the
// forward's scratch (the collapsed operator W, its transpose and the bias
// vector) lives in the fixed-size device array below, which exists on every
// GPU that loads this library until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/delimit.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB

// The scratch itself.  Host code must not use this name as a device address:
// the device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_lsc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[128] = {nullptr};

}  // namespace

extern "C" {

delimit_status delimit_lsc_forward_noalloc(const delimit_lsc_geometry* geom, const void* sh_in, const float* w,
                                           const float* b, void* sh_out, int64_t n_vox, int c_in, int c_out,
                                           int64_t ld_in, int64_t ld_out, delimit_dtype act_t, void* stream) {
  const size_t need = delimit_lsc_workspace_size(geom, n_vox, c_in, c_out, act_t, 0);
  if (need == 0) return delimit_lsc_forward(geom, sh_in, w, b, sh_out, n_vox, c_in, c_out, ld_in, ld_out, act_t, 0u,
                                            nullptr, 0, stream);  // reports the argument error
  if (need > kScratchBytes) {
    delimit::set_last_error("delimit_lsc_forward_noalloc: these sizes need " + std::to_string(need) +
                            " bytes of scratch, more than the fixed 16 MiB (16777216 bytes)");
    return DELIMIT_ERR_WORKSPACE;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    delimit::set_last_error("delimit_lsc_forward_noalloc: no current CUDA device");
    return DELIMIT_ERR_CUDA;
  }
  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      // first call on this device (the current one): resolve the array's device address
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_lsc_scratch);
      if (e != cudaSuccess || p == nullptr) {
        delimit::set_last_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        return DELIMIT_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    ptr = g_scratch_addr[dev];
  }
  return delimit_lsc_forward(geom, sh_in, w, b, sh_out, n_vox, c_in, c_out, ld_in, ld_out, act_t, 0u, ptr,
                             kScratchBytes, stream);
}

}  // extern "C"
