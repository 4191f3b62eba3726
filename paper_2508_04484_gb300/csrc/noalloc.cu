// dlra_kstep_noalloc: the stand-alone streaming K-step for callers that cannot
// allocate device memory. Some callers run where cudaMalloc is unavailable or
// forbidden: inside a memory pool they do not own, in code paths that must not
// synchronise the device (cudaMalloc/cudaFree can), or in embedded runtimes that
// hand out only pre-registered buffers. They pass inputs and outputs; the work
// space lives in a fixed static device array instead.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/dlra.h"
#include "kernels.h"

namespace {

// Work space shared by every call on a device: three n x rcap FP32 stage buffers,
// the packed P stack and the rank word. 32 MiB, held by every GPU that loads the
// library until the process exits.
constexpr size_t kNoAllocBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

namespace dlra {
void set_context_free_error(const char* msg);
int check_kstep_args(const dlra_kstep_args* a, char* msg, int msg_len);
}  // namespace dlra

extern "C" dlra_status dlra_kstep_noalloc(const dlra_kstep_args* args) {
  char msg[256];
  if (!args) {
    dlra::set_context_free_error("dlra_kstep_noalloc: null arguments");
    return DLRA_ERR_ARG;
  }
  const bool two_d = args->ny == 1 && args->dy == 0.0;
  if (dlra::check_kstep_args(args, msg, sizeof msg) != DLRA_OK) {
    dlra::set_context_free_error(msg);
    return DLRA_ERR_ARG;
  }
  const long long n = (long long)args->nx * args->ny * args->nz;
  const size_t need = dlra::kstep_scratch_bytes(n, args->r, two_d ? 2 : 3, args->stage_kernel);
  if (need == 0 || need > kNoAllocBytes) {
    std::snprintf(msg, sizeof msg,
                  "dlra_kstep_noalloc: n = %lld cells at r = %d need %zu bytes of work space; the static work space "
                  "holds %zu bytes",
                  n, args->r, need, kNoAllocBytes);
    dlra::set_context_free_error(msg);
    return DLRA_ERR_ARG;
  }
  // one-time set-up per device, with that device current: the device address of the
  // static array (its name in host code is only a host-side stand-in)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    dlra::set_context_free_error("dlra_kstep_noalloc: no current CUDA device");
    return DLRA_ERR_CUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        std::snprintf(msg, sizeof msg, "dlra_kstep_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        dlra::set_context_free_error(msg);
        return DLRA_ERR_CUDA;
      }
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  int s = dlra::run_kstep(args, base, kNoAllocBytes, msg, sizeof msg);
  if (s != DLRA_OK) dlra::set_context_free_error(msg);
  return (dlra_status)s;
}
