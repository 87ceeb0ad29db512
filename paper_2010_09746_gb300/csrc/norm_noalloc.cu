// Allocation-free norm: the FP64 norm read-out with its partial sums in a fixed device
// array instead of memory obtained from an allocator.
//
// The array lives in this file at namespace scope, so every GPU that loads the library
// holds it (kNoAllocParts doubles) until the process exits.  Host code cannot use the
// array's name as a device address; the address is looked up with cudaGetSymbolAddress once
// per device and context (the device current at the time) and cached under that context, so
// that a new context on the device (after cudaDeviceReset, say), whose copy of the module
// sits elsewhere, gets its own lookup instead of a stale address.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "qs_internal.h"

namespace qs {

namespace {

constexpr int kNoAllocParts = 1216;   // one partial sum per block of the fixed reduction grid
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_norm_scratch[kNoAllocParts];

// cached address per device, valid for the context it was looked up in
struct AddrCache {
  void* ctx = nullptr;
  void* addr = nullptr;
};
std::mutex g_addr_mu;
AddrCache g_addr[kMaxDevices];

// the calling thread's current driver context (entry point fetched through the runtime, so
// the library needs no link against the driver library)
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
void* current_context() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return (CtxGetCurrentFn)f;
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return (void*)c;
}

qs_status fail(qs_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" qs_status qs_norm_noalloc(const void* psi, int n, qs_dtype dtype, double* out_dev, void* stream) {
  if (!psi || !out_dev) return fail(QS_EINVAL, "qs_norm_noalloc: null state or output pointer");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "qs_norm_noalloc: unknown dtype");
  if (n < 1 || n > kMaxQubits)
    return fail(QS_EINVAL, "qs_norm_noalloc: n = " + std::to_string(n) +
                               " is outside 1..36 (the maximum is 2^36 amplitudes)");
  if (norm_num_partials() > kNoAllocParts)
    return fail(QS_EUNSUPPORTED, "qs_norm_noalloc: reduction grid larger than the fixed scratch array");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(QS_ECUDA, std::string("qs_norm_noalloc: no usable current device: ") + cudaGetErrorString(e));
  void* scratch = nullptr;
  {
    // NULL before the runtime has made a context current on this thread (first use)
    void* ctx = current_context();
    std::lock_guard<std::mutex> lk(g_addr_mu);
    AddrCache& c = g_addr[dev];
    if (ctx && c.addr && c.ctx == ctx) {
      scratch = c.addr;
    } else {   // first call in this context (or no context handle: look up every call)
      e = cudaGetSymbolAddress(&scratch, g_norm_scratch);
      if (e != cudaSuccess || !scratch)
        return fail(QS_ECUDA, std::string("qs_norm_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      if (ctx) {
        c.ctx = ctx;
        c.addr = scratch;
      }
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  // every partial is overwritten by its block, so nothing needs clearing between calls
  e = launch_norm_partials(psi, n, dtype == QS_C128, (double*)scratch, norm_num_partials(), s);
  if (e == cudaSuccess) e = launch_norm_final((const double*)scratch, norm_num_partials(), out_dev, s);
  if (e != cudaSuccess) return fail(QS_ECUDA, std::string("qs_norm_noalloc: launch failed: ") + cudaGetErrorString(e));
  return QS_OK;
}
