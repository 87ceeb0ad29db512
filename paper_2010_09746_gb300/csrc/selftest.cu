// Self-test of the bounded-wait path that every kernel of the library uses for its mbarrier
// waits: a kernel waits on an mbarrier that nothing ever arrives on, gives up after a short
// %globaltimer limit and reports QS_ETIMEOUT through a device status word.  Nothing faults
// and nothing hangs; the CUDA context stays usable.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qs_internal.h"

namespace qs {
namespace {

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void k_wait_selftest(unsigned long long limit_ns, int* status) {
  __shared__ alignas(8) uint64_t bar;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(1u) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const unsigned long long deadline = globaltimer() + limit_ns;
  uint32_t done = 0, spins = 0;
  for (;;) {   // the phase never completes: only the deadline ends the loop
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(b), "r"(0u)
        : "memory");
    if (done) break;
    if ((++spins & 255u) == 0 && globaltimer() > deadline) break;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *status = done ? (int)QS_OK : (int)QS_ETIMEOUT;
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
  }
}

}  // namespace
}  // namespace qs

extern "C" qs_status qs_selftest_bounded_wait(int limit_us, int* device_status) {
  if (limit_us < 1 || limit_us > 1000000 || !device_status) {
    qs::set_last_error("limit_us must be in [1, 1000000] and device_status non-null");
    return QS_EINVAL;
  }
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0xFF, sizeof(int));
  if (e == cudaSuccess) {
    qs::k_wait_selftest<<<1, 32>>>((unsigned long long)limit_us * 1000ull, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(device_status, d, sizeof(int), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) {
    qs::set_last_error(std::string("bounded-wait self-test: ") + cudaGetErrorString(e));
    return QS_ECUDA;
  }
  return QS_OK;
}
