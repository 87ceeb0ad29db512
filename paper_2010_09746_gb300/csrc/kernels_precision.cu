// Precision helpers around the gate path: FP64 inner product of two states (possibly of
// different storage types) and in-place renormalisation by a norm that is already on the
// device.  Both are plain streaming kernels: HBM-bound for complex64, FP64-pipe-bound for
// complex128 (the reductions stay in FP64 whatever the storage type).
#include "qs_internal.h"

namespace qs {
namespace {

constexpr int kThreads = 256;
// Determinism contract of the inner product: always this many partial sums, added in
// index order, so the result does not depend on the GPU's SM count.
constexpr int kInnerBlocks = 1216;

template <class S>
__device__ __forceinline__ double2 load_d(const S* p, uint64_t i) {
  S v = p[i];
  return make_double2((double)v.x, (double)v.y);
}

// <a|b> = sum_i conj(a_i) b_i: a fixed grid, each thread a fixed strided subset, a fixed
// shared-memory tree per block; the final kernel sums the partials in index order.
template <class SA, class SB>
__global__ void __launch_bounds__(kThreads) k_inner_partials(const SA* __restrict__ a, const SB* __restrict__ b,
                                                             uint64_t N, double2* partials) {
  __shared__ double rr[kThreads], ri[kThreads];
  double re = 0.0, im = 0.0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    double2 x = load_d(a, i), y = load_d(b, i);
    re = fma(x.x, y.x, re);
    re = fma(x.y, y.y, re);
    im = fma(x.x, y.y, im);
    im = fma(-x.y, y.x, im);
  }
  rr[threadIdx.x] = re;
  ri[threadIdx.x] = im;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rr[threadIdx.x] += rr[threadIdx.x + w];
      ri[threadIdx.x] += ri[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(rr[0], ri[0]);
}

__global__ void k_inner_final(const double2* partials, int nparts, double2* out) {
  __shared__ double rr[kThreads], ri[kThreads];
  double re = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    re += partials[i].x;
    im += partials[i].y;
  }
  rr[threadIdx.x] = re;
  ri[threadIdx.x] = im;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rr[threadIdx.x] += rr[threadIdx.x + w];
      ri[threadIdx.x] += ri[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = make_double2(rr[0], ri[0]);
}

// psi *= 1 / sqrt(*norm).  complex128 scales each component in FP64 (one rounding);
// complex64 scales in FP32 by the factor rounded once to float.  A norm that is not a
// positive finite number leaves the state unchanged.
__global__ void __launch_bounds__(kThreads) k_scale16(double2* psi, uint64_t N, const double* norm) {
  const double v = *norm;
  if (!(v > 0.0) || !(v < INFINITY)) return;
  const double s = 1.0 / sqrt(v);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    double2 x = psi[i];
    psi[i] = make_double2(x.x * s, x.y * s);
  }
}

// complex64: two amplitudes (16 B) per thread per step.
__global__ void __launch_bounds__(kThreads) k_scale8(float4* psi2, uint64_t N2, float2* tail, int has_tail,
                                                     const double* norm) {
  const double v = *norm;
  if (!(v > 0.0) || !(v < INFINITY)) return;
  const float s = (float)(1.0 / sqrt(v));
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N2; i += (uint64_t)gridDim.x * blockDim.x) {
    float4 x = psi2[i];
    psi2[i] = make_float4(x.x * s, x.y * s, x.z * s, x.w * s);
  }
  if (has_tail && blockIdx.x == 0 && threadIdx.x == 0) {
    float2 x = *tail;
    *tail = make_float2(x.x * s, x.y * s);
  }
}

unsigned grid_stream(uint64_t items) {
  const uint64_t per = (uint64_t)kThreads * 4;
  uint64_t g = (items + per - 1) / per;
  int sms = 0, dev = 0;   // the current device's SM count (the runtime answers from a cache)
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0) {
    cudaGetLastError();
    sms = 1;   // grid-stride loops stay correct with any grid
  }
  const uint64_t cap = (uint64_t)sms * 8 * 4;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

int inner_num_partials() { return kInnerBlocks; }

cudaError_t launch_inner(const void* a, int a_c128, const void* b, int b_c128, int n, double* partials2,
                         double* out2, cudaStream_t s) {
  const uint64_t N = 1ull << n;
  double2* p = (double2*)partials2;
  if (a_c128 && b_c128)
    k_inner_partials<double2, double2><<<kInnerBlocks, kThreads, 0, s>>>((const double2*)a, (const double2*)b, N, p);
  else if (a_c128)
    k_inner_partials<double2, float2><<<kInnerBlocks, kThreads, 0, s>>>((const double2*)a, (const float2*)b, N, p);
  else if (b_c128)
    k_inner_partials<float2, double2><<<kInnerBlocks, kThreads, 0, s>>>((const float2*)a, (const double2*)b, N, p);
  else
    k_inner_partials<float2, float2><<<kInnerBlocks, kThreads, 0, s>>>((const float2*)a, (const float2*)b, N, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_inner_final<<<1, kThreads, 0, s>>>(p, kInnerBlocks, (double2*)out2);
  return cudaGetLastError();
}

cudaError_t launch_scale(void* psi, int n, int is_c128, const double* norm_dev, cudaStream_t s) {
  const uint64_t N = 1ull << n;
  if (is_c128) {
    k_scale16<<<grid_stream(N), kThreads, 0, s>>>((double2*)psi, N, norm_dev);
  } else {
    const uint64_t N2 = N / 2;
    float2* tail = (float2*)psi + 2 * N2;
    k_scale8<<<grid_stream(N2 ? N2 : 1), kThreads, 0, s>>>((float4*)psi, N2, tail, (int)(N & 1), norm_dev);
  }
  return cudaGetLastError();
}

}  // namespace qs
