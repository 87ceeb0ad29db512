// Per-gate strided-pair kernels (K1), state initialisation, norm / probability read-outs.
//
// A gate on storage bit p updates the amplitude pairs (j, j + 2^p) with bit p of j clear
// (Sec. 2: gates are linear updates of amplitude pairs; controlled gates restrict the pairs
// to those whose control bits are 1).  Work item t enumerates the untouched bits: the
// storage index is t with zero bits inserted at the gate's target positions and one bits
// at its control positions, so a controlled gate launches only over its 2^(n-1-#controls)
// pairs and reads/writes only those bytes.  Consecutive threads take consecutive t, i.e.
// consecutive storage indices for every target bit above the lowest ones: each warp moves
// whole 128-byte lines (16-byte complex128 / 8-byte complex64 elements).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "arith.cuh"
#include "qs_internal.h"

namespace qs {

namespace {

constexpr int kThreads = 256;

struct Expand {
  int nz;            // number of inserted bit positions (sorted ascending)
  int pos[8];
  uint64_t ones;     // bits forced to one after insertion (controls)
};

__device__ __forceinline__ uint64_t expand(uint64_t t, const Expand& e) {
#pragma unroll 8
  for (int k = 0; k < 8; k++) {
    if (k < e.nz) {
      const int p = e.pos[k];
      t = ((t >> p) << (p + 1)) | (t & ((1ull << p) - 1));
    }
  }
  return t | e.ones;
}

int grid_for(uint64_t work) {
  int sms = 0, dev = 0;   // the current device's SM count (the runtime answers from a cache)
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0) {
    cudaGetLastError();
    sms = 1;   // grid-stride loops stay correct with any grid
  }
  uint64_t blocks = (work + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_u1(typename A::store_t* __restrict__ psi, uint64_t nwork,
                                                 Expand e, int p, const typename A::mat_t* __restrict__ m) {
  using R = typename A::reg_t;
  const typename A::mat_t u00 = m[0], u01 = m[1], u10 = m[2], u11 = m[3];
  const uint64_t s = 1ull << p;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = expand(t, e);
    R a = A::from_store(psi[i0]);
    R b = A::from_store(psi[i0 | s]);
    psi[i0] = A::to_store(A::mac2(u00, a, u01, b));
    psi[i0 | s] = A::to_store(A::mac2(u10, a, u11, b));
  }
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_rx(typename A::store_t* __restrict__ psi, uint64_t nwork,
                                                 Expand e, int p, const typename A::mat_t* __restrict__ m) {
  using R = typename A::reg_t;
  const typename A::mat_t cs = m[0];
  const uint64_t s = 1ull << p;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = expand(t, e);
    R a = A::from_store(psi[i0]);
    R b = A::from_store(psi[i0 | s]);
    psi[i0] = A::to_store(A::rx(cs, a, b));
    psi[i0 | s] = A::to_store(A::rx(cs, b, a));
  }
}

// diag(d0, d1) on bit p, amplitudes with the control bits set
template <class A>
__global__ void __launch_bounds__(kThreads) k_diag(typename A::store_t* __restrict__ psi, uint64_t nwork,
                                                   Expand e, int p, const typename A::mat_t* __restrict__ m) {
  const typename A::mat_t d0 = m[0], d1 = m[1];
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = expand(t, e);
    psi[i] = A::to_store(A::mul(((i >> p) & 1) ? d1 : d0, A::from_store(psi[i])));
  }
}

// multiply by d0 on the amplitudes whose fixed bits (the inserted positions) are all one
template <class A>
__global__ void __launch_bounds__(kThreads) k_phase(typename A::store_t* __restrict__ psi, uint64_t nwork,
                                                    Expand e, const typename A::mat_t* __restrict__ m) {
  const typename A::mat_t d = m[0];
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = expand(t, e);
    psi[i] = A::to_store(A::mul(d, A::from_store(psi[i])));
  }
}

// exact sign flip (CZ / Z): no arithmetic, bit-exact
template <class S>
__global__ void __launch_bounds__(kThreads) k_negate(S* __restrict__ psi, uint64_t nwork, Expand e) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = expand(t, e);
    S v = psi[i];
    v.x = -v.x;
    v.y = -v.y;
    psi[i] = v;
  }
}

// exchange psi[i0 | s0] and psi[i0 | s1] (X / CNOT with s0 = 0, SWAP with s0 = 2^k0, s1 = 2^k1)
template <class S>
__global__ void __launch_bounds__(kThreads) k_exchange(S* __restrict__ psi, uint64_t nwork, Expand e,
                                                       uint64_t s0, uint64_t s1) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = expand(t, e);
    S a = psi[i | s0], b = psi[i | s1];
    psi[i | s0] = b;
    psi[i | s1] = a;
  }
}

// complex64 with 16-byte accesses: every load and store moves two adjacent amplitudes (a
// float4).  Work item t expands to an index i0 with bit 0 clear.  A 2x2 (or RX) on bit 0
// finds its pair inside one word; on a bit p >= 1 the words at i0 and i0 + 2^p hold two
// pairs.  Controls never include bit 0 here (the launcher falls back otherwise).
template <bool kRX>
__global__ void __launch_bounds__(kThreads) k_pair_c64x2(float2* __restrict__ psi, uint64_t nwork, Expand e, int p,
                                                          const float2* __restrict__ m) {
  using A = AF32;
  const float2 u00 = m[0], u01 = kRX ? m[0] : m[1], u10 = kRX ? m[0] : m[2], u11 = kRX ? m[0] : m[3];
  float4* psi4 = reinterpret_cast<float4*>(psi);
  const uint64_t s = 1ull << p;
  auto upd = [&](float2 a, float2 b, float2& ra, float2& rb) {
    if (kRX) {
      ra = A::rx(u00, a, b);
      rb = A::rx(u00, b, a);
    } else {
      ra = A::mac2(u00, a, u01, b);
      rb = A::mac2(u10, a, u11, b);
    }
  };
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = expand(t, e);
    float2 r0, r1;
    if (p == 0) {
      const float4 v = psi4[i0 >> 1];
      upd(make_float2(v.x, v.y), make_float2(v.z, v.w), r0, r1);
      psi4[i0 >> 1] = make_float4(r0.x, r0.y, r1.x, r1.y);
    } else {
      const float4 va = psi4[i0 >> 1], vb = psi4[(i0 | s) >> 1];
      float2 r2, r3;
      upd(make_float2(va.x, va.y), make_float2(vb.x, vb.y), r0, r1);
      upd(make_float2(va.z, va.w), make_float2(vb.z, vb.w), r2, r3);
      psi4[i0 >> 1] = make_float4(r0.x, r0.y, r2.x, r2.y);
      psi4[(i0 | s) >> 1] = make_float4(r1.x, r1.y, r3.x, r3.y);
    }
  }
}

// complex64 diagonal factors on two adjacent amplitudes per 16-byte word (bit 0 not a
// control): kind 0 = diag(d0, d1) on bit p, 1 = multiply by d0, 2 = exact sign flip
template <int kKind>
__global__ void __launch_bounds__(kThreads) k_diag_c64x2(float2* __restrict__ psi, uint64_t nwork, Expand e, int p,
                                                          const float2* __restrict__ m) {
  using A = AF32;
  float4* psi4 = reinterpret_cast<float4*>(psi);
  const float2 d0 = kKind == 2 ? make_float2(0.f, 0.f) : m[0];
  const float2 d1 = kKind == 0 ? m[1] : d0;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = expand(t, e);
    float4 v = psi4[i >> 1];
    if (kKind == 2) {
      v = make_float4(-v.x, -v.y, -v.z, -v.w);
    } else {
      float2 f0 = d0, f1 = d0;
      if (kKind == 0) {
        if (p == 0) f1 = d1;
        else f0 = f1 = ((i >> p) & 1) ? d1 : d0;
      }
      const float2 a = A::mul(f0, make_float2(v.x, v.y)), b = A::mul(f1, make_float2(v.z, v.w));
      v = make_float4(a.x, a.y, b.x, b.y);
    }
    psi4[i >> 1] = v;
  }
}

// dense 2^K x 2^K on bits kq[0..K-1]: a block stages kThreads / 2^K groups of 2^K
// amplitudes in shared memory; thread (g, r) computes output row r of group g.
template <class A, int K>
__global__ void __launch_bounds__(kThreads) k_dense(typename A::store_t* __restrict__ psi, uint64_t nwork,
                                                    Expand e, DevOp op, const typename A::mat_t* __restrict__ m) {
  using R = typename A::reg_t;
  constexpr int D = 1 << K;
  constexpr int G = kThreads / D;
  __shared__ R buf[kThreads];
  const int r = threadIdx.x % D, gl = threadIdx.x / D;
  uint64_t off = 0;
#pragma unroll
  for (int b = 0; b < K; b++)
    if ((r >> b) & 1) off |= 1ull << op.kq[b];
  // all threads run the same number of iterations (uniform __syncthreads)
  const uint64_t ngroups_iter = (nwork + G - 1) / G;
  for (uint64_t it = blockIdx.x; it < ngroups_iter; it += gridDim.x) {
    const uint64_t t = it * G + gl;
    const bool live = t < nwork;
    const uint64_t i = live ? (expand(t, e) | off) : 0;
    if (live) buf[threadIdx.x] = A::from_store(psi[i]);
    __syncthreads();
    if (live) {
      R acc = A::zero();
      const R* x = buf + gl * D;
#pragma unroll 4
      for (int c = 0; c < D; c++) acc = A::mac(acc, m[r * D + c], x[c]);
      psi[i] = A::to_store(acc);
    }
    __syncthreads();
  }
}

// Build the enumeration for a gate: zero bits at `zero_bits`, one bits at controls.
Expand make_expand(int n, uint64_t zero_bits, uint64_t ones, uint64_t* nwork) {
  Expand e{};
  uint64_t fixed = zero_bits | ones;
  e.nz = 0;
  for (int b = 0; b < 64; b++)
    if ((fixed >> b) & 1) e.pos[e.nz++] = b;
  e.ones = ones;
  *nwork = 1ull << (n - e.nz);
  return e;
}

// complex64 gates that the 16-byte kernels cover; false = use the general kernels
bool launch_gate_c64x2(float2* psi, int n, const DevOp& op, const float2* mp, cudaStream_t st) {
  if (n < 2 || (op.cmask & 1ull) || __builtin_popcountll(op.cmask) > 6) return false;
  uint64_t nwork = 0;
  switch (op.type) {
    case OP_U1:
    case OP_RX: {
      const uint64_t zb = (op.k0 == 0) ? 1ull : ((1ull << op.k0) | 1ull);
      Expand e = make_expand(n, zb, op.cmask, &nwork);
      if (op.type == OP_U1) k_pair_c64x2<false><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, op.k0, mp);
      else k_pair_c64x2<true><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, op.k0, mp);
      return true;
    }
    case OP_DIAG: {
      Expand e = make_expand(n, 1ull, op.cmask, &nwork);
      k_diag_c64x2<0><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, op.k0, mp);
      return true;
    }
    case OP_PHASE: {
      Expand e = make_expand(n, 1ull, op.cmask, &nwork);
      if (op.mat < 0) k_diag_c64x2<2><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, 0, mp);
      else k_diag_c64x2<1><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, 0, mp);
      return true;
    }
    default:
      return false;
  }
}

template <class A>
cudaError_t launch_gate_t(void* psi_v, int n, const DevOp& op, const void* pool, cudaStream_t st) {
  using S = typename A::store_t;
  using M = typename A::mat_t;
  S* psi = (S*)psi_v;
  const M* mp = (const M*)pool + op.mat;
  uint64_t nwork = 0;
  if constexpr (std::is_same<A, AF32>::value) {   // complex64: 16-byte accesses where possible
    if (launch_gate_c64x2(psi, n, op, mp, st)) return cudaGetLastError();
  }
  switch (op.type) {
    case OP_U1: {
      Expand e = make_expand(n, 1ull << op.k0, op.cmask, &nwork);
      k_u1<A><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, op.k0, mp);
      break;
    }
    case OP_RX: {
      Expand e = make_expand(n, 1ull << op.k0, op.cmask, &nwork);
      k_rx<A><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, op.k0, mp);
      break;
    }
    case OP_DIAG: {
      Expand e = make_expand(n, 0, op.cmask, &nwork);
      k_diag<A><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, op.k0, mp);
      break;
    }
    case OP_PHASE: {
      if (op.mat < 0) {   // exact -1
        Expand e = make_expand(n, 0, op.cmask, &nwork);
        k_negate<S><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e);
      } else {
        Expand e = make_expand(n, 0, op.cmask, &nwork);
        k_phase<A><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, mp);
      }
      break;
    }
    case OP_X: {
      Expand e = make_expand(n, 1ull << op.k0, op.cmask, &nwork);
      k_exchange<S><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, 0ull, 1ull << op.k0);
      break;
    }
    case OP_SWAP: {
      Expand e = make_expand(n, (1ull << op.k0) | (1ull << op.k1), op.cmask, &nwork);
      k_exchange<S><<<grid_for(nwork), kThreads, 0, st>>>(psi, nwork, e, 1ull << op.k0, 1ull << op.k1);
      break;
    }
    case OP_U2:
    case OP_DENSE: {
      DevOp o = op;
      if (op.type == OP_U2) {
        o.nk = 2;
        o.kq[0] = op.k0;
        o.kq[1] = op.k1;
      }
      uint64_t zb = 0;
      for (int t = 0; t < o.nk; t++) zb |= 1ull << o.kq[t];
      Expand e = make_expand(n, zb, op.cmask, &nwork);
      const int g = grid_for(nwork << o.nk);
      switch (o.nk) {
        case 1: k_dense<A, 1><<<g, kThreads, 0, st>>>(psi, nwork, e, o, mp); break;
        case 2: k_dense<A, 2><<<g, kThreads, 0, st>>>(psi, nwork, e, o, mp); break;
        case 3: k_dense<A, 3><<<g, kThreads, 0, st>>>(psi, nwork, e, o, mp); break;
        case 4: k_dense<A, 4><<<g, kThreads, 0, st>>>(psi, nwork, e, o, mp); break;
        case 5: k_dense<A, 5><<<g, kThreads, 0, st>>>(psi, nwork, e, o, mp); break;
        case 6: k_dense<A, 6><<<g, kThreads, 0, st>>>(psi, nwork, e, o, mp); break;
        default: return cudaErrorInvalidValue;
      }
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
__global__ void k_init_zero16(double2* psi, uint64_t N) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
    psi[i] = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
}
__global__ void k_init_zero8(float2* psi, uint64_t N) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
    psi[i] = make_float2(i == 0 ? 1.0f : 0.0f, 0.0f);
}

// ---------------------------------------------------------------------------------------
// Norm: every thread of a fixed grid accumulates a fixed strided subset in FP64, a fixed
// shared-memory tree reduces the block, and a single block sums the per-block partials in
// index order: the result does not depend on timing.
// Determinism contract of every FP64 norm: the sum is always split into this many
// partial sums (block b adds the grid-stride elements b, b + 1216 * threads, ...) and the
// partials are added in index order, whatever GPU runs it, so a norm is the same bits on any
// device and in every entry point that shares this reduction.  (1216 fills a 152-SM GB300
// with 8 blocks per SM; on other SM counts it is still correct, only the balance differs.)
constexpr int kNormBlocks = 1216;

template <class S>
__global__ void __launch_bounds__(kThreads) k_norm_partials(const S* __restrict__ psi, uint64_t N, double* partials) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    S v = psi[i];
    double re = (double)v.x, im = (double)v.y;
    acc = fma(re, re, acc);
    acc = fma(im, im, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_norm_final(const double* partials, int nparts, double* out) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// ---------------------------------------------------------------------------------------
// Logical-order read-outs: output index i -> storage index j(i, sigma), through byte
// tables T_b[v] = sum over bits k of v of 2^{sigma(8b + k)} held in shared memory.
struct SigmaArg {
  int n;
  int sigma[kMaxQubits];
};

__device__ __forceinline__ void build_tables(uint64_t* tab, const SigmaArg& sa) {
  const int nbytes = (sa.n + 7) / 8;
  for (int e = threadIdx.x; e < nbytes * 256; e += blockDim.x) {
    const int b = e >> 8, v = e & 255;
    uint64_t o = 0;
    for (int k = 0; k < 8; k++) {
      const int q = 8 * b + k;
      if (q < sa.n && ((v >> k) & 1)) o |= 1ull << sa.sigma[q];
    }
    tab[e] = o;
  }
  __syncthreads();
}
__device__ __forceinline__ uint64_t map_index(uint64_t i, const uint64_t* tab, int nbytes) {
  uint64_t j = 0;
  for (int b = 0; b < nbytes; b++) j |= tab[(b << 8) | ((i >> (8 * b)) & 255)];
  return j;
}

template <class S>
__global__ void __launch_bounds__(kThreads) k_probs(const S* __restrict__ psi, uint64_t N, double* out,
                                                    SigmaArg sa, int logical) {
  __shared__ uint64_t tab[5 * 256];
  const int nbytes = (sa.n + 7) / 8;
  if (logical) build_tables(tab, sa);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = logical ? map_index(i, tab, nbytes) : i;
    S v = psi[j];
    double re = (double)v.x, im = (double)v.y;
    out[i] = re * re + im * im;
  }
}

template <class S>
__global__ void __launch_bounds__(kThreads) k_gather(const S* __restrict__ psi, uint64_t first, uint64_t count,
                                                     S* out, SigmaArg sa, int logical) {
  __shared__ uint64_t tab[5 * 256];
  const int nbytes = (sa.n + 7) / 8;
  if (logical) build_tables(tab, sa);
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = first + k;
    out[k] = psi[logical ? map_index(i, tab, nbytes) : i];
  }
}

// ---------------------------------------------------------------------------------------
// Batches: amplitude 0 of every state set to 1 after the buffer was cleared; per-state FP64
// norms, one CTA per state with a fixed reduction order.
template <class S>
__global__ void k_batch_ones(S* psi, const uint64_t* offs, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    S v;
    v.x = 1;
    v.y = 0;
    psi[offs[i]] = v;
  }
}

template <class S>
__global__ void __launch_bounds__(kThreads) k_batch_norms(const S* __restrict__ psi, const uint64_t* offs,
                                                          const int* ns, double* out) {
  __shared__ double red[kThreads];
  const S* p = psi + offs[blockIdx.x];
  const uint64_t N = 1ull << ns[blockIdx.x];
  double acc = 0.0;
  for (uint64_t i = threadIdx.x; i < N; i += kThreads) {
    const double re = (double)p[i].x, im = (double)p[i].y;
    acc = fma(re, re, acc);
    acc = fma(im, im, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

}  // namespace

cudaError_t launch_batch_init(void* psi, int store_bytes, const uint64_t* offs, int count, size_t total_elems,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(psi, 0, total_elems * store_bytes, s);
  if (e != cudaSuccess) return e;
  const int blocks = (count + kThreads - 1) / kThreads;
  if (store_bytes == 16)
    k_batch_ones<double2><<<blocks, kThreads, 0, s>>>((double2*)psi, offs, count);
  else
    k_batch_ones<float2><<<blocks, kThreads, 0, s>>>((float2*)psi, offs, count);
  return cudaGetLastError();
}

cudaError_t launch_batch_norms(const void* psi, int is_c128, const uint64_t* offs, const int* ns, int count,
                               double* out, cudaStream_t s) {
  if (is_c128)
    k_batch_norms<double2><<<count, kThreads, 0, s>>>((const double2*)psi, offs, ns, out);
  else
    k_batch_norms<float2><<<count, kThreads, 0, s>>>((const float2*)psi, offs, ns, out);
  return cudaGetLastError();
}

cudaError_t launch_gate(Policy pol, void* psi, int n, const DevOp& op, const void* pool, cudaStream_t s) {
  switch (pol) {
    case POL_F32: return launch_gate_t<AF32>(psi, n, op, pool, s);
    case POL_F64: return launch_gate_t<AF64>(psi, n, op, pool, s);
    case POL_DF: return launch_gate_t<ADF>(psi, n, op, pool, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_init_zero(void* psi, int n, int store_bytes, cudaStream_t s) {
  const uint64_t N = 1ull << n;
  if (store_bytes == 16)
    k_init_zero16<<<grid_for(N), kThreads, 0, s>>>((double2*)psi, N);
  else
    k_init_zero8<<<grid_for(N), kThreads, 0, s>>>((float2*)psi, N);
  return cudaGetLastError();
}

int norm_num_partials() { return kNormBlocks; }

cudaError_t launch_norm_partials(const void* psi, int n, int is_c128, double* partials, int nparts,
                                 cudaStream_t s) {
  const uint64_t N = 1ull << n;
  if (nparts != kNormBlocks) return cudaErrorInvalidValue;
  if (is_c128)
    k_norm_partials<double2><<<kNormBlocks, kThreads, 0, s>>>((const double2*)psi, N, partials);
  else
    k_norm_partials<float2><<<kNormBlocks, kThreads, 0, s>>>((const float2*)psi, N, partials);
  return cudaGetLastError();
}

cudaError_t launch_norm_final(const double* partials, int nparts, double* out, cudaStream_t s) {
  k_norm_final<<<1, kThreads, 0, s>>>(partials, nparts, out);
  return cudaGetLastError();
}

cudaError_t launch_probabilities(const void* psi, int n, int is_c128, double* out, const int* sigma,
                                 int logical, cudaStream_t s) {
  const uint64_t N = 1ull << n;
  SigmaArg sa{};
  sa.n = n;
  for (int q = 0; q < n; q++) sa.sigma[q] = sigma[q];
  if (is_c128)
    k_probs<double2><<<grid_for(N), kThreads, 0, s>>>((const double2*)psi, N, out, sa, logical);
  else
    k_probs<float2><<<grid_for(N), kThreads, 0, s>>>((const float2*)psi, N, out, sa, logical);
  return cudaGetLastError();
}

cudaError_t launch_gather_amplitudes(const void* psi, int n, int store_bytes, void* out, uint64_t first,
                                     uint64_t count, const int* sigma, int logical, cudaStream_t s) {
  SigmaArg sa{};
  sa.n = n;
  for (int q = 0; q < n; q++) sa.sigma[q] = sigma[q];
  if (store_bytes == 16)
    k_gather<double2><<<grid_for(count), kThreads, 0, s>>>((const double2*)psi, first, count, (double2*)out, sa, logical);
  else
    k_gather<float2><<<grid_for(count), kThreads, 0, s>>>((const float2*)psi, first, count, (float2*)out, sa, logical);
  return cudaGetLastError();
}

}  // namespace qs
