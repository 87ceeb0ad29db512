// Tile pass (K2): one HBM read and one HBM write of the whole state apply a fused list
// of gates.
//
// The paper makes gates on "local" qubits cheap and moves qubits between local and global
// positions with PermuteQubits (Sec. 2-3).  Here the local set of a pass is a set T of L
// storage bits: a CTA owns the 2^L amplitudes that share one value of the other n - L bits
// (the block id b, deposited into those bit positions), stages them in shared memory,
// applies every gate of the pass whose non-diagonal qubits lie in T, and writes them back.
// Diagonal factors and controls on bits outside T are constants of the block (a predicate
// or a scalar).  T always contains the `c` lowest storage bits, so the tile is 2^(L-c)
// contiguous segments of 2^c amplitudes; each segment is moved by one TMA bulk copy
// (cp.async.bulk, completion counted on an mbarrier for loads, bulk groups for stores).
// Choosing T per pass is the multi-qubit PermuteQubits folded into the addressing: no
// separate permutation pass is needed to make a qubit "local".
//
// Persistent grid: CTAs stride over the 2^(n-L) blocks; several CTAs per SM overlap one
// tile's copies with another tile's arithmetic.  Every mbarrier wait is bounded by a
// %globaltimer deadline; on expiry the whole CTA (a block-wide vote) records QS_ETIMEOUT in
// *status and returns.  A pass that timed out leaves the state undefined.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

#include "arith.cuh"
#include "qs_internal.h"

namespace qs {

namespace {

constexpr int kTileThreads = 256;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: true when the phase completed, false when the deadline passed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long deadline) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 255u) == 0 && globaltimer() > deadline) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_load(uint32_t dst_smem, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst_smem),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, uint32_t src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src_smem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// insert zero bits at the sorted positions pos[0..nz-1], then OR `ones`
__device__ __forceinline__ uint32_t texpand(uint32_t t, const int* pos, int nz, uint32_t ones) {
  for (int k = 0; k < nz; k++) {
    const int p = pos[k];
    t = ((t >> p) << (p + 1)) | (t & ((1u << p) - 1u));
  }
  return t | ones;
}
// sorted list of set bits of m (tile-local masks, < 2^14)
__device__ __forceinline__ int bit_list(uint32_t m, int* pos) {
  int k = 0;
  while (m) {
    const int b = __ffs(m) - 1;
    pos[k++] = b;
    m &= m - 1;
  }
  return k;
}

// Shared-memory tile addressing: element i sits at i + (i >> c) * padE, i.e. every 2^c-element
// segment is followed by 16 bytes of padding, which spreads the register-stage accesses of a
// warp over the banks.
struct Pad {
  int c, padE;
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return i + (i >> c) * padE; }
};

// Dense 2^k x 2^k block in shared memory (kept out of line: its per-thread arrays would
// otherwise give every tile kernel a large stack frame).
template <class A>
__device__ __noinline__ void apply_dense_op(typename A::reg_t* Tm, int L, const DevOp& op,
                                            const typename A::mat_t* __restrict__ pool, Pad px) {
  using R = typename A::reg_t;
  using M = typename A::mat_t;
  const int tid = threadIdx.x;
  const uint32_t cm = (uint32_t)op.cmask;
  int pos[8];
  const int K = op.nk;
  const int D = 1 << K;
  uint32_t zb = cm;
  for (int b = 0; b < K; b++) zb |= 1u << op.kq[b];
  const int nz = bit_list(zb, pos);
  const uint32_t nw = 1u << (L - nz);
  const M* m = pool + op.mat;
  for (uint32_t t = tid; t < nw; t += kTileThreads) {
    const uint32_t i = texpand(t, pos, nz, cm);
    R x[1 << kMaxDenseK];
    uint32_t off[1 << kMaxDenseK];
    for (int r = 0; r < D; r++) {
      uint32_t o = 0;
      for (int b = 0; b < K; b++)
        if ((r >> b) & 1) o |= 1u << op.kq[b];
      off[r] = px(i | o);
      x[r] = Tm[off[r]];
    }
    for (int r = 0; r < D; r++) {
      R acc = A::zero();
      for (int c = 0; c < D; c++) acc = A::mac(acc, A::ld(m + r * D + c), x[c]);
      Tm[off[r]] = acc;
    }
  }
}

// Apply one tile op to the shared-memory tile (2^L elements in policy register format).
template <class A>
__device__ __forceinline__ void apply_op(typename A::reg_t* Tm, int L, const DevOp& op,
                                         const typename A::mat_t* __restrict__ pool, uint64_t base, Pad px) {
  using R = typename A::reg_t;
  using M = typename A::mat_t;
  struct TV {
    R* t;
    Pad px;
    __device__ __forceinline__ R& operator[](uint32_t i) const { return t[px(i)]; }
  } T{Tm, px};
  const int tid = threadIdx.x;
  const uint32_t cm = (uint32_t)op.cmask;
  int pos[8];
  switch (op.type) {
    case OP_U1:
    case OP_RX: {
      const int nz = bit_list(cm | (1u << op.k0), pos);
      const uint32_t nw = 1u << (L - nz);
      const uint32_t s = 1u << op.k0;
      if (op.type == OP_U1) {
        const M* u = pool + op.mat;
        for (uint32_t t = tid; t < nw; t += kTileThreads) {
          const uint32_t i = texpand(t, pos, nz, cm);
          const R a = T[i], b = T[i | s];
          T[i] = A::mac2(A::ld(u), a, A::ld(u + 1), b);
          T[i | s] = A::mac2(A::ld(u + 2), a, A::ld(u + 3), b);
        }
      } else if constexpr (A::kFrame) {
        const auto c = A::ld_real(pool + op.mat), sn = A::ld_real(pool + op.mat + 1);   // (c, 0), (s, 0)
        for (uint32_t t = tid; t < nw; t += kTileThreads) {
          const uint32_t i = texpand(t, pos, nz, cm);
          R a2, b2;
          A::rot_r(c, sn, T[i], T[i | s], a2, b2);
          T[i] = a2;
          T[i | s] = b2;
        }
      } else {
        const M cs = pool[op.mat];
        for (uint32_t t = tid; t < nw; t += kTileThreads) {
          const uint32_t i = texpand(t, pos, nz, cm);
          const R a = T[i], b = T[i | s];
          T[i] = A::rx(cs, a, b);
          T[i | s] = A::rx(cs, b, a);
        }
      }
      break;
    }
    case OP_DIAG: {
      const int nz = bit_list(cm, pos);
      const uint32_t nw = 1u << (L - nz);
      const M d0 = pool[op.mat], d1 = pool[op.mat + 1];
      if (op.k0 >= 0) {
        for (uint32_t t = tid; t < nw; t += kTileThreads) {
          const uint32_t i = texpand(t, pos, nz, cm);
          T[i] = A::mul(((i >> op.k0) & 1u) ? d1 : d0, T[i]);
        }
      } else {
        const M d = ((base >> op.gbit) & 1ull) ? d1 : d0;
        for (uint32_t t = tid; t < nw; t += kTileThreads) {
          const uint32_t i = texpand(t, pos, nz, cm);
          T[i] = A::mul(d, T[i]);
        }
      }
      break;
    }
    case OP_PHASE: {
      const int nz = bit_list(cm, pos);
      const uint32_t nw = 1u << (L - nz);
      if (op.mat < 0) {
        for (uint32_t t = tid; t < nw; t += kTileThreads) {
          const uint32_t i = texpand(t, pos, nz, cm);
          T[i] = A::neg(T[i]);
        }
      } else {
        const M d = pool[op.mat];
        for (uint32_t t = tid; t < nw; t += kTileThreads) {
          const uint32_t i = texpand(t, pos, nz, cm);
          T[i] = A::mul(d, T[i]);
        }
      }
      break;
    }
    case OP_X:
    case OP_SWAP: {
      uint32_t s0, s1, zb;
      if (op.type == OP_X) {
        s0 = 0;
        s1 = 1u << op.k0;
        zb = s1;
      } else {
        s0 = 1u << op.k0;
        s1 = 1u << op.k1;
        zb = s0 | s1;
      }
      const int nz = bit_list(cm | zb, pos);
      const uint32_t nw = 1u << (L - nz);
      // in the phase frame X is [[0, i], [-i, 0]]; SWAP exchanges equal popcounts
      const bool framed_x = A::kFrame && op.type == OP_X;
      for (uint32_t t = tid; t < nw; t += kTileThreads) {
        const uint32_t i = texpand(t, pos, nz, cm);
        const R a = T[i | s0], b = T[i | s1];
        if constexpr (A::kFrame) {
          T[i | s0] = framed_x ? A::rot_q(b, 3u) : b;
          T[i | s1] = framed_x ? A::rot_q(a, 1u) : a;
        } else {
          T[i | s0] = b;
          T[i | s1] = a;
        }
      }
      break;
    }
    case OP_U2: {
      const uint32_t s0 = 1u << op.k0, s1 = 1u << op.k1;
      const int nz = bit_list(cm | s0 | s1, pos);
      const uint32_t nw = 1u << (L - nz);
      const M* m = pool + op.mat;
      for (uint32_t t = tid; t < nw; t += kTileThreads) {
        const uint32_t i = texpand(t, pos, nz, cm);
        const uint32_t idx[4] = {i, i | s0, i | s1, i | s0 | s1};
        R x[4];
#pragma unroll
        for (int r = 0; r < 4; r++) x[r] = T[idx[r]];
#pragma unroll
        for (int r = 0; r < 4; r++) {
          R acc = A::mac2(A::ld(m + 4 * r + 0), x[0], A::ld(m + 4 * r + 1), x[1]);
          acc = A::mac(acc, A::ld(m + 4 * r + 2), x[2]);
          acc = A::mac(acc, A::ld(m + 4 * r + 3), x[3]);
          T[idx[r]] = acc;
        }
      }
      break;
    }
    case OP_DENSE:
      apply_dense_op<A>(Tm, L, op, pool, px);
      break;
    default:
      break;
  }
}

// ------------------------------------------------------------------------------------------
// Register stages
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pdep32(uint32_t g, uint32_t mask) {
  uint32_t r = 0;
  for (uint32_t m = mask; m; m &= m - 1u) {
    if (g & 1u) r |= m & (0u - m);
    g >>= 1;
  }
  return r;
}

// single-slot updates carry no register-slot controls (the compiler turns a controlled
// update into a 4x4 block on the (target, control) slots); X keeps its predicate
template <class A, int K, int S>
__device__ __forceinline__ void r_u1(typename A::reg_t (&x)[1 << K], const typename A::mat_t* m, uint32_t csl) {
#pragma unroll
  for (int j = 0; j < (1 << K); j++) {
    if (j & (1 << S)) continue;
    const typename A::reg_t a = x[j], b = x[j | (1 << S)];
    x[j] = A::mac2(A::ld(m + 0), a, A::ld(m + 1), b);
    x[j | (1 << S)] = A::mac2(A::ld(m + 2), a, A::ld(m + 3), b);
  }
}
template <class A, int K, int S>
__device__ __forceinline__ void r_rx(typename A::reg_t (&x)[1 << K], const typename A::mat_t* m, uint32_t csl) {
  if constexpr (A::kFrame) {   // real rotation, entries (c, 0) and (s, 0)
    const auto c = A::ld_real(m), sn = A::ld_real(m + 1);
#pragma unroll
    for (int j = 0; j < (1 << K); j++) {
      if (j & (1 << S)) continue;
      A::rot_r(c, sn, x[j], x[j | (1 << S)], x[j], x[j | (1 << S)]);
    }
  } else {
    const typename A::mat_t cs = m[0];
#pragma unroll
    for (int j = 0; j < (1 << K); j++) {
      if (j & (1 << S)) continue;
      const typename A::reg_t a = x[j], b = x[j | (1 << S)];
      x[j] = A::rx(cs, a, b);
      x[j | (1 << S)] = A::rx(cs, b, a);
    }
  }
}
// phase frame (double-float policy): tangent-form RX mode 0 is [[1, t], [-t, 1]], mode 1 is
// [[t, 1], [-1, t]], both real
template <class A, int K, int S, class T>
__device__ __forceinline__ void r_rxt_frame(typename A::reg_t (&x)[1 << K], const T& t, uint32_t mode) {
  if (mode == 0) {
#pragma unroll
    for (int j = 0; j < (1 << K); j++) {
      if (j & (1 << S)) continue;
      const typename A::reg_t a = x[j], b = x[j | (1 << S)];
      x[j] = A::axpy_r(t, b, a);
      x[j | (1 << S)] = A::axmy_r(t, a, b);
    }
  } else {
#pragma unroll
    for (int j = 0; j < (1 << K); j++) {
      if (j & (1 << S)) continue;
      const typename A::reg_t a = x[j], b = x[j | (1 << S)];
      x[j] = A::axpy_r(t, a, b);
      x[j | (1 << S)] = A::ymx_r(t, b, a);
    }
  }
}
// tangent-form RX on slot S: mode 0 applies I - i t X, mode 1 applies t I - i X (the
// compiler moves the dropped factor cos or sin into one full-form RX of the same pass)
template <class A, int K, int S>
__device__ __forceinline__ void r_rxt(typename A::reg_t (&x)[1 << K], const typename A::mat_t* m, uint32_t mode) {
  if constexpr (A::kFrame) {
    r_rxt_frame<A, K, S>(x, A::ld_real(m), mode);
  } else {
    const typename A::mat_t t = m[0];
    if (mode == 0) {
#pragma unroll
      for (int j = 0; j < (1 << K); j++) {
        if (j & (1 << S)) continue;
        const typename A::reg_t a = x[j], b = x[j | (1 << S)];
        x[j] = A::axpy(t, A::mul_mi(b), a);
        x[j | (1 << S)] = A::axpy(t, A::mul_mi(a), b);
      }
    } else {
#pragma unroll
      for (int j = 0; j < (1 << K); j++) {
        if (j & (1 << S)) continue;
        const typename A::reg_t a = x[j], b = x[j | (1 << S)];
        x[j] = A::axpy(t, a, A::mul_mi(b));
        x[j | (1 << S)] = A::axpy(t, b, A::mul_mi(a));
      }
    }
  }
}
// several tangent-form RX on distinct slots (slot mask sm, form bits fm), one decode
template <class A, int K>
__device__ __forceinline__ void r_rxt_multi(typename A::reg_t (&x)[1 << K], const typename A::mat_t* m, uint32_t sm,
                                            uint32_t fm) {
  int idx = 0;
  if constexpr (K > 0) if (sm & 1u) { r_rxt<A, K, 0>(x, m + idx, fm & 1u); idx++; }
  if constexpr (K > 1) if (sm & 2u) { r_rxt<A, K, (K > 1 ? 1 : 0)>(x, m + idx, (fm >> 1) & 1u); idx++; }
  if constexpr (K > 2) if (sm & 4u) { r_rxt<A, K, (K > 2 ? 2 : 0)>(x, m + idx, (fm >> 2) & 1u); idx++; }
  if constexpr (K > 3) if (sm & 8u) { r_rxt<A, K, (K > 3 ? 3 : 0)>(x, m + idx, (fm >> 3) & 1u); idx++; }
  if constexpr (K > 4) if (sm & 16u) { r_rxt<A, K, (K > 4 ? 4 : 0)>(x, m + idx, (fm >> 4) & 1u); idx++; }
  (void)idx;
}
template <class A, int K, int S>
__device__ __forceinline__ void r_x(typename A::reg_t (&x)[1 << K], const typename A::mat_t*, uint32_t csl) {
#pragma unroll
  for (int j = 0; j < (1 << K); j++) {
    if (j & (1 << S)) continue;
    if ((j & csl) != csl) continue;
    const typename A::reg_t a = x[j];
    if constexpr (A::kFrame) {   // [[0, i], [-i, 0]] in the phase frame
      x[j] = A::rot_q(x[j | (1 << S)], 3u);
      x[j | (1 << S)] = A::rot_q(a, 1u);
    } else {
      x[j] = x[j | (1 << S)];
      x[j | (1 << S)] = a;
    }
  }
}


template <class A, int K, int S0, int S1>
__device__ __forceinline__ void r_u2(typename A::reg_t (&x)[1 << K], const typename A::mat_t* m, uint32_t csl) {
  using R = typename A::reg_t;
#pragma unroll
  for (int j = 0; j < (1 << K); j++) {
    if (j & ((1 << S0) | (1 << S1))) continue;
    if (csl && (j & csl) != csl) continue;
    const int i0 = j, i1 = j | (1 << S0), i2 = j | (1 << S1), i3 = j | (1 << S0) | (1 << S1);
    const R x0 = x[i0], x1 = x[i1], x2 = x[i2], x3 = x[i3];
    R y[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      R acc = A::mac2(A::ld(m + 4 * r + 0), x0, A::ld(m + 4 * r + 1), x1);
      acc = A::mac(acc, A::ld(m + 4 * r + 2), x2);
      y[r] = A::mac(acc, A::ld(m + 4 * r + 3), x3);
    }
    x[i0] = y[0];
    x[i1] = y[1];
    x[i2] = y[2];
    x[i3] = y[3];
  }
}

// slot dispatch (the pair structure of the register array must be known at compile time)
#define QS_SLOT_DISPATCH(FN, s, ...)                                  \
  do {                                                                \
    if constexpr (K > 0) if ((s) == 0) { FN<A, K, 0>(__VA_ARGS__); break; } \
    if constexpr (K > 1) if ((s) == 1) { FN<A, K, 1>(__VA_ARGS__); break; } \
    if constexpr (K > 2) if ((s) == 2) { FN<A, K, 2>(__VA_ARGS__); break; } \
    if constexpr (K > 3) if ((s) == 3) { FN<A, K, 3>(__VA_ARGS__); break; } \
    if constexpr (K > 4) if ((s) == 4) { FN<A, K, 4>(__VA_ARGS__); break; } \
  } while (0)

template <class A, int K, int S0>
__device__ __forceinline__ void r_u2_s1(typename A::reg_t (&x)[1 << K], int s1, const typename A::mat_t* m,
                                        uint32_t csl) {
  if constexpr (K > 0 && S0 != 0) if (s1 == 0) { r_u2<A, K, S0, 0>(x, m, csl); return; }
  if constexpr (K > 1 && S0 != 1) if (s1 == 1) { r_u2<A, K, S0, (K > 1 ? 1 : 0)>(x, m, csl); return; }
  if constexpr (K > 2 && S0 != 2) if (s1 == 2) { r_u2<A, K, S0, (K > 2 ? 2 : 0)>(x, m, csl); return; }
  if constexpr (K > 3 && S0 != 3) if (s1 == 3) { r_u2<A, K, S0, (K > 3 ? 3 : 0)>(x, m, csl); return; }
  if constexpr (K > 4 && S0 != 4) if (s1 == 4) { r_u2<A, K, S0, (K > 4 ? 4 : 0)>(x, m, csl); return; }
}

// multiply register element j by table entry j where bit j of csl is set (the others are 1)
template <class A, int K>
__device__ __forceinline__ void r_dtab(typename A::reg_t (&x)[1 << K], const typename A::mat_t* m, uint32_t csl) {
  using M = typename A::mat_t;
  if constexpr (sizeof(M) == 8 && K >= 1) {
    // 8-byte entries: the compiler aligns every table to 16 bytes, load two at a time.
    // FP32 multiplies are cheaper than testing the mask (entries outside it are exactly
    // 1, so multiplying by them changes nothing)
    const float4* t4 = reinterpret_cast<const float4*>(m);
#pragma unroll
    for (int j = 0; j < (1 << K); j += 2) {
      const float4 v = t4[j >> 1];
      x[j] = A::mul(M{v.x, v.y}, x[j]);
      x[j + 1] = A::mul(M{v.z, v.w}, x[j + 1]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < (1 << K); j++)
      if ((csl >> j) & 1u) x[j] = A::mul(A::ld(m + j), x[j]);
  }
}

template <class A, int K>
__device__ __forceinline__ void apply_regop(typename A::reg_t (&x)[1 << K], const RegOp& op,
                                            const typename A::mat_t* __restrict__ pool, uint32_t gidx,
                                            uint64_t base) {
  using R = typename A::reg_t;
  using M = typename A::mat_t;
  if ((gidx & op.cot) != op.cot) return;   // a control outside the registers is 0 for this group
  const M* m = pool + op.mat;
  const uint32_t csl = op.csl;
  switch (op.type) {
    case OP_U1: QS_SLOT_DISPATCH(r_u1, op.s0, x, m, csl); break;
    case OP_RX: QS_SLOT_DISPATCH(r_rx, op.s0, x, m, csl); break;
    case OP_RXT: QS_SLOT_DISPATCH(r_rxt, op.s0, x, m, (uint32_t)op.s1); break;
    case OP_RXTM: r_rxt_multi<A, K>(x, m, csl, (uint32_t)(uint8_t)op.neg); break;
    case OP_X: QS_SLOT_DISPATCH(r_x, op.s0, x, m, csl); break;
    case OP_U2: {
      if constexpr (K >= 2) {
        const int s1 = op.s1;
        QS_SLOT_DISPATCH(r_u2_s1, op.s0, x, s1, m, csl);
      }
      break;
    }
    case OP_DIAG: {
      const M d0 = m[0], d1 = m[1];
      if (op.s0 >= 0) {
        const int s0 = op.s0;
#pragma unroll
        for (int j = 0; j < (1 << K); j++)
          if ((j & csl) == csl) x[j] = A::mul(((j >> s0) & 1) ? d1 : d0, x[j]);
      } else {
        const M d = (op.tb >= 0) ? (((gidx >> op.tb) & 1u) ? d1 : d0) : (((base >> op.gbit) & 1ull) ? d1 : d0);
        if (csl == 0) {
#pragma unroll
          for (int j = 0; j < (1 << K); j++) x[j] = A::mul(d, x[j]);
        } else {
#pragma unroll
          for (int j = 0; j < (1 << K); j++)
            if ((j & csl) == csl) x[j] = A::mul(d, x[j]);
        }
      }
      break;
    }
    case OP_DTAB: r_dtab<A, K>(x, m, csl); break;
    case OP_PHASE: {
      if (op.neg) {
#pragma unroll
        for (int j = 0; j < (1 << K); j++)
          if ((j & csl) == csl) x[j] = A::neg(x[j]);
      } else {
        const M d = m[0];
#pragma unroll
        for (int j = 0; j < (1 << K); j++)
          if ((j & csl) == csl) x[j] = A::mul(d, x[j]);
      }
      break;
    }
    default:
      break;
  }
  (void)sizeof(R);
}

// A register op is read by every thread of the CTA: two 16-byte read-only loads instead of
// one load per field.
__device__ __forceinline__ RegOp load_regop(const RegOp* p) {
  static_assert(sizeof(RegOp) == 32 && alignof(RegOp) <= 16, "RegOp is loaded as two 16-byte words");
  const uint4* q = reinterpret_cast<const uint4*>(p);
  const uint4 a = __ldg(q), b = __ldg(q + 1);
  RegOp r;
  uint4* w = reinterpret_cast<uint4*>(&r);
  w[0] = a;
  w[1] = b;
  return r;
}

// Phase frame of the double-float policy: while in register format, an element is held as
// (-i)^popcount(its storage address) times its value, i.e. tile element i of the block at
// `base` carries (-i)^(popcount(i) + popcount(base)).  Within a pass that is the tile frame times a
// factor common to the tile, which every op of the pass (all linear) carries along; and a
// permutation of address bits keeps every popcount, so the double-float storage form a plan
// keeps between its passes stays in this frame: only binary64 loads and stores rotate.
// wb = popcount(base) mod 4.
template <class A>
__device__ __forceinline__ typename A::reg_t load_framed(typename A::store_t v, uint32_t q, bool df) {
  if constexpr (A::kFrame) return df ? A::from_df(v) : A::rot_q(A::from_store(v), q & 3u);
  else return A::from_store_f(v, df);
}
template <class A>
__device__ __forceinline__ typename A::store_t store_framed(typename A::reg_t v, uint32_t q, bool df) {
  if constexpr (A::kFrame) return df ? A::to_df(v) : A::to_store(A::rot_q(v, (0u - q) & 3u));
  else return A::to_store_f(v, df);
}

// One register stage over the whole tile.  from_store / to_store: the shared-memory tile
// holds storage-format elements before / after the stage (policies whose register format
// differs from the storage format convert here instead of in a separate pass); df_in /
// df_out: that storage form is the double-float one a plan keeps between its passes.
template <class A, int K, bool Lite>
__device__ __forceinline__ void run_reg_stage(typename A::reg_t* T, const StageRec& sr, const RegOp* __restrict__ rops,
                                              const typename A::mat_t* __restrict__ pool, int L, Pad px,
                                              uint64_t base, bool from_store, bool to_store, bool df_in,
                                              bool df_out, uint32_t wb) {
  using R = typename A::reg_t;
  using S = typename A::store_t;
  const uint32_t tile_mask = (L >= 32) ? 0xFFFFFFFFu : ((1u << L) - 1u);
  const uint32_t omask = tile_mask & ~(uint32_t)sr.rmask;
  const uint32_t ngroups = 1u << (L - K);
  // px(a | b) = px(a) + px(b) for disjoint bit sets (no carries), so an element's padded
  // position is the group's position plus a sum of per-register-bit offsets
  uint32_t pb[K];
#pragma unroll
  for (int b = 0; b < K; b++) pb[b] = px(1u << sr.rbits[b]);
  // 8-byte elements with tile bit 0 in register slot 0: elements j and j + 1 are adjacent and
  // 16-byte aligned, so one 16-byte access moves both (half the instructions, and lanes that
  // differ in segment bits no longer share banks)
  constexpr bool kPairable = std::is_same<R, S>::value && sizeof(R) == 8 && K >= 1;
  const bool pair = kPairable && sr.rbits[0] == 0 && pb[0] == 1u;   // bit 0 inside the segments
  for (uint32_t g = threadIdx.x; g < ngroups; g += kTileThreads) {
    const uint32_t gidx = pdep32(g, omask);
    const uint32_t gpos = px(gidx);
    const uint32_t wg = __popc(gidx);   // phase frame: element j carries (-i)^(wg + popcount j)
    R x[1 << K];
    if constexpr (kPairable) {
      if (pair) {
#pragma unroll
        for (int j = 0; j < (1 << K); j += 2) {
          uint32_t p = gpos;
#pragma unroll
          for (int b = 1; b < K; b++)
            if ((j >> b) & 1) p += pb[b];
          const float4 v = *reinterpret_cast<const float4*>(&T[p]);
          x[j] = make_float2(v.x, v.y);
          x[j + 1] = make_float2(v.z, v.w);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < (1 << K); j++) {
      if constexpr (kPairable)
        if (pair) break;
      uint32_t p = gpos;
#pragma unroll
      for (int b = 0; b < K; b++)
        if ((j >> b) & 1) p += pb[b];
      if constexpr (std::is_same<R, S>::value) {
        x[j] = T[p];
      } else if constexpr (A::kFrame) {
        x[j] = from_store ? load_framed<A>(reinterpret_cast<const S*>(T)[p], wb + wg + __popc(j), df_in) : T[p];
      } else {
        x[j] = from_store ? A::from_store_f(reinterpret_cast<const S*>(T)[p], df_in) : T[p];
      }
    }
    for (int k = 0; k < sr.nops; k++) {
      const RegOp op = load_regop(rops + sr.op0 + k);
      if ((base & op.gmask) != op.gmask) continue;
      // the two most frequent ops (merged tangent-form RX runs and phase tables) skip the
      // general dispatch; neither carries controls outside the registers
      if (op.type == OP_RXTM) {
        r_rxt_multi<A, K>(x, pool + op.mat, op.csl, (uint32_t)(uint8_t)op.neg);
      } else if (op.type == OP_DTAB) {
        r_dtab<A, K>(x, pool + op.mat, op.csl);
      } else if constexpr (Lite) {
        // passes whose register ops are all of the four kinds below (the host checks): the
        // remaining two inline, without the general dispatch's code for the other kinds
        if ((gidx & op.cot) != op.cot) continue;
        if (op.type == OP_PHASE) {
          const uint32_t csl = op.csl;
          if (op.neg) {
#pragma unroll
            for (int j = 0; j < (1 << K); j++)
              if ((j & csl) == csl) x[j] = A::neg(x[j]);
          } else {
            const typename A::mat_t d = pool[op.mat];
#pragma unroll
            for (int j = 0; j < (1 << K); j++)
              if ((j & csl) == csl) x[j] = A::mul(d, x[j]);
          }
        } else if (op.type == OP_RX) {
          QS_SLOT_DISPATCH(r_rx, op.s0, x, pool + op.mat, op.csl);
        }
      } else {
        apply_regop<A, K>(x, op, pool, gidx, base);
      }
    }
    // recompute the store addresses from a value the compiler cannot equate with the load
    // addresses, so that 2^K addresses are not kept live across the op loop
    uint32_t spos = gpos;
    asm volatile("" : "+r"(spos));
    if constexpr (kPairable) {
      if (pair) {
#pragma unroll
        for (int j = 0; j < (1 << K); j += 2) {
          uint32_t p = spos;
#pragma unroll
          for (int b = 1; b < K; b++)
            if ((j >> b) & 1) p += pb[b];
          *reinterpret_cast<float4*>(&T[p]) = make_float4(x[j].x, x[j].y, x[j + 1].x, x[j + 1].y);
        }
        continue;
      }
    }
#pragma unroll
    for (int j = 0; j < (1 << K); j++) {
      uint32_t p = spos;
#pragma unroll
      for (int b = 0; b < K; b++)
        if ((j >> b) & 1) p += pb[b];
      if constexpr (std::is_same<R, S>::value) {
        T[p] = x[j];
      } else if constexpr (A::kFrame) {
        if (to_store) reinterpret_cast<S*>(T)[p] = store_framed<A>(x[j], wb + wg + __popc(j), df_out);
        else T[p] = x[j];
      } else {
        if (to_store) reinterpret_cast<S*>(T)[p] = A::to_store_f(x[j], df_out);
        else T[p] = x[j];
      }
    }
  }
}

// Shared memory of a tile CTA: the mbarrier in the first 16 bytes, the tile from byte 128.
constexpr uint32_t kTileSmemOffset = 128;

// Process block b of tile pass tp on the state at psi: load, stages, store.  Returns false
// when the load's bounded wait expired (the status word is set).
template <class A, int K, bool Lite>
__device__ __forceinline__ bool process_block(const typename A::store_t* psi, typename A::store_t* dst,
                                              const TilePass& tp, uint64_t b,
                                              const StageRec* __restrict__ stages, const RegOp* __restrict__ rops,
                                              const DevOp* __restrict__ dops, const typename A::mat_t* __restrict__ pool,
                                              int* __restrict__ status, unsigned char* smem, uint32_t bar,
                                              uint32_t& phase) {
  using S = typename A::store_t;
  using R = typename A::reg_t;
  static_assert(sizeof(R) == sizeof(S), "in-place conversion needs equal element sizes");
  constexpr bool kConv = !std::is_same<R, S>::value;
  const int L = tp.L, c = tp.c;
  const Pad px{c, (int)(16 / sizeof(S))};
  const uint32_t nelem = 1u << L;
  const uint32_t nseg = 1u << (L - c);
  const uint32_t seg_bytes = (uint32_t)sizeof(S) << c;
  const uint32_t seg_stride = seg_bytes + 16u;
  R* T = reinterpret_cast<R*>(smem + kTileSmemOffset);
  const uint32_t tile_s = smem_u32(T);
  const int tid = threadIdx.x;
  const int nout = tp.n - L;
  uint64_t base = 0;
  for (int k = 0; k < nout; k++)
    if ((b >> k) & 1ull) base |= 1ull << tp.npos[k];

  // ---- load: 2^(L-c) bulk copies of 2^c contiguous amplitudes, counted on the mbarrier
  if (tid == 0) mbar_arrive_expect_tx(bar, nseg * seg_bytes);
  __syncthreads();
  for (uint32_t s = tid; s < nseg; s += kTileThreads) {
    uint64_t off = 0;
    for (int k = 0; k < L - c; k++)
      if ((s >> k) & 1u) off |= 1ull << tp.tpos[c + k];
    bulk_load(tile_s + s * seg_stride, psi + (base | off), seg_bytes, bar);
  }
  // every thread waits with its own bounded deadline; the CTA then decides as one whether
  // to go on, so that no thread is left at a later barrier when another gave up.  After a
  // timeout the tile's contents (and this pass's result) are undefined.
  const bool loaded = mbar_wait(bar, phase, globaltimer() + kWaitNs);
  if (__syncthreads_or(!loaded)) {
    if (tid == 0) atomicExch(status, (int)QS_ETIMEOUT);
    return false;
  }
  phase ^= 1u;

  // ---- stages
  const bool df_in = (tp.flags & kPassInDF) != 0, df_out = (tp.flags & kPassOutDF) != 0;
  const uint32_t wb = (uint32_t)__popcll(base) & 3u;   // the block's share of the storage-address frame
  bool in_store = true;   // the tile holds storage-format elements
  for (int k = 0; k < tp.nst; k++) {
    const StageRec sr = stages[tp.st0 + k];
    const bool last = (k == tp.nst - 1);
    if (sr.kind == 0) {
      run_reg_stage<A, K, Lite>(T, sr, rops, pool, L, px, base, in_store, last, df_in, df_out, wb);
      in_store = last;
    } else {
      if (kConv && in_store) {
        S* Ts = reinterpret_cast<S*>(T);
        for (uint32_t i = tid; i < nelem; i += kTileThreads) T[px(i)] = load_framed<A>(Ts[px(i)], wb + __popc(i), df_in);
        __syncthreads();
      }
      in_store = false;
      for (int o = 0; o < sr.nops; o++) {
        const DevOp& op = dops[sr.op0 + o];
        if ((base & op.gmask) != op.gmask) continue;
        apply_op<A>(T, L, op, pool, base, px);
        __syncthreads();
      }
    }
    __syncthreads();
  }
  if (kConv && !in_store) {
    S* Ts = reinterpret_cast<S*>(T);
    for (uint32_t i = tid; i < nelem; i += kTileThreads) {
      const R v = T[px(i)];
      Ts[px(i)] = store_framed<A>(v, wb + __popc(i), df_out);
    }
  }
  // ---- store: bulk copies back (to dst); the tile is reused only after they have been
  // read.  A PermuteQubits fused into the pass exchanges storage bits swap_a and swap_b of
  // every address (both >= c, so segments stay contiguous; dst is then another buffer).
  fence_async_smem();
  __syncthreads();
  const int sa = tp.swap_a, sb = tp.swap_b;
  for (uint32_t s = tid; s < nseg; s += kTileThreads) {
    uint64_t off = 0;
    for (int k = 0; k < L - c; k++)
      if ((s >> k) & 1u) off |= 1ull << tp.tpos[c + k];
    uint64_t addr = base | off;
    const uint64_t d = ((addr >> sa) ^ (addr >> sb)) & 1ull;   // 0 when sa == sb
    addr ^= (d << sa) | (d << sb);
    bulk_store(dst + addr, tile_s + s * seg_stride, seg_bytes);
  }
  bulk_commit();
  bulk_wait_read0();
  __syncthreads();
  return true;
}

__device__ __forceinline__ uint32_t init_tile_barrier(unsigned char* smem) {
  const uint32_t bar = smem_u32(smem);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_async_smem();
  }
  __syncthreads();
  return bar;
}

template <class A, int K, bool Lite>
__global__ void __launch_bounds__(kTileThreads, 2)
    k_tile_staged(const typename A::store_t* psi, typename A::store_t* dst, const TilePass tp,
                  const StageRec* __restrict__ stages,
                  const RegOp* __restrict__ rops, const DevOp* __restrict__ dops,
                  const typename A::mat_t* __restrict__ pool, int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t bar = init_tile_barrier(smem);
  const uint64_t nblocks = 1ull << (tp.n - tp.L);
  uint32_t phase = 0;
  for (uint64_t b = blockIdx.x; b < nblocks; b += gridDim.x)
    if (!process_block<A, K, Lite>(psi, dst, tp, b, stages, rops, dops, pool, status, smem, bar, phase)) return;
  bulk_wait0();
}

// Many independent tile passes in one persistent launch: work item i is block
// i - prefix[p] of pass p, where prefix[p] <= i < prefix[p + 1]; pass p acts on the state
// at psi + passes[p].psi_off.
template <class A, int K>
__global__ void __launch_bounds__(kTileThreads, 2)
    k_tile_batched(typename A::store_t* __restrict__ psi, const BatchPass* __restrict__ passes,
                   const uint64_t* __restrict__ prefix, int npass, const StageRec* __restrict__ stages,
                   const RegOp* __restrict__ rops, const DevOp* __restrict__ dops,
                   const typename A::mat_t* __restrict__ pool, int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t bar = init_tile_barrier(smem);
  const uint64_t total = prefix[npass];
  uint32_t phase = 0;
  for (uint64_t i = blockIdx.x; i < total; i += gridDim.x) {
    int lo = 0, hi = npass - 1;   // last p with prefix[p] <= i
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    const BatchPass& bp = passes[lo];
    if (!process_block<A, K, false>(psi + bp.psi_off, psi + bp.psi_off, bp.tp, i - prefix[lo], stages, rops, dops,
                                    pool, status, smem, bar, phase))
      return;
  }
  bulk_wait0();
}

// The shared-memory opt-in and the SM count belong to each device's context: one bit per
// device records that the attribute is set, the SM count is read on every launch (cheap).
template <class F>
cudaError_t tile_kernel_setup(F* kernel, std::atomic<uint64_t>& configured, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0;
  if (!bit || !(configured.load() & bit)) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit);
  }
  return cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
}

template <class A, int K, bool Lite>
cudaError_t launch_staged_t(const void* psi, void* dst, const TilePass& tp, const StageRec* stages, const RegOp* rops,
                            const DevOp* dops, const void* pool, int* status, cudaStream_t st) {
  using S = typename A::store_t;
  const size_t smem = kTileSmemOffset + ((size_t)1 << (tp.L - tp.c)) * (((size_t)sizeof(S) << tp.c) + 16);
  static std::atomic<uint64_t> configured{0};
  int sms = 0;
  cudaError_t e = tile_kernel_setup(k_tile_staged<A, K, Lite>, configured, &sms);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_staged<A, K, Lite>, kTileThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t nblocks = 1ull << (tp.n - tp.L);
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > nblocks) grid = nblocks;
  k_tile_staged<A, K, Lite><<<(unsigned)grid, kTileThreads, smem, st>>>((const S*)psi, (S*)dst, tp, stages, rops,
                                                                         dops, (const typename A::mat_t*)pool, status);
  return cudaGetLastError();
}

// The lighter dispatch is built for the complex64 policy at its default register width,
// where it was measured faster (9 % on the 30-qubit circuit); for double-float it was slower.
template <class A, int K>
cudaError_t launch_staged(const void* psi, void* dst, const TilePass& tp, const StageRec* stages, const RegOp* rops,
                          const DevOp* dops, const void* pool, int* status, cudaStream_t st) {
  if constexpr (std::is_same<A, AF32>::value && K == 5)
    if (tp.flags & kPassLite) return launch_staged_t<A, K, true>(psi, dst, tp, stages, rops, dops, pool, status, st);
  return launch_staged_t<A, K, false>(psi, dst, tp, stages, rops, dops, pool, status, st);
}

template <class A, int K>
cudaError_t launch_batched_t(void* psi, const BatchPass* passes, const uint64_t* prefix, int npass, uint64_t total_blocks,
                             int maxL, int minc, const StageRec* stages, const RegOp* rops, const DevOp* dops,
                             const void* pool, int* status, cudaStream_t st) {
  using S = typename A::store_t;
  const size_t smem = kTileSmemOffset + ((size_t)1 << (maxL - minc)) * (((size_t)sizeof(S) << minc) + 16);
  static std::atomic<uint64_t> configured{0};
  int sms = 0;
  cudaError_t e = tile_kernel_setup(k_tile_batched<A, K>, configured, &sms);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_batched<A, K>, kTileThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > total_blocks) grid = total_blocks;
  if (grid < 1) return cudaSuccess;
  k_tile_batched<A, K><<<(unsigned)grid, kTileThreads, smem, st>>>((S*)psi, passes, prefix, npass, stages, rops, dops,
                                                                    (const typename A::mat_t*)pool, status);
  return cudaGetLastError();
}

template <class A>
cudaError_t launch_batched_k(int K, void* psi, const BatchPass* passes, const uint64_t* prefix, int npass,
                             uint64_t total, int maxL, int minc, const StageRec* stages, const RegOp* rops,
                             const DevOp* dops, const void* pool, int* status, cudaStream_t st) {
  switch (K) {
    case 1: return launch_batched_t<A, 1>(psi, passes, prefix, npass, total, maxL, minc, stages, rops, dops, pool, status, st);
    case 2: return launch_batched_t<A, 2>(psi, passes, prefix, npass, total, maxL, minc, stages, rops, dops, pool, status, st);
    case 3: return launch_batched_t<A, 3>(psi, passes, prefix, npass, total, maxL, minc, stages, rops, dops, pool, status, st);
    case 4: return launch_batched_t<A, 4>(psi, passes, prefix, npass, total, maxL, minc, stages, rops, dops, pool, status, st);
    case 5:
      if constexpr (sizeof(typename A::reg_t) <= 8)
        return launch_batched_t<A, 5>(psi, passes, prefix, npass, total, maxL, minc, stages, rops, dops, pool, status, st);
      break;
  }
  return cudaErrorInvalidValue;
}

template <class A>
cudaError_t launch_tile_t(const void* psi, void* dst, const TilePass& tp, const StageRec* stages, const RegOp* rops,
                          const DevOp* dops, const void* pool, int* status, cudaStream_t st) {
  switch (tp.K) {
    case 1: return launch_staged<A, 1>(psi, dst, tp, stages, rops, dops, pool, status, st);
    case 2: return launch_staged<A, 2>(psi, dst, tp, stages, rops, dops, pool, status, st);
    case 3: return launch_staged<A, 3>(psi, dst, tp, stages, rops, dops, pool, status, st);
    case 4: return launch_staged<A, 4>(psi, dst, tp, stages, rops, dops, pool, status, st);
    case 5:
      if constexpr (sizeof(typename A::reg_t) <= 8)
        return launch_staged<A, 5>(psi, dst, tp, stages, rops, dops, pool, status, st);
      break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int tile_pass_smem_bytes(Policy pol, int L) {
  const int e = (pol == POL_F32) ? 8 : 16;
  return (e << L) + (16 << L) + 16;   // upper bound (padding for c = 0)
}

cudaError_t launch_tile_batched(Policy pol, int K, void* psi, const BatchPass* passes, const uint64_t* prefix,
                                int npass, uint64_t total_blocks, int maxL, int minc, const StageRec* stages,
                                const RegOp* rops, const DevOp* dops, const void* pool, int* status, cudaStream_t s) {
  switch (pol) {
    case POL_F32: return launch_batched_k<AF32>(K, psi, passes, prefix, npass, total_blocks, maxL, minc, stages, rops, dops, pool, status, s);
    case POL_F64: return launch_batched_k<AF64>(K, psi, passes, prefix, npass, total_blocks, maxL, minc, stages, rops, dops, pool, status, s);
    case POL_DF: return launch_batched_k<ADF>(K, psi, passes, prefix, npass, total_blocks, maxL, minc, stages, rops, dops, pool, status, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tile_pass(Policy pol, const void* psi, void* dst, const TilePass& tp, const StageRec* stages_dev,
                             const RegOp* regops_dev, const DevOp* ops_dev, const void* pool, int* status_dev,
                             cudaStream_t s) {
  if (tp.nst == 0 && tp.swap_a == tp.swap_b && psi == dst) return cudaSuccess;
  switch (pol) {
    case POL_F32: return launch_tile_t<AF32>(psi, dst, tp, stages_dev, regops_dev, ops_dev, pool, status_dev, s);
    case POL_F64: return launch_tile_t<AF64>(psi, dst, tp, stages_dev, regops_dev, ops_dev, pool, status_dev, s);
    case POL_DF: return launch_tile_t<ADF>(psi, dst, tp, stages_dev, regops_dev, ops_dev, pool, status_dev, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qs
