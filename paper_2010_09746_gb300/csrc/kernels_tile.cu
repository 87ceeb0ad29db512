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
// %globaltimer deadline; on expiry the CTA records QS_ETIMEOUT in *status and returns.
#include <cuda_runtime.h>
#include <stdint.h>

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

// Apply one tile op to the shared-memory tile T (2^L elements in policy register format).
template <class A>
__device__ __forceinline__ void apply_op(typename A::reg_t* T, int L, const DevOp& op,
                                         const typename A::mat_t* __restrict__ pool, uint64_t base) {
  using R = typename A::reg_t;
  using M = typename A::mat_t;
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
        const M u00 = pool[op.mat], u01 = pool[op.mat + 1], u10 = pool[op.mat + 2], u11 = pool[op.mat + 3];
        for (uint32_t t = tid; t < nw; t += kTileThreads) {
          const uint32_t i = texpand(t, pos, nz, cm);
          const R a = T[i], b = T[i | s];
          T[i] = A::mac2(u00, a, u01, b);
          T[i | s] = A::mac2(u10, a, u11, b);
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
      for (uint32_t t = tid; t < nw; t += kTileThreads) {
        const uint32_t i = texpand(t, pos, nz, cm);
        const R a = T[i | s0];
        T[i | s0] = T[i | s1];
        T[i | s1] = a;
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
          R acc = A::mac2(m[4 * r + 0], x[0], m[4 * r + 1], x[1]);
          acc = A::mac(acc, m[4 * r + 2], x[2]);
          acc = A::mac(acc, m[4 * r + 3], x[3]);
          T[idx[r]] = acc;
        }
      }
      break;
    }
    case OP_DENSE: {
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
          off[r] = i | o;
          x[r] = T[off[r]];
        }
        for (int r = 0; r < D; r++) {
          R acc = A::zero();
          for (int c = 0; c < D; c++) acc = A::mac(acc, m[r * D + c], x[c]);
          T[off[r]] = acc;
        }
      }
      break;
    }
    default:
      break;
  }
}

template <class A>
__global__ void __launch_bounds__(kTileThreads) k_tile_pass(typename A::store_t* __restrict__ psi, const TilePass tp,
                                                            const DevOp* __restrict__ ops,
                                                            const typename A::mat_t* __restrict__ pool,
                                                            int* __restrict__ status) {
  using S = typename A::store_t;
  using R = typename A::reg_t;
  static_assert(sizeof(R) == sizeof(S), "in-place conversion needs equal element sizes");
  extern __shared__ __align__(128) unsigned char smem[];
  const int L = tp.L, c = tp.c;
  const uint32_t nelem = 1u << L;
  const uint32_t nseg = 1u << (L - c);
  const uint32_t seg_bytes = (uint32_t)sizeof(S) << c;
  R* T = reinterpret_cast<R*>(smem);
  uint64_t* seg_off = reinterpret_cast<uint64_t*>(smem + (size_t)nelem * sizeof(R));
  uint64_t* bar_p = seg_off + nseg;
  const uint32_t bar = smem_u32(bar_p);
  const uint32_t tile_s = smem_u32(T);
  const int tid = threadIdx.x;

  // segment offsets: deposit the segment index into tile bits c .. L-1
  for (uint32_t s = tid; s < nseg; s += kTileThreads) {
    uint64_t o = 0;
    for (int k = 0; k < L - c; k++)
      if ((s >> k) & 1u) o |= 1ull << tp.tpos[c + k];
    seg_off[s] = o;
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_async_smem();
  }
  __syncthreads();

  const uint64_t nblocks = 1ull << (tp.n - L);
  const int nout = tp.n - L;
  uint32_t phase = 0;
  for (uint64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
    uint64_t base = 0;
    for (int k = 0; k < nout; k++)
      if ((b >> k) & 1ull) base |= 1ull << tp.npos[k];

    // ---- load: 2^(L-c) bulk copies into the tile, counted on the mbarrier
    if (tid == 0) mbar_arrive_expect_tx(bar, nseg * seg_bytes);
    __syncthreads();
    for (uint32_t s = tid; s < nseg; s += kTileThreads)
      bulk_load(tile_s + s * seg_bytes, psi + (base | seg_off[s]), seg_bytes, bar);
    if (!mbar_wait(bar, phase, globaltimer() + kWaitNs)) {
      if (tid == 0) atomicExch(status, (int)QS_ETIMEOUT);
      return;
    }
    phase ^= 1u;

    // ---- convert storage -> register format in place (double-float policy)
    if constexpr (!std::is_same<R, S>::value) {
      S* Ts = reinterpret_cast<S*>(smem);
      for (uint32_t i = tid; i < nelem; i += kTileThreads) T[i] = A::from_store(Ts[i]);
      __syncthreads();
    }

    // ---- the pass's gates
    for (int k = 0; k < tp.nops; k++) {
      const DevOp& op = ops[tp.op0 + k];
      if ((base & op.gmask) != op.gmask) continue;   // block-uniform predicate
      apply_op<A>(T, L, op, pool, base);
      __syncthreads();
    }

    if constexpr (!std::is_same<R, S>::value) {
      S* Ts = reinterpret_cast<S*>(smem);
      for (uint32_t i = tid; i < nelem; i += kTileThreads) {
        const R v = T[i];
        Ts[i] = A::to_store(v);
      }
    }
    // ---- store: bulk copies back; smem is reused only after they have been read
    fence_async_smem();
    __syncthreads();
    for (uint32_t s = tid; s < nseg; s += kTileThreads)
      bulk_store(psi + (base | seg_off[s]), tile_s + s * seg_bytes, seg_bytes);
    bulk_commit();
    bulk_wait_read0();
    __syncthreads();
  }
  bulk_wait0();
}

template <class A>
cudaError_t launch_tile_t(void* psi, const TilePass& tp, const DevOp* ops, const void* pool, int* status,
                          cudaStream_t st) {
  const int smem = (int)((sizeof(typename A::reg_t) << tp.L) + (8u << (tp.L - tp.c)) + 16);
  static int configured_bytes = 0;
  static int sms = 0;
  if (smem > configured_bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_tile_pass<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    configured_bytes = 227 * 1024;
  }
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_pass<A>, kTileThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t nblocks = 1ull << (tp.n - tp.L);
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > nblocks) grid = nblocks;
  k_tile_pass<A><<<(unsigned)grid, kTileThreads, smem, st>>>(
      (typename A::store_t*)psi, tp, ops, (const typename A::mat_t*)pool, status);
  return cudaGetLastError();
}

}  // namespace

int tile_pass_smem_bytes(Policy pol, int L) {
  const int reg = (pol == POL_F32) ? 8 : 16;
  return (reg << L) + (8 << L) + 16;   // upper bound (segment table for c = 0)
}

cudaError_t launch_tile_pass(Policy pol, void* psi, const TilePass& tp, const DevOp* ops_dev, const void* pool,
                             int* status_dev, cudaStream_t s) {
  switch (pol) {
    case POL_F32: return launch_tile_t<AF32>(psi, tp, ops_dev, pool, status_dev, s);
    case POL_F64: return launch_tile_t<AF64>(psi, tp, ops_dev, pool, status_dev, s);
    case POL_DF: return launch_tile_t<ADF>(psi, tp, ops_dev, pool, status_dev, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qs
