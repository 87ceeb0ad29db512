// K4: a dense k-qubit block (k <= 6) on the lowest storage bits of a complex64 state, on
// the 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// The block acts on storage bits 0..k-1.  Seen as rows of 64 complex64 amplitudes (storage
// bits 0..5 inside a row), the state is a row-major matrix Psi with 2^(n-6) rows of 128
// floats (re, im interleaved), and the gate is Psi' = Psi W with one 128 x 128 real matrix W
// (the complex 2^k x 2^k block, replicated on the diagonal over storage bits k..5 when k < 6,
// written as a real matrix that maps interleaved (re, im) inputs to interleaved outputs).
//
// Each MMA computes D[j][r] = sum_c W^T[j][c] Psi[r][c] for the 128 output columns j and a
// tile of 64 rows r: A = W^T lives in tensor memory for the whole launch, B = the state tile
// is read from shared memory (K-major, no swizzle), D (128 lanes x 64 columns FP32) is read
// back one output column per thread.  Near-FP32 accuracy from TF32
// operands with the three-term split x = x_big + x_small (x_big = x rounded to TF32,
// x_small = x - x_big rounded to TF32, so each factor is kept to about 2^-22 relative):
// W^T_big x_big + W^T_small x_big + W^T_big x_small, accumulated in FP32.  The tensor core
// rounds each accumulation toward zero, which biases magnitudes downward by a fraction of
// an ulp per MMA; the big x big products therefore go to one accumulator (16 MMAs) and the
// cross terms (2^-11 smaller) to a second, summed with round-to-nearest in the epilogue.
//
// Persistent grid, one CTA per SM (225 KiB of shared memory), warp-specialised so that the
// tensor core works while the threads move data.  Warps 0-15 (four per tensor-memory lane
// quarter) bring 32 KiB row tiles (64 rows) into a ring of 3 row-major staging buffers with
// bulk copies (mbarrier completion, loads issued 3 tiles ahead) and split tile j into operand
// buffer j & 1; one lane of warp 16 issues tile j's 48 MMAs into accumulator set j & 1 as soon
// as the split is handed over (mbarrier), and commits them to another mbarrier.  While the
// MMAs of tile j + 1 run, warps 0-15 read tile j back (one output column and 16 rows per thread,
// `tcgen05.ld`), store the rows to HBM straight from the registers (each warp store
// instruction writes one full 128-byte line) and release the accumulator set.  A staging
// slot is refilled as soon as its tile is split.
// Every wait is bounded by a 2 s %globaltimer deadline; on expiry the CTA records
// QS_ETIMEOUT, waits (bounded) for its copies and MMAs in flight, frees its tensor memory
// and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "qs_internal.h"

namespace qs {
namespace {

constexpr int kThreads = 512;                        // data warps 0-15 (four per tensor-memory lane quarter)
constexpr int kMmaWarp = kThreads / 32;              // the warp that issues the MMAs
constexpr int kBlockThreads = kThreads + 32;
constexpr int kRowFloats = 128;                      // 64 complex64 amplitudes
constexpr int kRows = 64;                            // rows per tile = MMA N (32 rows measured slower)
constexpr int kTileFloats = kRows * kRowFloats;      // 8192
constexpr uint32_t kTileBytes = kTileFloats * 4;     // 32 KiB
constexpr int kStages = 3;                           // row-major staging buffers for loads
constexpr int kOpBytes = 2 * (int)kTileBytes;        // one operand buffer: big then small (K-major)
constexpr int kOffOp = kStages * (int)kTileBytes;    // two operand buffers follow the staging ring
constexpr int kOffBar = kOffOp + 2 * kOpBytes;
constexpr int kSmemUsed = kOffBar + 256;             // barriers, tensor-memory address, abort flag
constexpr int kSmemAlloc = kSmemUsed + 1024;         // slack for aligning the base to 1 KiB
// tensor memory columns: [0,128) W^T big, [128,256) W^T small, then two accumulator sets
// (tile parity b) of two 64-column FP32 accumulators: at 256 + 128 b the big x big
// products, at 320 + 128 b the two small cross terms
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColWBig = 0, kColWSmall = 128, kColAcc = 256;
constexpr uint32_t kLBO = kRows * 16;                // K-direction stride between 8x16 B core matrices
constexpr uint32_t kSBO = 128;                       // N-direction stride between 8-row groups
// instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kRows >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
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
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- tensor memory and MMA ---------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
               ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
               : "r"(taddr)
               : "memory");
}
// D[d] (+)= A[a] (tensor memory) * B (shared-memory descriptor)
__device__ __forceinline__ void mma_tf32(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// shared-memory matrix descriptor: start address, leading (K) and stride (N) byte offsets
// in 16-byte units, the fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
         (1ull << 46);
}

// round to the nearest TF32 value (10 significand bits), ties away from zero in magnitude,
// with two integer operations on the binary32 fields (finite inputs of magnitude below
// 2^127); the result has its low 13 bits clear, so the tensor core reads it exactly
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void tf32_split(float x, float& big, float& small) {
  big = tf32_rna(x);
  small = tf32_rna(x - big);   // x - big is exact; |x - big| <= 2^-11 |x|
}

// One tile = 64 rows.  Tile j's operands live in operand buffer j & 1 and its products in
// accumulator set j & 1, so the tensor core runs tile j + 1's MMAs while the threads read
// back tile j and split tile j + 2.
struct DenseSmem {
  unsigned char* base;
  __device__ float* stage(int s) const { return (float*)(base + s * (int)kTileBytes); }
  __device__ unsigned char* big(int b) const { return base + kOffOp + b * kOpBytes; }
  __device__ unsigned char* small(int b) const { return base + kOffOp + b * kOpBytes + (int)kTileBytes; }
};

// split the row-major tile into the K-major operand layout: element group (row r, 4-float
// panel p) goes to p * kLBO + r * 16.  The 8 threads of each shared-memory phase take
// distinct r mod 8 and distinct p mod 8, so reads and writes are conflict-free.
__device__ __forceinline__ void split_tile(const float* stg, unsigned char* big, unsigned char* small, int tid) {
  const float4* src = (const float4*)stg;
#pragma unroll 4
  for (int it = 0; it < kTileFloats / 4 / kThreads; it++) {
    const int g = it * kThreads + tid;
    const int i8 = g & 7, rest = g >> 3;
    const int r = ((rest % (kRows / 8)) << 3) | i8;
    const int p = ((rest / (kRows / 8)) + i8) & 31;
    const float4 x = src[r * 32 + p];
    float4 hb, lo;
    tf32_split(x.x, hb.x, lo.x);
    tf32_split(x.y, hb.y, lo.y);
    tf32_split(x.z, hb.z, lo.z);
    tf32_split(x.w, hb.w, lo.w);
    const uint32_t off = (uint32_t)p * kLBO + (uint32_t)r * 16u;
    *(float4*)(big + off) = hb;
    *(float4*)(small + off) = lo;
  }
}

// 48 MMAs of one tile into accumulator set b, committed to bar (thread 0 only)
__device__ __forceinline__ void issue_tile_mma(uint32_t tmem, const unsigned char* big, const unsigned char* small,
                                               int b, uint32_t bar) {
  tc_fence_after();
  const uint32_t dm = tmem + kColAcc + 2u * kRows * (uint32_t)b, dx = dm + (uint32_t)kRows;
  const uint32_t bb = smem_u32(big), sb = smem_u32(small);
#pragma unroll
  for (int kk = 0; kk < 16; kk++) {
    const uint64_t db = smem_desc(bb + kk * 2 * kLBO), ds = smem_desc(sb + kk * 2 * kLBO);
    mma_tf32(dm, tmem + kColWBig + kk * 8, db, kk > 0 ? 1u : 0u);
    mma_tf32(dx, tmem + kColWSmall + kk * 8, db, kk > 0 ? 1u : 0u);
    mma_tf32(dx, tmem + kColWBig + kk * 8, ds, 1u);
  }
  mma_commit(bar);
}

// barrier 1 over the 512 data threads, OR-reducing a predicate
__device__ __forceinline__ bool data_bar_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, 512, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void data_bar() { asm volatile("bar.sync 1, 512;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Barriers (shared memory, 8 bytes each): full[s] (load of stage s landed), opf[b] (operand
// buffer b split, MMAs may start), accf[b] (MMAs of set b complete, tcgen05.commit),
// acce[b] (accumulator set b read back, may be overwritten).
__global__ void __launch_bounds__(kBlockThreads, 1)
    k_dense_mma(float* __restrict__ psi, uint64_t ntiles, const float* __restrict__ wT, int* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  const DenseSmem sm{(unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023)};
  const uint32_t full0 = smem_u32(sm.base + kOffBar);
  const uint32_t opf0 = full0 + 8 * kStages, accf0 = opf0 + 16, acce0 = accf0 + 16;
  uint32_t* tmem_slot = (uint32_t*)(sm.base + kOffBar + 128);
  volatile int* abort_flag = (volatile int*)(sm.base + kOffBar + 136);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint64_t T = (ntiles > blockIdx.x) ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;   // my tiles
  auto tile_of = [&](uint64_t j) { return blockIdx.x + j * gridDim.x; };

  if (tid == 0) {
    for (int s = 0; s < kStages; s++) mbar_init(full0 + 8 * s, 1);
    for (int b = 0; b < 2; b++) {
      mbar_init(opf0 + 8 * b, 1);
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 1);
    }
    *abort_flag = 0;
    fence_async_smem();
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kMmaWarp) {
    // ---- MMA warp: one lane issues every tile's 48 MMAs in order -----------------------
    if ((tid & 31) == 0) {
      uint64_t j = 0;
      uint32_t open = 0;   // accumulator sets with a commit the data warps have not consumed
      for (; j < T; j++) {
        const int b = (int)(j & 1);
        const uint32_t ph = (uint32_t)((j >> 1) & 1);
        bool ok = true;
        const unsigned long long dl = globaltimer() + kWaitNs;
        while (ok && !mbar_try_wait(opf0 + 8 * b, ph)) ok = !*abort_flag && globaltimer() <= dl;
        while (ok && !mbar_try_wait(acce0 + 8 * b, ph ^ 1u)) ok = !*abort_flag && globaltimer() <= dl;
        if (!ok) {
          *abort_flag = 1;
          break;
        }
        issue_tile_mma(tmem, sm.big(b), sm.small(b), b, accf0 + 8 * b);
        open |= 1u << b;
        (void)open;
      }
      if (*abort_flag) {   // let the MMAs issued so far finish before the memory is released
        const unsigned long long dl = globaltimer() + kWaitNs;
        for (uint64_t q = (j >= 2 ? j - 2 : 0); q < j; q++)
          mbar_wait(accf0 + 8 * (int)(q & 1), (uint32_t)((q >> 1) & 1), dl);
      }
    }
  } else {
    // ---- data warps: loads, splits, read-back, stores ---------------------------------
    // warp w reaches tensor-memory lanes 32 (w mod 4) .. + 31; four warps share each quarter
    const int quarter = warp & 3, slice = warp >> 2;   // slice 0..3
    const int row = quarter * 32 + (tid & 31);   // W^T row = output column of this thread
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    // W^T into tensor memory: slices 0, 1 the big part's columns 0-63 / 64-127, slices 2, 3
    // the small part's
    {
      const int part = slice >> 1;
      for (int c0 = 64 * (slice & 1); c0 < 64 * (slice & 1) + 64; c0 += 32) {
        uint32_t v[32];
        const float4* src = (const float4*)(wT + part * 16384 + row * 128 + c0);
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const float4 f = __ldg(src + q);
          v[4 * q] = __float_as_uint(f.x);
          v[4 * q + 1] = __float_as_uint(f.y);
          v[4 * q + 2] = __float_as_uint(f.z);
          v[4 * q + 3] = __float_as_uint(f.w);
        }
        tmem_st32(tmem + lane_base + (part ? kColWSmall : kColWBig) + c0, v);
      }
    }
    tmem_wait_st();
    tc_fence_before();

    uint64_t issued = 0;   // thread 0: loads issued for tiles < issued
    auto issue_load = [&](uint64_t j) {
      const int s = (int)(j % kStages);
      mbar_arrive_expect_tx(full0 + 8 * s, kTileBytes);
      bulk_load(smem_u32(sm.stage(s)), psi + tile_of(j) * kTileFloats, kTileBytes, full0 + 8 * s);
      issued = j + 1;
    };
    if (tid == 0)
      for (uint64_t j = 0; j < (uint64_t)kStages && j < T; j++) issue_load(j);

    int fail = 0;
    // split tile j into operand buffer j & 1 and hand it to the MMA warp (the MMAs of tile
    // j - 2, the buffer's last reader, completed before tile j - 2 was read back); its stage
    // slot is refilled at once with tile j + kStages's input
    auto split_and_hand = [&](uint64_t j) -> bool {
      const bool ok = mbar_wait(full0 + 8 * (int)(j % kStages), (uint32_t)((j / kStages) & 1), globaltimer() + kWaitNs);
      if (data_bar_or(!ok || *abort_flag)) return false;
      const int b = (int)(j & 1);
      split_tile(sm.stage((int)(j % kStages)), sm.big(b), sm.small(b), tid);
      fence_async_smem();
      data_bar();
      if (tid == 0) {
        mbar_arrive(opf0 + 8 * b);
        if (j + kStages < T) issue_load(j + kStages);
      }
      return true;
    };
    uint64_t i = 0;
    if (T > 0 && !split_and_hand(0)) fail = 1;
    for (; !fail && i < T; i++) {
      const int b = (int)(i & 1);
      if (i + 1 < T && !split_and_hand(i + 1)) {
        fail = 1;
        break;
      }
      // read tile i back once its MMAs are complete and write it to HBM straight from the
      // registers: for each row, the 32 lanes of a warp hold 32 consecutive output floats,
      // so every store instruction writes one full 128-byte line
      const unsigned long long dl = globaltimer() + kWaitNs;
      bool ok = true;
      while (ok && !mbar_try_wait(accf0 + 8 * b, (uint32_t)((i >> 1) & 1))) ok = !*abort_flag && globaltimer() <= dl;
      if (data_bar_or(!ok)) {
        fail = 1;
        break;
      }
      tc_fence_after();
      float* out = psi + tile_of(i) * kTileFloats;
      {   // this warp: output column `row`, tile rows 16 slice .. 16 slice + 15
        const int c0 = (kRows / 4) * slice;
        uint32_t vm[kRows / 4], vx[kRows / 4];
        const uint32_t acc = tmem + lane_base + kColAcc + 2u * kRows * (uint32_t)b + (uint32_t)c0;
        tmem_ld16(acc, vm);
        tmem_ld16(acc + (uint32_t)kRows, vx);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < kRows / 4; c++)
          out[(c0 + c) * kRowFloats + row] = __fadd_rn(__uint_as_float(vm[c]), __uint_as_float(vx[c]));
      }
      tc_fence_before();
      data_bar();
      if (tid == 0) mbar_arrive(acce0 + 8 * b);
    }
    if (tid == 0) {
      if (fail) {
        *abort_flag = 1;
        atomicExch(status, (int)QS_ETIMEOUT);
        // loads still owed to their barriers: wait (bounded) before shared memory is released
        const unsigned long long dl = globaltimer() + kWaitNs;
        for (uint64_t j = (issued > (uint64_t)kStages ? issued - kStages : 0); j < issued; j++)
          mbar_wait(full0 + 8 * (int)(j % kStages), (uint32_t)((j / kStages) & 1), dl);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace


cudaError_t launch_dense_mma(void* psi, int n, const float* wT_dev, int* status, int num_sms, cudaStream_t s) {
  if (n < 12) return cudaErrorInvalidValue;
  // the shared-memory opt-in is a property of the function in each device's context
  static std::atomic<uint64_t> attr_set{0};   // bit d: set on device d (d < 64)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0;
  if (!bit || !(attr_set.load() & bit)) {
    e = cudaFuncSetAttribute(k_dense_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAlloc);
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(bit);
  }
  const uint64_t ntiles = (1ull << (n - 6)) / kRows;   // 2^(n-6) rows of 64 amplitudes
  const uint64_t g = ntiles < (uint64_t)num_sms ? ntiles : (uint64_t)num_sms;
  k_dense_mma<<<(unsigned)g, kBlockThreads, kSmemAlloc, s>>>((float*)psi, ntiles, wT_dev, status);
  return cudaGetLastError();
}

}  // namespace qs
