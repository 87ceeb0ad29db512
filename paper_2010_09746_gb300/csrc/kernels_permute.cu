// Qubit permutation (K3): PermuteQubits(sigma') as a bit-index transpose (Sec. 2, App. A).
//
// The vector stored under sigma is rewritten under sigma': out[j'] = in[j] where storage bit
// p of j' carries the logical qubit that sat at storage bit src_of[p] of j
// (src_of = sigma o sigma'^{-1}).  A pure move of whole elements: bit-exact.
//
// Each CTA stages a tile in shared memory: the tile bits are the c lowest output bits and
// the input bits they come from, plus the c lowest input bits and the output bits they go
// to (at most 2c bits of each index), so that both the HBM reads and the HBM writes are
// 2^c-element contiguous segments (128-byte lines and up for c >= 3 at 16-byte elements).
// The remaining bits enumerate tiles; their input->output mapping is a byte-table lookup.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qs_internal.h"

namespace qs {

namespace {

constexpr int kPermThreads = 256;
// elements staged per CTA and iteration, and resident CTAs per SM: 8 CTAs of ~20 KiB keep
// about 128 KiB of reads in flight per SM
constexpr int kPermElems = 1024;
constexpr int kPermCtasPerSm = 8;

struct PermArgs {
  int n;
  int tb;                       // tile bits (input side), ascending in tin[]
  int tin[16];                  // input storage bits of the tile, ascending
  int wk[16];                   // rank-th lowest output tile bit comes from tile bit wk[rank]
  int wp[16];                   // and sits at output position wp[rank]
  int nrest;                    // remaining bits
  int rin[kMaxQubits];          // their input positions (ascending)
  int rout[kMaxQubits];         // and output positions
};

// shared-memory layout of the permutation kernel (byte offsets, every region 16-byte aligned)
struct PermSmem {
  size_t off_in, off_out, r_of, bin, bout, buf;
};
__host__ __device__ inline size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline PermSmem perm_smem_layout(int T, int tiles_per_iter) {
  PermSmem L;
  L.off_in = 0;
  L.off_out = round16(L.off_in + 8 * (size_t)T);
  L.r_of = round16(L.off_out + 8 * (size_t)T);
  L.bin = round16(L.r_of + 4 * (size_t)T);
  L.bout = round16(L.bin + 8 * (size_t)tiles_per_iter);
  L.buf = round16(L.bout + 8 * (size_t)tiles_per_iter);
  return L;
}

// one padding element per 128 bytes of staged tile: the write phase reads the tile in the
// output's bit order, and without padding 8 consecutive output elements that come from
// input bits >= 3 would sit 128 bytes apart in one bank group
template <class S>
__device__ __forceinline__ int pad_idx(int i) {
  return i + (i >> (sizeof(S) == 16 ? 3 : 4));
}

template <class S>
__global__ void __launch_bounds__(kPermThreads) k_permute_tiled(S* __restrict__ dst, const S* __restrict__ src,
                                                               const PermArgs a, int tiles_per_iter) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = 1 << a.tb;
  // tables shared by every tile: input offset of tile-local index r, output offset of
  // output-ordered index w and the tile-local index r it reads
  const PermSmem L = perm_smem_layout(T, tiles_per_iter);
  uint64_t* off_in = reinterpret_cast<uint64_t*>(smem + L.off_in);
  uint64_t* off_out = reinterpret_cast<uint64_t*>(smem + L.off_out);
  int* r_of = reinterpret_cast<int*>(smem + L.r_of);
  uint64_t* bin = reinterpret_cast<uint64_t*>(smem + L.bin);
  uint64_t* bout = reinterpret_cast<uint64_t*>(smem + L.bout);
  S* buf = reinterpret_cast<S*>(smem + L.buf);
  for (int r = threadIdx.x; r < T; r += kPermThreads) {
    uint64_t oi = 0, oo = 0;
    int rr = 0;
    for (int k = 0; k < a.tb; k++) {
      if ((r >> k) & 1) oi |= 1ull << a.tin[k];
      if ((r >> k) & 1) {
        rr |= 1 << a.wk[k];
        oo |= 1ull << a.wp[k];
      }
    }
    off_in[r] = oi;
    off_out[r] = oo;
    r_of[r] = rr;
  }
  const uint64_t ntiles = 1ull << a.nrest;
  for (uint64_t tile0 = (uint64_t)blockIdx.x * tiles_per_iter; tile0 < ntiles;
       tile0 += (uint64_t)gridDim.x * tiles_per_iter) {
    const int cnt = (int)((ntiles - tile0) < (uint64_t)tiles_per_iter ? (ntiles - tile0) : tiles_per_iter);
    for (int u = threadIdx.x; u < cnt; u += kPermThreads) {
      const uint64_t t = tile0 + u;
      uint64_t ji = 0, jo = 0;
      for (int k = 0; k < a.nrest; k++)
        if ((t >> k) & 1ull) {
          ji |= 1ull << a.rin[k];
          jo |= 1ull << a.rout[k];
        }
      bin[u] = ji;
      bout[u] = jo;
    }
    __syncthreads();
    // read: tile-local index r enumerates the input tile bits in ascending order, so the
    // lowest input bits vary fastest (contiguous segments)
    for (int idx = threadIdx.x; idx < cnt * T; idx += kPermThreads) {
      const int u = idx >> a.tb, r = idx & (T - 1);
      buf[pad_idx<S>(idx)] = src[bin[u] | off_in[r]];
    }
    __syncthreads();
    // write: w enumerates the output tile bits in ascending output order
    for (int idx = threadIdx.x; idx < cnt * T; idx += kPermThreads) {
      const int u = idx >> a.tb, w = idx & (T - 1);
      dst[bout[u] | off_out[w]] = buf[pad_idx<S>((u << a.tb) | r_of[w])];
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_permute(void* dst, const void* src, int n, int store_bytes, const int* src_of, cudaStream_t s) {
  // output bit p takes input bit src_of[p]; dst_of[input bit] = output bit
  int dst_of[kMaxQubits];
  for (int p = 0; p < n; p++) dst_of[src_of[p]] = p;
  const int c = (store_bytes == 16) ? 3 : 4;   // 128-byte segments
  const int cc = c < n ? c : n;
  bool in_tile[kMaxQubits] = {};
  for (int p = 0; p < cc; p++) {
    in_tile[p] = true;            // lowest input bits
    in_tile[src_of[p]] = true;    // input bits that become the lowest output bits
  }
  PermArgs a{};
  a.n = n;
  a.tb = 0;
  a.nrest = 0;
  int tout[16];
  for (int b = 0; b < n; b++) {
    if (in_tile[b]) {
      a.tin[a.tb] = b;
      tout[a.tb] = dst_of[b];
      a.tb++;
    } else {
      a.rin[a.nrest] = b;
      a.rout[a.nrest] = dst_of[b];
      a.nrest++;
    }
  }
  // output tile bits in ascending output position
  int rank = 0;
  for (int p = 0; p < n; p++)
    for (int k = 0; k < a.tb; k++)
      if (tout[k] == p) {
        a.wk[rank] = k;
        a.wp[rank] = p;
        rank++;
      }
  const int T = 1 << a.tb;
  int tiles_per_iter = kPermElems / T;
  if (tiles_per_iter < 1) tiles_per_iter = 1;
  const size_t elems = (size_t)tiles_per_iter * T;
  const size_t pad = elems / (store_bytes == 16 ? 8 : 16) + 1;
  const size_t smem = perm_smem_layout(T, tiles_per_iter).buf + (elems + pad) * store_bytes;
  int sms = 0, dev = 0;   // per device: the SM count of the current one
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint64_t ntiles = 1ull << a.nrest;
  uint64_t grid = (ntiles + tiles_per_iter - 1) / tiles_per_iter;
  const uint64_t cap = (uint64_t)sms * kPermCtasPerSm;
  if (grid > cap) grid = cap;
  if (store_bytes == 16) {
    cudaFuncSetAttribute(k_permute_tiled<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    k_permute_tiled<double2><<<(unsigned)grid, kPermThreads, smem, s>>>((double2*)dst, (const double2*)src, a,
                                                                        tiles_per_iter);
  } else {
    cudaFuncSetAttribute(k_permute_tiled<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    k_permute_tiled<float2><<<(unsigned)grid, kPermThreads, smem, s>>>((float2*)dst, (const float2*)src, a,
                                                                       tiles_per_iter);
  }
  return cudaGetLastError();
}

}  // namespace qs
