// Internal declarations shared by the host runtime, the compiler and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/qs.h"

namespace qs {

using cd = std::complex<double>;

constexpr int kMaxQubits = 36;
constexpr int kMaxTileBits = 14;
constexpr int kMaxDenseK = 6;

// Arithmetic policy selector.
enum Policy : int { POL_F32 = 0, POL_F64 = 1, POL_DF = 2 };

// ------------------------------------------------------------------------------------------
// Device op records.  Bit positions are storage bits for per-gate ops and tile-local bit
// indices for tile ops.  Matrix entries live in a pool (one entry = one complex number in
// the policy's format); `mat` is the index of the first entry.
// ------------------------------------------------------------------------------------------
enum OpType : int32_t {
  OP_U1 = 1,     // general 2x2 on bit k0 (controls cmask)
  OP_RX = 2,     // c*I - i*s*X on bit k0: one pool entry (c, s)
  OP_DIAG = 3,   // diag(d0, d1) on bit k0 (tile op: k0 < 0 -> storage bit `gbit`, block factor)
  OP_X = 4,      // swap of the pair on bit k0 (CNOT / X), controls cmask
  OP_PHASE = 5,  // multiply by d0 where all cmask bits (and gmask bits) are 1: CZ, CP, Z, S, T
  OP_U2 = 6,     // general 4x4 on bits (k0, k1), r = b(k0) + 2 b(k1)
  OP_DENSE = 7,  // general 2^nk x 2^nk on bits kq[0..nk-1]
  OP_SWAP = 8,   // exchange bits k0 and k1 (controls cmask)
  OP_DTAB = 9,   // register stages only: multiply register element j by table entry j
                 // where bit j of csl is set (the other entries are exactly 1)
  OP_RXT = 10,   // register stages only: tangent-form RX, (I - i t X) if s1 == 0 else
                 // (t I - i X); one pool entry (t, 0).  The factor it drops is applied by
                 // a full-form OP_RX of the same pass
  OP_RXTM = 11,  // register stages only: tangent-form RX on every register slot in csl, in
                 // ascending slot order; pool entries (t, 0) per slot, form bits in neg
};

struct DevOp {
  int32_t type;
  int32_t k0, k1;
  int32_t nk;
  uint64_t cmask;     // control bits inside the addressed space (tile-local or storage)
  uint64_t gmask;     // tile ops: storage-bit controls outside the tile (block predicate)
  int32_t mat;        // first pool entry
  int32_t gbit;       // tile OP_DIAG on a bit outside the tile: its storage bit
  int32_t kq[6];
};
static_assert(sizeof(DevOp) == 64, "DevOp layout");

// Register-stage op: a tile op whose target bits are held in registers.  Slots index the
// stage's register bits; controls are split into register slots (csl) and tile bits
// outside the registers (cot); gmask is the block predicate (storage bits outside the tile).
struct alignas(16) RegOp {
  int32_t type;       // OP_U1, OP_RX, OP_RXT, OP_X, OP_DIAG, OP_PHASE, OP_U2, OP_DTAB
  int8_t s0, s1;      // register slots of the target bit(s), -1 if none (OP_RXT: s1 = form)
  int8_t tb;          // OP_DIAG on a tile bit outside the registers, -1 if none
  int8_t neg;         // OP_PHASE: exact sign flip; OP_RXTM: form bit per slot
  uint32_t csl;       // control mask over register slots
  uint32_t cot;       // control mask over tile-local bits outside the registers
  int32_t mat;        // first pool entry
  int32_t gbit;       // OP_DIAG on a storage bit outside the tile, -1 if none
  uint64_t gmask;     // block predicate
};
static_assert(sizeof(RegOp) == 32, "RegOp layout");

// A stage of a tile pass: either K tile bits held in registers by every thread (2^K
// amplitudes per thread) with a list of RegOps, or a list of shared-memory DevOps.
struct StageRec {
  int32_t kind;       // 0 = register stage, 1 = shared-memory stage
  int32_t op0, nops;  // RegOp range (kind 0) or DevOp range (kind 1)
  int32_t rmask;      // kind 0: tile-local bits held in registers
  int32_t rbits[8];   // kind 0: those bits in slot order
};
static_assert(sizeof(StageRec) == 48, "StageRec layout");

// TilePass.flags: every register op of the pass is OP_RXTM, OP_DTAB, OP_PHASE or OP_RX
constexpr int32_t kPassLite = 1;
// TilePass.flags (double-float policy): the pass reads / writes the state in the
// double-float storage form instead of binary64 -- set by the compiler between tile passes
// that follow one another (permutations in between move 16-byte elements unchanged)
constexpr int32_t kPassInDF = 2;
constexpr int32_t kPassOutDF = 4;

// Tile pass launch description.
struct TilePass {
  int32_t L;          // tile bits
  int32_t c;          // low storage bits of every segment (tpos[i] = i for i < c)
  int32_t n;
  int32_t K;          // register bits per thread in register stages
  int32_t st0, nst;   // stage range in the plan's stage array
  int32_t flags;      // kPass* bits
  int32_t swap_a, swap_b;   // PermuteQubits fused into the store: storage bits exchanged in every
                            // stored address (both >= c; equal = none), written to another buffer
  int32_t tpos[kMaxTileBits];        // storage positions of tile bits, ascending
  int32_t npos[kMaxQubits];          // storage positions of the other bits, ascending
};

// One pass of a batch: a tile pass on the state that starts psi_off elements into the batch's
// state buffer.
struct BatchPass {
  TilePass tp;
  uint64_t psi_off;
};

// One plan step.
enum StepKind : int32_t { ST_PASS = 0, ST_GATE = 1, ST_PERMUTE = 2, ST_RENORM = 3, ST_DENSE = 4 };
struct Step {
  StepKind kind;
  TilePass pass{};           // ST_PASS
  DevOp op{};                // ST_GATE (storage bits)
  std::vector<int> perm;     // ST_PERMUTE: new sigma (logical -> storage)
  std::vector<int> src_of;   // ST_PERMUTE: storage bit p of the output takes input bit src_of[p]
  int32_t dense_idx = -1;    // ST_DENSE: block index into CompileResult::dense_w / dense_u
  double bytes = 0;          // algorithmic HBM bytes
  double alu = 0;            // arithmetic instructions the policy's formulas need (all amplitudes)
};

// ------------------------------------------------------------------------------------------
// Kernel launchers (kernels_*.cu).  All take the stream and return cudaError_t of the
// launch.  `pool` is a device array of policy-format matrix entries.
// ------------------------------------------------------------------------------------------
cudaError_t launch_init_zero(void* psi, int n, int store_bytes, cudaStream_t s);
cudaError_t launch_gate(Policy pol, void* psi, int n, const DevOp& op, const void* pool, cudaStream_t s);
// reads the state at psi, writes it to dst (the same buffer unless the pass carries a fused
// permutation, tp.swap_a != tp.swap_b)
cudaError_t launch_tile_pass(Policy pol, const void* psi, void* dst, const TilePass& tp, const StageRec* stages_dev,
                             const RegOp* regops_dev, const DevOp* ops_dev, const void* pool, int* status_dev,
                             cudaStream_t s);
cudaError_t launch_tile_batched(Policy pol, int K, void* psi, const BatchPass* passes, const uint64_t* prefix,
                                int npass, uint64_t total_blocks, int maxL, int minc, const StageRec* stages,
                                const RegOp* rops, const DevOp* dops, const void* pool, int* status, cudaStream_t s);
cudaError_t launch_permute(void* dst, const void* src, int n, int store_bytes, const int* src_of,
                           cudaStream_t s);
cudaError_t launch_norm_partials(const void* psi, int n, int is_c128, double* partials, int nparts,
                                 cudaStream_t s);
cudaError_t launch_norm_final(const double* partials, int nparts, double* out, cudaStream_t s);
cudaError_t launch_probabilities(const void* psi, int n, int is_c128, double* out, const int* sigma,
                                 int logical, cudaStream_t s);
cudaError_t launch_gather_amplitudes(const void* psi, int n, int store_bytes, void* out,
                                     uint64_t first, uint64_t count, const int* sigma, int logical,
                                     cudaStream_t s);
int tile_pass_smem_bytes(Policy pol, int L);
int tile_pass_ctas_per_sm(Policy pol, int L);
int norm_num_partials();
// <a|b> in FP64 into out2[0..1] (device); partials2 holds inner_num_partials() double pairs.
cudaError_t launch_inner(const void* a, int a_c128, const void* b, int b_c128, int n, double* partials2,
                         double* out2, cudaStream_t s);
int inner_num_partials();
// Dense block on storage bits 0..5 of a complex64 state on the tensor cores: every row of
// 64 amplitudes times the 128 x 128 real matrix whose transpose's TF32 split (big, small;
// 2 x 128 x 128 floats) is at wT_dev.  n >= dense_mma_min_qubits().
cudaError_t launch_dense_mma(void* psi, int n, const float* wT_dev, int* status, int num_sms, cudaStream_t s);
constexpr int kDenseMinQubits = 12;   // the tensor-core kernel needs rows of 64 amplitudes x 64
inline int dense_mma_min_qubits() { return kDenseMinQubits; }
// psi *= 1 / sqrt(*norm_dev), skipped on the device if *norm_dev is not positive and finite.
cudaError_t launch_scale(void* psi, int n, int is_c128, const double* norm_dev, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Host gate model shared by the runtime and the compiler.
// ------------------------------------------------------------------------------------------
enum QCls : int { CLS_Z = 0, CLS_X = 1, CLS_N = 2 };

struct HGate {
  int kind;                   // QS_OP_*
  int nq;
  int q[6];                   // logical qubits
  double param;
  std::vector<cd> U;          // full 2^nq x 2^nq matrix over q[] (r = sum b(q_t) 2^t)
  int cls[6];                 // action class per qubit
};

// Build the HGate of an ABI op (validates qubits and matrix offsets).
bool make_hgate(int n, const qs_op& op, const double* mats, size_t nmats, HGate* out, std::string* err);

// A single-qubit gate on logical qubit q with the 2x2 matrix m (row-major), classified.
HGate make_1q_gate(int q, const cd m[4]);
// U = d2 . rx . d1 for a 2x2 unitary U: d1 = diag(1, e^{i d}), rx = c I - i s X (c, s >= 0),
// d2 diagonal (the Euler angles of U about Z, X, Z).  False if the factors miss U by more
// than 1e-13 in some entry.
bool euler_split(const cd U[4], cd d1[4], cd rx[4], cd d2[4]);
// Gate fusion for QS_MODE_TILE: every maximal run of single-qubit gates on one qubit (no
// multi-qubit gate on that qubit in between) that holds at least two non-diagonal gates, a
// general one (neither RX nor X in form), or only diagonal ones, is replaced by its product,
// re-expressed as at most three gates
// (diagonal, RX, diagonal).  The origin lists the input gates each output gate stands for
// (empty for the extra factors of a product); every input gate appears exactly once.  The
// input gates are moved into the output (`in` is consumed).
struct FuseOrigin {
  std::vector<int> off, idx;   // output gate i stands for input gates idx[off[i] .. off[i + 1])
  int count(size_t i) const { return off[i + 1] - off[i]; }
};
void fuse_single_qubit_runs(int n, std::vector<HGate>& in, std::vector<HGate>* out, FuseOrigin* origin);
// Matrix pool in policy format.
struct Pool {
  std::vector<double> f64;  // (re, im) pairs
  int add(const cd& z) {
    f64.push_back(z.real());
    f64.push_back(z.imag());
    return (int)(f64.size() / 2 - 1);
  }
  size_t entries() const { return f64.size() / 2; }
  // serialised for a policy: F32 -> float2, F64 -> double2, DF -> 48-byte lane patterns
  std::vector<unsigned char> serialise(Policy pol) const;
  void serialise_into(Policy pol, unsigned char* dst) const;   // entries() * entry_bytes(pol) bytes
  static size_t entry_bytes(Policy pol);
};

// Lower one gate to device ops with positions mapped through `bitpos` (logical qubit ->
// target bit index in the addressed space) for gates whose non-diagonal qubits are all
// addressable; `ctrl_outside` receives storage-bit controls that are not addressable
// (tile ops only).  Returns false if the gate needs a bit that is not addressable.
struct LowerCtx {
  const int* sigma;           // logical -> storage bit
  bool tile;                  // lowering for a tile pass
  int tile_index[64];         // storage bit -> tile-local index, -1 if outside
};
bool lower_gate(const HGate& g, const LowerCtx& ctx, Pool& pool, std::vector<DevOp>& out);

// ------------------------------------------------------------------------------------------
// Compiler (compiler.cpp)
// ------------------------------------------------------------------------------------------
struct CompileResult {
  int store_bytes = 16;
  Policy pol = POL_DF;
  int reg_bits = 0;              // requested register bits (0 = default)
  bool full_rx = false;          // QS_FLAG_FULL_RX: no tangent-form RX in register stages
  std::vector<Step> steps;
  std::vector<std::pair<int, int>> trace;   // QS_MODE_PAPER: (0 local gate | 1 non-local gate | 2 permute, value)
  std::vector<DevOp> tile_ops;   // shared-memory ops of all passes, concatenated
  std::vector<RegOp> reg_ops;    // register-stage ops of all passes
  std::vector<StageRec> stages;  // stages of all passes
  Pool pool;
  // ST_DENSE blocks: the fused 64 x 64 unitary on storage bits 0..5 (row / column index =
  // those bits), and the tensor-core kernel's operand made from it (kDenseWFloats each)
  std::vector<cd> dense_u;
  std::vector<float> dense_w;
  qs_cost_model cost{};          // the model the compiler used (also for predicted_ms)
  std::vector<int> sigma_final;
  qs_plan_stats stats{};
};
bool compile_circuit(int n, std::vector<HGate> gates, const std::vector<int>& sigma0,
                     const qs_compile_opts& o, CompileResult* out, std::string* err);

// Cost model the compiler uses when the caller gives none: per-launch coefficients measured
// on GB300 for the policy's kernels.
qs_cost_model default_cost_model(Policy pol);
// predicted time of one step under a model
double step_cost_ms(const qs_cost_model& m, const Step& s);

// Floats of one dense block operand: W^T of the real 128 x 128 matrix, split into its nearest
// TF32 values and the TF32-rounded remainders.
constexpr size_t kDenseWFloats = 2 * 128 * 128;
// That operand for the 2^k x 2^k complex block U (row / column r = sum_t b(q_t) 2^t) whose qubit
// t sits on storage bit bits[t] (a permutation of 0..k-1), replicated over storage bits k..5.
void dense_mma_weights(const double* U, int k, const int* bits, float* out);

// Dependency DAG with commutation-pruned edges: immediate predecessors per gate.
std::vector<std::vector<int>> build_dag(const std::vector<HGate>& gates);

// Thread-local error text returned by qs_last_error (capi.cpp).
void set_last_error(const std::string& msg);

int default_tile_bits(int dtype);
int default_low_bits(int dtype);
// Validate compile options and fill in the defaults (tile and low bits for the dtype,
// clamped to the state); false with a message if they are invalid.
bool normalize_compile_opts(int n, qs_compile_opts* o, std::string* err);
int register_bits(int dtype, int L, int requested);

// Split a pass's op list (tile-local DevOps, program order) into register / shared-memory
// stages with K register bits; appends to out->stages / reg_ops / tile_ops.
void build_stages(const std::vector<DevOp>& ops, int L, int K, CompileResult* out, int* st0, int* nst);

// Arithmetic instructions per amplitude of a pass's stages (shared-memory and register ops)
// as the arithmetic policy's formulas count them: the ALU-work numerator of the roofline.
double stage_alu_per_amp(const CompileResult& cr, int st0, int nst);
// the same for one per-gate op
double op_alu_per_amp(Policy pol, const DevOp& op);
// arithmetic per amplitude a gate adds to a tile pass (register stages, tables shared by
// several diagonal gates): the compiler's estimate of what moving it elsewhere saves
double gate_tile_alu_per_amp(Policy pol, const HGate& g);

}  // namespace qs
