/*
 * qs.h -- C ABI of the GB300 (sm_103a) state-vector simulator library (libqs.so).
 *
 * The library implements the hot path of the Schroedinger-type simulator in
 * "Fast simulation of quantum algorithms using circuit optimization"
 * (arXiv 2010.09746): 1- and 2-qubit (and fused k-qubit) gates applied to a vector
 * of 2^n complex amplitudes, the qubit-order permutation instruction PermuteQubits,
 * and the compiler pass that inserts permutations so that most gates run without
 * "communication".  On one GPU the paper's local/global qubit split (Sec. 2) becomes
 * the split between the storage bits of a shared-memory tile and the others: a tile
 * pass applies every gate whose non-diagonal qubits sit in the tile in one HBM read
 * and one HBM write.
 *
 * Conventions (all calls):
 *  - Qubit q of a gate is a LOGICAL qubit.  Amplitude alpha_i, i = sum_q i_q 2^q, is
 *    stored at component j(i, sigma) = sum_q i_q 2^{sigma(q)} of the device vector
 *    (Sec. 2); sigma starts as the identity and changes only through qs_permute or
 *    plans that contain permutations.
 *  - Matrices are host memory owned by the caller, read during the call, row-major,
 *    complex entries as (re, im) pairs of doubles.  For a k-qubit matrix on qubits
 *    (q_0 .. q_{k-1}) the row/column index is r = sum_t b(q_t) 2^t (first listed qubit
 *    is the least significant bit).  Controlled gates list (control, target).
 *  - Calls that only enqueue GPU work are asynchronous on the state's stream; read-outs
 *    (qs_probabilities, qs_get_amplitudes, qs_norm) synchronise that stream.
 *  - Every call returns a qs_status; on failure qs_last_error() gives a thread-local
 *    message.  No call throws across the ABI.  Bad arguments return QS_EINVAL and leave
 *    the state unchanged.
 *  - Device memory comes from the allocator installed with qs_set_allocator, else from
 *    cudaMallocAsync on the state's stream.
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qs_state* qs_handle;   /* opaque, owned by the library */
typedef struct qs_plan* qs_plan_t;    /* opaque compiled circuit, owned by the library */

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

typedef enum {
  QS_OK = 0,
  QS_EINVAL = 1,       /* invalid argument (qubit out of range, duplicate qubits, ...) */
  QS_ENOMEM = 2,       /* device allocation failed */
  QS_ECUDA = 3,        /* a CUDA call failed */
  QS_ETIMEOUT = 4,     /* a bounded device-side wait ran out (status word set by a kernel) */
  QS_EBUSY = 5,        /* resource in use */
  QS_EUNSUPPORTED = 6, /* valid request this build does not implement */
  QS_ECANCELED = 7     /* a served request was cancelled before it ran (qs_server_cancel) */
} qs_status;

/* Arithmetic used for complex128 states (complex64 always computes in FP32). */
typedef enum {
  QS_ARITH_AUTO = 0,   /* QS_ARITH_DF for complex128 */
  QS_ARITH_DF = 1,     /* double-float (pairs of FP32) arithmetic, FP64 storage */
  QS_ARITH_F64 = 2     /* native FP64 arithmetic */
} qs_arith;

/* Gate kinds of qs_op.kind (definitions as in the standard literature):
 * H = (X+Z)/sqrt2, RZ(t) = exp(-i t Z/2), RX(t) = exp(-i t X/2), RY(t) = exp(-i t Y/2),
 * P(t) = diag(1, e^{it}), S = P(pi/2), T = P(pi/4), CP(t) = controlled P(t). */
enum {
  QS_OP_U1 = 0,   /* arbitrary 2x2, matrix at mats[mat .. mat+7] */
  QS_OP_H = 1, QS_OP_X = 2, QS_OP_Y = 3, QS_OP_Z = 4, QS_OP_S = 5, QS_OP_T = 6,
  QS_OP_RZ = 7, QS_OP_RX = 8, QS_OP_RY = 9, QS_OP_P = 10,
  QS_OP_CNOT = 11, QS_OP_CZ = 12, QS_OP_CP = 13,
  QS_OP_CU = 14,  /* controlled arbitrary 2x2, matrix at mats[mat .. mat+7] */
  QS_OP_SWAP = 15,
  QS_OP_U2 = 16,  /* arbitrary 4x4, 32 doubles at mats[mat ..] */
  QS_OP_UK = 17,  /* arbitrary 2^k x 2^k (k = nq <= 6), 2*4^k doubles at mats[mat ..] */
  QS_OP_RELABEL = 18  /* Emulated-SWAP (Appendix B): the two qubits exchange storage positions
                         in sigma, no amplitude moves; preceded by a SWAP it is the paper's
                         PermuteQubits of one transposition.  QS_MODE_PERGATE only. */
};

/* One gate of a circuit.  48 bytes, no padding. */
typedef struct {
  int32_t kind;    /* QS_OP_* */
  int32_t nq;      /* number of qubits used in q[] */
  int32_t q[6];    /* logical qubits */
  double param;    /* angle for RZ/RX/RY/P/CP */
  int64_t mat;     /* offset in doubles into the caller's matrix buffer, -1 if unused */
} qs_op;

/* Compilation modes of qs_compile / qs_run. */
typedef enum {
  QS_MODE_PERGATE = 0,  /* one strided-pair kernel launch per gate, no reordering */
  QS_MODE_PAPER = 1,    /* Algorithm 1 (Sec. 3) with m = tile bits: runs of local gates fused
                           into tile passes over storage bits [0, L), one local<->global
                           transposition per PermuteQubits, non-local gates per gate */
  QS_MODE_TILE = 2      /* tile passes over gathered bit sets: each pass picks the L storage
                           bits (the low `low_bits` always included) that let the most gates
                           run; equivalent to a multi-transposition permutation folded into
                           the pass's addressing, so no separate permutation pass is needed */
} qs_mode;

/* qs_compile_opts.flags.  QS_FLAG_FULL_RX: by default an uncontrolled RX held in registers
 * is applied in the cheaper tangent form, (I - i tan X) or (cot I - i X), with the dropped
 * cos / sin factors of a tile pass multiplied into one full-form RX of that pass (same result
 * up to rounding); this flag keeps every RX in full form.  QS_FLAG_NO_DENSE: never emit dense
 * tensor-core blocks (see qs_cost_model).  QS_FLAG_NO_FUSE: QS_MODE_TILE fuses, by default,
 * every run of single-qubit gates on one qubit with no multi-qubit gate on that qubit in
 * between (gate fusion, Sec. 1) when the run holds two or more non-diagonal gates, a general
 * one (neither RX nor X in form) or only diagonal ones: the run's product is applied as
 * diag . RX . diag (an exact identity for
 * every 2x2 unitary) just before the next multi-qubit gate on that qubit (or at the end);
 * the result equals the unfused
 * plan's up to rounding and the trace still lists every input gate once.  This flag turns
 * fusion off. */
enum { QS_FLAG_FULL_RX = 1, QS_FLAG_NO_DENSE = 2, QS_FLAG_NO_FUSE = 4 };

/* Cost of one launch of each kernel class for the plan's dtype,
 *   t [ms] = c[0] + c[1] * (algorithmic HBM bytes) + c[2] * (counted arithmetic instructions),
 * the least-squares model that tuning.py fits to CUDA-event kernel times (Sec. 3 of the paper
 * suggests compiler passes that use the simulator's measured benchmarks).  The compiler uses
 * it in QS_MODE_TILE to decide, before each tile pass, whether the gates that are ready on
 * storage bits 0..5 alone should instead run as one dense 64 x 64 block on the tensor cores
 * (complex64, n >= 12): it does so when the block's predicted time is below the tile-pass
 * time those gates are predicted to cost.  Every plan reports the model's prediction of its
 * own execution time (qs_plan_stats.predicted_ms). */
typedef struct {
  double tile[3];      /* tile pass */
  double gate[3];      /* per-gate kernel */
  double permute[3];   /* permutation kernel */
  double dense[3];     /* dense 6-qubit block on the tensor cores */
} qs_cost_model;

/* The model the compiler uses when qs_compile_opts.cost is NULL, for plans of this dtype and
 * arithmetic (coefficients measured on GB300). */
qs_status qs_default_cost_model(qs_dtype dtype, qs_arith arith, qs_cost_model* out);

typedef struct {
  int32_t mode;       /* qs_mode */
  int32_t dtype;      /* qs_dtype of the states the plan will run on */
  int32_t arith;      /* qs_arith */
  int32_t tile_bits;  /* L: amplitudes per tile = 2^L, 1..14; 0 = default for the dtype.
                         QS_MODE_PAPER: the number m of local qubits, 1..n (runs of local
                         gates execute gate by gate when m > 14) */
  int32_t low_bits;   /* storage bits always inside a tile (contiguous segment = 2^low_bits
                         amplitudes); 0 = default */
  int32_t max_ops;    /* cap on gates per tile pass, 0 = none */
  int32_t scoring;    /* Algorithm 1 candidate score: 0 = closure (default), 1 = frontier */
  int32_t flags;      /* QS_FLAG_* bits; others must be 0 */
  int32_t reg_bits;   /* tile bits each thread holds in registers in a register stage (2^reg_bits
                         amplitudes per thread), 1..5 (complex128 1..4); 0 = default (4 for
                         complex128, 5 for complex64) */
  int32_t renorm_every; /* periodic renormalisation (no counterpart in the paper): after every
                           `renorm_every` kernels of the plan (tile passes, per-gate kernels,
                           permutations) the state is divided by the square root of its FP64
                           norm, as by qs_renormalize; 0 = never.  Each costs one read for the
                           norm and one read + write for the scaling. */
  const qs_cost_model* cost; /* kernel cost model; NULL = the library's defaults (GB300, measured) */
} qs_compile_opts;

typedef struct {
  int64_t n_gates;        /* gates in the input circuit */
  int64_t n_passes;       /* tile passes */
  int64_t n_pergate;      /* gates executed by per-gate kernels */
  int64_t n_permutes;     /* PermuteQubits instructions (QS_MODE_PAPER: local<->global
                             transpositions); see n_permute_kernels */
  int64_t n_comm_gates;   /* QS_MODE_PAPER: gates executed non-locally */
  double hbm_bytes;       /* algorithmic HBM bytes of one execution (reads + writes) */
  double alu_instr;       /* arithmetic instructions of one execution as the arithmetic's
                             formulas count them (FP32 FMA-pipe instructions for complex64 and
                             double-float, DFMA for native FP64), all amplitudes */
  double compile_ms;      /* host time spent compiling */
  int64_t n_dense;        /* dense 6-qubit blocks on the tensor cores (QS_MODE_TILE, complex64) */
  double predicted_ms;    /* the cost model's prediction of one execution */
  int64_t n_permute_kernels; /* permutation kernel launches: a PermuteQubits right after a tile
                                pass is folded into that pass's store (the pass writes under the
                                new sigma to a second buffer) whenever the local qubit's storage
                                bit is not one of the pass's contiguous segment bits */
  int64_t n_fused;        /* QS_MODE_TILE: input gates absorbed into fused single-qubit products
                             (see QS_FLAG_NO_FUSE); 0 otherwise */
} qs_plan_stats;

/* Per-kernel-class timing collected while profiling is on (qs_set_profiling). */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;        /* sum of CUDA-event durations on the state's stream */
  double bytes;           /* algorithmic HBM bytes of those launches */
  double alu;             /* arithmetic instructions of those launches (see qs_plan_stats) */
} qs_kernel_stat;

/* ---- library ------------------------------------------------------------------------ */

/* Thread-local description of the last failure of the calling thread ("" if none). */
const char* qs_last_error(void);

/* Library version string. */
const char* qs_version(void);

/* Install a device allocator used by every later allocation: alloc(bytes, ctx, stream)
 * returns a device pointer or NULL; free(ptr, bytes, ctx, stream) releases it.  Pass
 * NULLs to restore the default (cudaMallocAsync/cudaFreeAsync).  The callbacks must stay
 * valid until the last state / plan is destroyed. */
qs_status qs_set_allocator(void* (*alloc_fn)(size_t bytes, void* ctx, void* stream),
                           void (*free_fn)(void* ptr, size_t bytes, void* ctx, void* stream),
                           void* ctx);

/* ---- states (Sec. 2: the 2^n-amplitude vector and its qubit permutation sigma) ------ */

/* Allocate a state of n qubits (1 <= n <= 36) on the current device, set to |0...0>
 * with sigma = identity (synchronises the legacy default stream).  Work is enqueued on the
 * default stream until qs_set_stream. */
qs_status qs_create(int n, qs_dtype dtype, qs_handle* out);
/* The same, with the allocation and initialisation enqueued on `stream` (cudaStream_t),
 * which becomes the state's stream; returns without waiting for the device. */
qs_status qs_create_async(int n, qs_dtype dtype, void* stream, qs_handle* out);
qs_status qs_destroy(qs_handle h);

/* Stream (cudaStream_t) on which all later work of this state is enqueued. */
qs_status qs_set_stream(qs_handle h, void* stream);

/* Arithmetic for complex128 gate application through the qs_apply_* calls. */
qs_status qs_set_arith(qs_handle h, qs_arith arith);

/* Record CUDA events around every kernel launch of this state (per-kernel-class totals
 * in qs_get_kernel_stats).  Costs two events per launch. */
qs_status qs_set_profiling(qs_handle h, int on);
qs_status qs_get_kernel_stats(qs_handle h, qs_kernel_stat* out, int max, int* count);
qs_status qs_reset_kernel_stats(qs_handle h);

/* Re-initialise to |0...0> and sigma = identity (state preparation, Sec. 2). */
qs_status qs_reset(qs_handle h);

/* n, dtype, the device address of the amplitude vector and its size in bytes (any output
 * may be NULL).  The address is valid until the next call that moves the vector: a
 * permutation (qs_permute, a plan containing permutation steps, qs_apply_dense on the tensor
 * path when it permutes first) writes into a second buffer of the same size and swaps the
 * two.  That second buffer is allocated by the first such call and kept until qs_destroy,
 * so a state that has permuted holds 2x `bytes` of device memory. */
qs_status qs_get_info(qs_handle h, int* n, qs_dtype* dtype, void** device_ptr, size_t* bytes);
qs_status qs_sync(qs_handle h);

/* ---- gates (Sec. 2: arbitrary 1-qubit gates, controlled 1-qubit gates) ------------- */

/* Arbitrary 1-qubit gate U (8 doubles) on logical qubit q: for every amplitude pair
 * differing only in qubit q, (a0, a1) <- U (a0, a1). */
qs_status qs_apply_1q(qs_handle h, const double* U, int q);

/* Arbitrary 2-qubit gate U (32 doubles, r = b(q0) + 2 b(q1)) on logical qubits q0 != q1. */
qs_status qs_apply_2q(qs_handle h, const double* U, int q0, int q1);

/* Controlled 1-qubit gate: U applied to qubit t on the amplitudes whose qubit c is 1
 * (CNOT is U = X). */
qs_status qs_apply_controlled(qs_handle h, const double* U, int c, int t);

/* Dense k-qubit gate (1 <= k <= 6, 2*4^k doubles) on distinct logical qubits[0..k-1].
 * Fusing gates into such blocks is the prior work the paper builds on (Sec. 1).  Two
 * engines (qs_set_dense_path): the strided kernel on the CUDA cores (every dtype), and for
 * complex64 states with n >= 12 the tensor-core kernel, which applies the block to storage
 * bits 0..5 as one real 128 x 128 matrix product per row of 64 amplitudes (TF32 operands
 * with a three-term split, FP32 accumulation: complex64 accuracy).  If the qubits are not
 * on storage bits 0..k-1 the tensor path first permutes the state so that qubits[t] is on
 * storage bit t (one permutation kernel, Sec. 2 PermuteQubits; sigma changes). */
qs_status qs_apply_dense(qs_handle h, const double* U, int k, const int* qubits);

typedef enum {
  QS_DENSE_AUTO = 0,        /* tensor cores for complex64 when k >= 5 with the qubits already on
                               storage bits 0..k-1, or k = 6 (after a permutation); else CUDA cores */
  QS_DENSE_CUDA_CORES = 1,  /* always the strided CUDA-core kernel */
  QS_DENSE_TENSOR = 2       /* always the tensor-core kernel (QS_EINVAL unless complex64, n >= 12) */
} qs_dense_path;

/* Engine for this state's later qs_apply_dense calls (default QS_DENSE_AUTO). */
qs_status qs_set_dense_path(qs_handle h, int path);

/* ---- qubit permutation (Sec. 2 PermuteQubits; Appendix A) -------------------------- */

/* PermuteQubits(sigma'): perm[q] is the new storage bit of logical qubit q (a
 * permutation of 0..n-1, else QS_EINVAL).  Rewrites the vector so that alpha_i moves
 * from j(i, sigma) to j(i, sigma'); a pure move, bit-exact.  Uses a scratch vector the
 * size of the state unless sigma' differs from sigma only inside one tile. */
qs_status qs_permute(qs_handle h, const int* perm);
/* Current sigma: perm_out[q] = storage bit of logical qubit q (n ints). */
qs_status qs_get_permutation(qs_handle h, int* perm_out);

/* ---- circuits and the compiler pass (Sec. 3, Algorithm 1) -------------------------- */

/* Compile n-qubit circuit `ops` (matrix data in `mats`, nmats doubles) for states whose
 * permutation is currently sigma0 (NULL = identity).  opts NULL = defaults (QS_MODE_TILE,
 * complex128).  The plan holds copies of everything it needs, on host and device. */
qs_status qs_compile(int n, const qs_op* ops, size_t nops, const double* mats, size_t nmats,
                     const int* sigma0, const qs_compile_opts* opts, qs_plan_t* out);
/* Release a plan.  Never waits for the device: device buffers still needed by executions
 * enqueued earlier are released later, once those executions have completed (checked
 * without blocking whenever a plan is compiled or destroyed). */
qs_status qs_plan_destroy(qs_plan_t p);
qs_status qs_plan_get_stats(qs_plan_t p, qs_plan_stats* out);
/* sigma after the plan has run (n ints). */
qs_status qs_plan_final_permutation(qs_plan_t p, int* perm_out);

/* The schedule the compiler emitted: entry i is (kinds[i], values[i]) with
 * kind 0 = gate run locally / inside a tile pass (value = gate index), 1 = gate run by the
 * per-gate kernel as a non-local gate (QS_MODE_PAPER), 2 = permutation exchanging logical
 * qubits l and g (value = 64 l + g, QS_MODE_PAPER), 3 and 4 = start of a tile pass whose
 * storage-bit set is (value of 3) | (value of 4) << 31 (QS_MODE_TILE), 5 = start of a dense
 * tensor-core block on storage bits 0..5 fusing the next `value` gates (QS_MODE_TILE).  Up to
 * `max` entries are written; *count gets the total.  Empty for QS_MODE_PERGATE. */
qs_status qs_plan_get_trace(qs_plan_t p, int32_t* kinds, int32_t* values, size_t max, size_t* count);

/* Enqueue the plan on the state's stream.  The state must have the plan's n and dtype and
 * the permutation the plan was compiled for; afterwards sigma is the plan's final one.
 * Complex128 with double-float arithmetic: between consecutive tile passes of the plan the
 * state buffer holds an internal double-float form (four floats per element); it holds
 * binary64 again once the plan's work on the stream has completed, which is when any read
 * through this API or the device pointer is ordered.  A plan whose execution failed (for
 * example QS_ETIMEOUT) leaves the state undefined. */
qs_status qs_execute(qs_handle h, qs_plan_t p);

/* qs_compile + qs_execute + qs_plan_destroy; asynchronous like qs_execute. */
qs_status qs_run(qs_handle h, const qs_op* ops, size_t nops, const double* mats, size_t nmats,
                 const qs_compile_opts* opts);

/* ---- batches of independent circuits ----------------------------------------------- *
 * Many small circuits (each its own state) run together: every circuit is compiled as by
 * qs_compile in QS_MODE_TILE, and "wave" w -- pass w of every circuit that has one -- is one
 * persistent kernel launch over all those passes' tiles.  After the first (eager) run the
 * sequence init -> waves -> per-circuit norms is replayed from a captured CUDA graph when a
 * non-default stream is set.  A circuit's amplitudes are bitwise those of a solo qs_execute
 * with the same options.  opts->renorm_every must be 0 (QS_EINVAL otherwise). */
typedef struct qs_batch* qs_batch_t;

typedef struct {
  int64_t n_circuits;
  int64_t n_gates;
  int64_t n_passes;       /* tile passes over all circuits */
  int64_t n_waves;        /* launches per run (plus init and norms) */
  double state_bytes;     /* device bytes of all states */
  double hbm_bytes;       /* algorithmic bytes of one run's passes */
  double alu_instr;       /* arithmetic instructions of one run's passes (see qs_plan_stats) */
  double compile_ms;
} qs_batch_stats;

/* count circuits; circuit i has n[i] qubits (1..30) and the ops ops[op_offsets[i] ..
 * op_offsets[i+1]) whose matrix offsets index `mats`.  opts: mode must be QS_MODE_TILE (or
 * opts NULL: complex64, defaults); tile_bits is capped at each circuit's n. */
qs_status qs_batch_create(int count, const int* n, const qs_op* ops, const int64_t* op_offsets,
                          const double* mats, size_t nmats, const qs_compile_opts* opts, qs_batch_t* out);
qs_status qs_batch_set_stream(qs_batch_t b, void* stream);
/* 1 (default) = replay a captured graph from the second run on a non-default stream. */
qs_status qs_batch_set_graph(qs_batch_t b, int on);
/* Enqueue one run: every state to |0...0>, every circuit, every norm.  Asynchronous. */
qs_status qs_batch_run(qs_batch_t b);
/* Wait for the batch's stream; QS_ETIMEOUT if a device-side wait expired. */
qs_status qs_batch_sync(qs_batch_t b);
/* FP64 norm of every state after the last run (count doubles, host). */
qs_status qs_batch_norms(qs_batch_t b, double* out);
/* Amplitudes first .. first+count-1 of circuit i (storage = logical order), host memory. */
qs_status qs_batch_get_amplitudes(qs_batch_t b, int i, void* out, uint64_t first, uint64_t count);
qs_status qs_batch_get_stats(qs_batch_t b, qs_batch_stats* out);
qs_status qs_batch_destroy(qs_batch_t b);

/* ---- serving: continuous batching (no counterpart in the paper) --------------------- *
 * A server runs independent requests (an n-qubit circuit and a dtype, each simulated from
 * |0...0>) as they arrive.  Host threads compile every request's plan (QS_MODE_TILE) as
 * soon as it is submitted; one admission thread starts a compiled request as soon as one of
 * the server's slots (each its own CUDA stream) and its state's bytes within the memory
 * budget are free, without waiting for the requests already on the GPU, so work of
 * different requests overlaps on the device.  Small requests (n <= batch_small_n) that are
 * ready together share one slot as one batch (persistent tile-pass launches over all their
 * states, as qs_batch_*).  Every request runs the same per-tile code on its own state
 * whatever else is in flight, so its result is bitwise its result alone.  A finished
 * request leaves the FP64 norm and its first amplitudes in host memory until taken.
 * Device memory of the server's states comes from cudaMallocAsync on the slot streams, not
 * from an allocator installed with qs_set_allocator. */
typedef struct qs_server* qs_server_t;

typedef struct {
  int32_t slots;           /* requests (or batches) on the GPU at once, one stream each; 0 = 8 */
  int32_t compile_threads; /* host threads compiling plans; 0 = 4 */
  int64_t mem_budget;      /* device bytes for resident states; 0 = 3/4 of the free memory */
  int32_t readout;         /* amplitudes kept per request: the first min(2^n, readout); 0 = 256 */
  int32_t batch_small_n;   /* requests with n <= this that are ready together share a slot; 0 = 16,
                              negative = never */
  int32_t batch_max;       /* most requests sharing one slot; 0 = 64 */
  int32_t order;           /* admission order: 0 = arrival, 1 = least estimated device work first */
  int32_t max_wait_ms;     /* order 1: a request that has waited this long goes first; 0 = 1000 */
  int32_t tile_bits;       /* compile option of every request (0 = the dtype's default) */
  int32_t reserved;        /* must be 0 */
} qs_server_opts;

typedef struct {
  int64_t id;
  int32_t status;          /* qs_status of the request (compile or device failure) */
  int32_t n;
  int32_t dtype;
  int32_t batched;         /* 1 if it shared a slot with other requests */
  double norm;             /* FP64 norm of the final state */
  double t_submit_s, t_admit_s, t_done_s;   /* server clock (seconds since qs_server_create) */
  uint64_t amplitudes;     /* amplitudes kept for qs_server_take */
  char error[128];         /* failure text, "" if none */
} qs_server_result;

typedef struct {
  int64_t submitted, completed, in_flight, waiting, batches, batched_requests, peak_in_flight;
  double peak_mem_bytes, mem_used_bytes;
  double now_s;            /* server clock */
} qs_server_stats;

/* Start a server on the current device (opts NULL = defaults). */
qs_status qs_server_create(const qs_server_opts* opts, qs_server_t* out);
/* Queue one request (1 <= n <= 30; ops / mats as qs_compile, copied); *id identifies it.
 * Returns at once; QS_EINVAL if the state alone exceeds the memory budget. */
qs_status qs_server_submit(qs_server_t s, int n, qs_dtype dtype, const qs_op* ops, size_t nops, const double* mats,
                           size_t nmats, int64_t* id);
/* Up to `max` finished requests not reported before (each reported once), waiting up to
 * timeout_ms for the first one when none is ready (0 = do not wait). */
qs_status qs_server_poll(qs_server_t s, qs_server_result* out, int max, int* count, int timeout_ms);
/* Copy the first `count` kept amplitudes of finished request `id` (interleaved (re, im) in
 * its dtype) into HOST memory and release the result. */
qs_status qs_server_take(qs_server_t s, int64_t id, void* amps, uint64_t count);
/* Withdraw a request that has not started on the GPU: it finishes at once with status
 * QS_ECANCELED (reported by qs_server_poll like any result).  QS_EBUSY if it is already on
 * the GPU or finished (taken or not), QS_EINVAL for an id this server never issued. */
qs_status qs_server_cancel(qs_server_t s, int64_t id);
qs_status qs_server_get_stats(qs_server_t s, qs_server_stats* out);
/* Finish every submitted request, then stop the threads and release everything (results
 * not taken are dropped). */
qs_status qs_server_destroy(qs_server_t s);

/* ---- read-outs (Sec. 2: measurement) ------------------------------------------------ */

enum { QS_ORDER_LOGICAL = 0, QS_ORDER_STORAGE = 1 };

/* p[i] = |alpha_i|^2 for all 2^n i into HOST memory `out` (logical order: index i;
 * storage order: index j).  Synchronises the stream. */
qs_status qs_probabilities(qs_handle h, double* out, int order);

/* `count` amplitudes starting at index `first` (logical or storage order) into HOST memory
 * `out`, as interleaved (re, im) in the state's dtype (float for complex64, double for
 * complex128).  Synchronises the stream. */
qs_status qs_get_amplitudes(qs_handle h, void* out, uint64_t first, uint64_t count, int order);

/* Overwrite the whole vector from HOST memory (storage order under the current sigma,
 * interleaved, the state's dtype); for checkpoint / restore and tests. */
qs_status qs_set_amplitudes(qs_handle h, const void* in);

/* Copy storage elements first .. first+count-1 between the state and DEVICE memory `dev`
 * (interleaved, the state's dtype): to_state = 0 reads the state into dev, 1 writes dev into
 * the state.  Enqueued on the state's stream, which the call synchronises before returning
 * (so another stream or a communication library may use `dev` at once).  Used to exchange
 * halves of a state slice between processes (global-qubit sharding, Sec. 2 / Appendix A). */
qs_status qs_copy_range_device(qs_handle h, void* dev, uint64_t first, uint64_t count, int to_state);

/* The full matrix of one gate as the library defines it: 2^k x 2^k complex entries, row-major,
 * (re, im) pairs, row / column r = sum_t b(op->q[t]) 2^t, written to U_out (room for 2 * 4^6
 * doubles); *k_out = k.  op and mats as for qs_compile (n bounds the qubit indices). */
qs_status qs_gate_matrix(int n, const qs_op* op, const double* mats, size_t nmats, double* U_out, int* k_out);

/* sum_i |alpha_i|^2 accumulated in FP64 with a fixed reduction order (deterministic).
 * Synchronises the stream. */
qs_status qs_norm(qs_handle h, double* out);

/* ---- precision helpers (no counterpart in the paper) ------------------------------- *
 * A state stored as complex64 drifts from unit norm by rounding, about 2^-24 relative per
 * gate application; these calls measure that drift against another state and remove it,
 * with every reduction in FP64. */

/* <a|b> = sum_i conj(alpha_i) beta_i over logical indices i, accumulated in FP64 with a
 * fixed reduction order; out[0] = real part, out[1] = imaginary part (HOST memory).  The
 * two states may have different dtypes (complex64 against complex128 is the precision
 * study) but must have the same n and the same sigma (else QS_EINVAL: permute one of them
 * first).  Runs on a's stream after b's stream has reached the point of the call (an
 * event), uses a temporary device buffer of 1216 * 16 + 16 bytes from the allocator, and
 * synchronises a's stream. */
qs_status qs_inner(qs_handle a, qs_handle b, double* out);

/* psi <- psi / sqrt(<psi|psi>): the FP64 norm as qs_norm computes it, then an in-place
 * scaling by a factor read on the device (complex128: each component multiplied in FP64;
 * complex64: by the factor rounded once to float).  Enqueued on the state's stream.  If
 * norm_out is not NULL the call synchronises the stream and stores the norm before the
 * scaling there (HOST memory); with NULL it does not synchronise.  A norm that is zero or
 * not finite leaves the state unchanged. */
qs_status qs_renormalize(qs_handle h, double* norm_out);

/* ---- allocation-free read-out (no counterpart in the paper) ------------------------- *
 *
 * FP64 norm sum_j |psi[j]|^2 of a state vector the caller owns, written to *out_dev (a
 * device double), computed by the same fixed-order reduction as qs_norm, so the two agree
 * bit for bit.  For callers that may not allocate device memory: a host program that has
 * already divided the whole GPU among its own buffers and allows no further allocation, or
 * a latency-critical loop that must not enter the allocator.  The call allocates nothing:
 * the reduction's 1216 partial sums live in one fixed device array (9.5 KiB) that every GPU
 * loading the library keeps until the process exits.
 *   psi      device pointer to 2^n interleaved (re, im) elements of `dtype`
 *   n        1..36; larger states are rejected with QS_EINVAL (the limit of the library)
 *   out_dev  device pointer to one double; written asynchronously on `stream`
 *   stream   cudaStream_t (NULL = the legacy default stream)
 * The first call on each device (and again the first after the device's context changed,
 * e.g. after cudaDeviceReset) looks up the device address of the fixed array
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture begins.  All calls share the one array and each call overwrites all of it, so
 * calls whose kernels overlap on the GPU (different streams, no ordering) race and give
 * wrong results; calls on one stream are safe.  Asynchronous: synchronise the stream
 * before reading *out_dev. */
qs_status qs_norm_noalloc(const void* psi, int n, qs_dtype dtype, double* out_dev, void* stream);

/* ---- self-test of the bounded waits (no counterpart in the paper) ------------------ *
 * Every kernel that waits on an mbarrier (bulk copies, tensor-core commits) gives up after
 * a %globaltimer limit and reports QS_ETIMEOUT instead of hanging.  This call exercises that
 * path on purpose: one CTA waits on an mbarrier nothing arrives on, with a limit of limit_us
 * microseconds (1 .. 1000000), and writes its verdict to *device_status (HOST memory):
 * QS_ETIMEOUT when the wait expired as designed.  Synchronous on the default stream;
 * returns QS_OK unless a CUDA call failed (QS_ECUDA) or the arguments are invalid. */
qs_status qs_selftest_bounded_wait(int limit_us, int* device_status);

#ifdef __cplusplus
}
#endif
#endif /* QS_H */
