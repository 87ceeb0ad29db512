// C ABI (include/qs.h): states, plans, device memory, streams, read-outs, profiling.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.h"

using namespace qs;

namespace {

thread_local std::string g_err;

qs_status fail(qs_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
qs_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA;
}
#define CUDA_TRY(call, where)                  \
  do {                                         \
    cudaError_t _e = (call);                   \
    if (_e != cudaSuccess) return cuda_fail(_e, where); \
  } while (0)

}  // namespace

namespace qs {

// ---- allocator -----------------------------------------------------------------------------
namespace {
void* (*g_alloc)(size_t, void*, void*) = nullptr;
void (*g_free)(void*, size_t, void*, void*) = nullptr;
void* g_alloc_ctx = nullptr;
}  // namespace

namespace {
thread_local bool t_native_alloc = false;
}  // namespace

void set_thread_native_alloc(bool on) { t_native_alloc = on; }
bool dev_alloc_native() { return t_native_alloc || g_alloc == nullptr; }

void* dev_alloc(size_t bytes, cudaStream_t s) { return dev_alloc_as(bytes, s, dev_alloc_native()); }

void* dev_alloc_as(size_t bytes, cudaStream_t s, bool native) {
  if (bytes == 0) bytes = 256;
  if (!native && g_alloc) return g_alloc(bytes, g_alloc_ctx, (void*)s);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free_as(void* p, size_t bytes, cudaStream_t s, bool native) {
  if (!p) return;
  if (!native && g_free) {
    g_free(p, bytes == 0 ? 256 : bytes, g_alloc_ctx, (void*)s);
    return;
  }
  cudaFreeAsync(p, s);
}

void dev_free(void* p, size_t bytes, cudaStream_t s) { dev_free_as(p, bytes, s, dev_alloc_native()); }

Policy policy_for(qs_dtype dt, qs_arith a) {
  if (dt == QS_C64) return POL_F32;
  return a == QS_ARITH_F64 ? POL_F64 : POL_DF;
}

}  // namespace qs

namespace qs {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace qs

namespace {

cudaEvent_t get_event(qs_state* h) {
  if (!h->free_events.empty()) {
    cudaEvent_t e = h->free_events.back();
    h->free_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// run `launch` on the state's stream, bracketed by events when profiling
template <class F>
cudaError_t timed(qs_state* h, const char* name, double bytes, F&& launch, double alu = 0.0) {
  if (!h->profiling) return launch();
  KernelRecord r;
  r.name = name;
  r.bytes = bytes;
  r.alu = alu;
  r.e0 = get_event(h);
  r.e1 = get_event(h);
  cudaEventRecord(r.e0, h->stream);
  cudaError_t e = launch();
  cudaEventRecord(r.e1, h->stream);
  h->pending.push_back(r);
  return e;
}

void collect_stats(qs_state* h) {
  if (h->pending.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (KernelRecord& r : h->pending) {
    float ms = 0;
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    qs_kernel_stat* st = nullptr;
    for (auto& s : h->stats)
      if (r.name == s.name) st = &s;
    if (!st) {
      h->stats.emplace_back();
      st = &h->stats.back();
      memset(st, 0, sizeof(*st));
      strncpy(st->name, r.name.c_str(), sizeof(st->name) - 1);
    }
    st->launches++;
    st->total_ms += ms;
    st->bytes += r.bytes;
    st->alu += r.alu;
    h->free_events.push_back(r.e0);
    h->free_events.push_back(r.e1);
  }
  h->pending.clear();
}

qs_status check_status(qs_state* h) {
  int st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, h->status_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "status read");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "stream sync");
  if (st != 0) {
    int zero = 0;
    cudaMemcpyAsync(h->status_dev, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream);
    cudaStreamSynchronize(h->stream);
    return fail((qs_status)st, "a device-side wait timed out");
  }
  return QS_OK;
}

bool valid_perm(int n, const int* p) {
  std::vector<char> seen(n, 0);
  for (int q = 0; q < n; q++) {
    if (p[q] < 0 || p[q] >= n || seen[p[q]]) return false;
    seen[p[q]] = 1;
  }
  return true;
}

const char* step_name(const Step& s, Policy pol) {
  if (s.kind == ST_PASS) return pol == POL_F32 ? "tile_pass_c64" : (pol == POL_DF ? "tile_pass_c128_df" : "tile_pass_c128_f64");
  if (s.kind == ST_PERMUTE) return "permute";
  if (s.kind == ST_DENSE) return "dense_mma_c64";
  return pol == POL_F32 ? "gate_c64" : (pol == POL_DF ? "gate_c128_df" : "gate_c128_f64");
}

// apply one lowered gate through the per-gate kernel
qs_status apply_hgate(qs_state* h, const HGate& g) {
  Pool pool;
  std::vector<DevOp> ops;
  LowerCtx ctx;
  ctx.sigma = h->sigma.data();
  ctx.tile = false;
  if (!lower_gate(g, ctx, pool, ops)) return fail(QS_EINVAL, "gate could not be lowered");
  const Policy pol = policy_for(h->dtype, h->arith);
  std::vector<unsigned char> ser = pool.serialise(pol);
  if (ser.size() > h->gate_pool_bytes) {
    dev_free_as(h->gate_pool, h->gate_pool_bytes, h->stream, h->native_alloc);
    h->gate_pool_bytes = std::max<size_t>(ser.size(), 64 * 1024);
    h->gate_pool = dev_alloc_as(h->gate_pool_bytes, h->stream, h->native_alloc);
    if (!h->gate_pool) return fail(QS_ENOMEM, "gate matrix buffer allocation failed");
  }
  if (!ser.empty())
    CUDA_TRY(cudaMemcpyAsync(h->gate_pool, ser.data(), ser.size(), cudaMemcpyHostToDevice, h->stream), "matrix upload");
  for (const DevOp& o : ops) {
    Step s;
    s.kind = ST_GATE;
    CUDA_TRY(timed(h, step_name(s, pol), 0.0, [&] { return launch_gate(pol, h->psi, h->n, o, h->gate_pool, h->stream); }),
             "gate launch");
  }
  return QS_OK;
}

qs_status ensure_scratch(qs_state* h) {
  if (h->scratch) return QS_OK;
  h->scratch = dev_alloc_as(h->bytes, h->stream, h->native_alloc);
  if (!h->scratch) return fail(QS_ENOMEM, "permutation scratch allocation failed");
  return QS_OK;
}

qs_status do_permute(qs_state* h, const std::vector<int>& src_of, const std::vector<int>& new_sigma, double bytes) {
  qs_status st = ensure_scratch(h);
  if (st != QS_OK) return st;
  CUDA_TRY(timed(h, "permute", bytes,
                 [&] { return launch_permute(h->scratch, h->psi, h->n, h->store_bytes, src_of.data(), h->stream); }),
           "permute launch");
  std::swap(h->psi, h->scratch);
  h->sigma = new_sigma;
  return QS_OK;
}

// Which engine QS_DENSE_AUTO picks for a complex64 block of k qubits (the CUDA-core
// kernel is arithmetic-bound from k = 5 on; the tensor-core kernel is bandwidth-bound for
// every k, and worth a permutation pass first only at k = 6).
bool dense_auto_tensor(int k, bool low) { return low ? k >= 5 : k >= 6; }

qs_status apply_dense_tensor(qs_state* h, const double* U, int k, const int* qubits, bool low) {
  if (!low) {   // PermuteQubits: qubits[t] -> storage bit t, displaced qubits take the freed bits
    std::vector<int> ns = h->sigma;
    for (int t = 0; t < k; t++) {
      const int q = qubits[t];
      if (ns[q] == t) continue;
      for (int q2 = 0; q2 < h->n; q2++)
        if (ns[q2] == t) {
          std::swap(ns[q], ns[q2]);
          break;
        }
    }
    std::vector<int> src_of(h->n);
    for (int q = 0; q < h->n; q++) src_of[ns[q]] = h->sigma[q];
    qs_status st = do_permute(h, src_of, ns, 2.0 * (double)h->bytes);
    if (st != QS_OK) return st;
  }
  int bits[6];
  for (int t = 0; t < k; t++) bits[t] = h->sigma[qubits[t]];
  std::vector<float> w(2 * 128 * 128);
  dense_mma_weights(U, k, bits, w.data());
  if (!h->dense_w) {
    h->dense_w = (float*)dev_alloc_as(kDenseWBytes, h->stream, h->native_alloc);
    if (!h->dense_w) return fail(QS_ENOMEM, "dense weight buffer allocation failed");
  }
  if (!h->num_sms) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "device query");
    CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  }
  CUDA_TRY(cudaMemcpyAsync(h->dense_w, w.data(), kDenseWBytes, cudaMemcpyHostToDevice, h->stream), "weight upload");
  CUDA_TRY(timed(h, "dense_mma_c64", 2.0 * (double)h->bytes,
                 [&] { return launch_dense_mma(h->psi, h->n, h->dense_w, h->status_dev, h->num_sms, h->stream); }),
           "dense MMA launch");
  return QS_OK;
}

// FP64 norm into norm_buf[np], then scale by it on the device (no host round trip).
qs_status renormalize(qs_state* h) {
  const int np = norm_num_partials();
  CUDA_TRY(timed(h, "norm", (double)h->bytes,
                 [&] { return launch_norm_partials(h->psi, h->n, h->dtype == QS_C128, h->norm_buf, np, h->stream); }),
           "norm partials");
  CUDA_TRY(launch_norm_final(h->norm_buf, np, h->norm_buf + np, h->stream), "norm final");
  CUDA_TRY(timed(h, "scale", 2.0 * (double)h->bytes,
                 [&] { return launch_scale(h->psi, h->n, h->dtype == QS_C128, h->norm_buf + np, h->stream); }),
           "scale launch");
  return QS_OK;
}

// Device buffers of destroyed plans whose last executions may still be running.  They are
// released once every recorded event has completed, checked (without blocking) whenever a
// plan is compiled or destroyed; a plan's destruction never waits for the device.
struct DeferredFree {
  std::vector<std::pair<void*, size_t>> bufs;
  std::vector<cudaEvent_t> events;
  bool native = true;   // allocated by cudaMallocAsync (else by the installed allocator)
};
std::mutex g_deferred_mu;
std::vector<DeferredFree> g_deferred;

bool events_done(const std::vector<cudaEvent_t>& evs) {
  for (cudaEvent_t e : evs) {
    const cudaError_t q = cudaEventQuery(e);
    if (q == cudaErrorNotReady) return false;
    if (q != cudaSuccess) cudaGetLastError();   // an event that failed is treated as finished
  }
  return true;
}

void release_deferred(DeferredFree& d) {
  for (auto& b : d.bufs) dev_free_as(b.first, b.second, nullptr, d.native);
  for (cudaEvent_t e : d.events) cudaEventDestroy(e);
  d.bufs.clear();
  d.events.clear();
}

void reap_deferred() {
  std::vector<DeferredFree> ready;
  {
    std::lock_guard<std::mutex> lk(g_deferred_mu);
    size_t w = 0;
    for (size_t r = 0; r < g_deferred.size(); r++) {
      if (events_done(g_deferred[r].events)) ready.push_back(std::move(g_deferred[r]));
      else g_deferred[w++] = std::move(g_deferred[r]);
    }
    g_deferred.resize(w);
  }
  for (DeferredFree& d : ready) release_deferred(d);
}

}  // namespace

namespace qs {

qs_status note_plan_use(qs_plan* p, cudaStream_t s) {
  cudaEvent_t ev = nullptr;
  for (auto& u : p->uses)
    if (u.first == s) ev = u.second;
  if (!ev) {
    CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "plan event");
    p->uses.push_back({s, ev});
  }
  CUDA_TRY(cudaEventRecord(ev, s), "plan event record");
  return QS_OK;
}


qs_status state_create_on(int n, qs_dtype dtype, cudaStream_t stream, qs_state** out) {
  *out = nullptr;
  if (n < 1 || n > kMaxQubits) return fail(QS_EINVAL, "n must be in [1, 36]");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "unknown dtype");
  qs_state* h = new qs_state();
  h->n = n;
  h->dtype = dtype;
  h->stream = stream;
  h->native_alloc = dev_alloc_native();
  h->store_bytes = dtype == QS_C128 ? 16 : 8;
  h->bytes = (size_t)h->store_bytes << n;
  h->sigma.resize(n);
  for (int q = 0; q < n; q++) h->sigma[q] = q;
  h->psi = dev_alloc(h->bytes, stream);
  h->status_dev = (int*)dev_alloc(256, stream);
  h->norm_buf = (double*)dev_alloc(sizeof(double) * (norm_num_partials() + 1), stream);
  if (!h->psi || !h->status_dev || !h->norm_buf) {
    const size_t b = h->bytes;
    qs_destroy(h);
    return fail(QS_ENOMEM, "state allocation failed (" + std::to_string(b) + " bytes)");
  }
  cudaError_t e = cudaMemsetAsync(h->status_dev, 0, 256, stream);
  if (e == cudaSuccess) e = launch_init_zero(h->psi, n, h->store_bytes, stream);
  if (e != cudaSuccess) {
    qs_destroy(h);
    return cuda_fail(e, "init");
  }
  *out = h;
  return QS_OK;
}

}  // namespace qs

extern "C" {

const char* qs_last_error(void) { return g_err.c_str(); }
const char* qs_version(void) { return "qs-gb300 0.1 (sm_103a)"; }

qs_status qs_set_allocator(void* (*alloc_fn)(size_t, void*, void*), void (*free_fn)(void*, size_t, void*, void*),
                           void* ctx) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) return fail(QS_EINVAL, "allocator needs both callbacks");
  g_alloc = alloc_fn;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return QS_OK;
}

qs_status qs_create(int n, qs_dtype dtype, qs_handle* out) {
  if (!out) return fail(QS_EINVAL, "null output handle");
  qs_status st = state_create_on(n, dtype, nullptr, out);
  if (st != QS_OK) return st;
  CUDA_TRY(cudaStreamSynchronize(nullptr), "init");
  return QS_OK;
}

qs_status qs_create_async(int n, qs_dtype dtype, void* stream, qs_handle* out) {
  if (!out) return fail(QS_EINVAL, "null output handle");
  return state_create_on(n, dtype, (cudaStream_t)stream, out);
}

qs_status qs_destroy(qs_handle h) {
  if (!h) return QS_OK;
  // buffers go back in stream order: nothing here waits for the device, except that the
  // profiling events still pending are read first
  if (!h->pending.empty()) collect_stats(h);
  for (auto e : h->free_events) cudaEventDestroy(e);
  // an installed allocator may hand the memory to other streams at once: let this
  // state's work finish first (the default pool orders the frees itself)
  if (!h->native_alloc) cudaStreamSynchronize(h->stream);
  const bool nat = h->native_alloc;
  dev_free_as(h->psi, h->bytes, h->stream, nat);
  dev_free_as(h->scratch, h->bytes, h->stream, nat);
  dev_free_as(h->status_dev, 256, h->stream, nat);
  dev_free_as(h->norm_buf, sizeof(double) * (norm_num_partials() + 1), h->stream, nat);
  dev_free_as(h->gate_pool, h->gate_pool_bytes, h->stream, nat);
  dev_free_as(h->dense_w, kDenseWBytes, h->stream, nat);
  delete h;
  return QS_OK;
}

qs_status qs_set_stream(qs_handle h, void* stream) {
  if (!h) return fail(QS_EINVAL, "null handle");
  // work already enqueued on the old stream completes before the new stream sees the state
  CUDA_TRY(cudaStreamSynchronize(h->stream), "stream switch");
  h->stream = (cudaStream_t)stream;
  return QS_OK;
}

qs_status qs_set_arith(qs_handle h, qs_arith a) {
  if (!h) return fail(QS_EINVAL, "null handle");
  if (a != QS_ARITH_AUTO && a != QS_ARITH_DF && a != QS_ARITH_F64) return fail(QS_EINVAL, "unknown arith");
  h->arith = a;
  return QS_OK;
}

qs_status qs_set_profiling(qs_handle h, int on) {
  if (!h) return fail(QS_EINVAL, "null handle");
  h->profiling = on != 0;
  return QS_OK;
}

qs_status qs_get_kernel_stats(qs_handle h, qs_kernel_stat* out, int max, int* count) {
  if (!h || !count) return fail(QS_EINVAL, "null argument");
  collect_stats(h);
  const int k = std::min<int>(max, (int)h->stats.size());
  for (int i = 0; i < k; i++) out[i] = h->stats[i];
  *count = (int)h->stats.size();
  return QS_OK;
}

qs_status qs_reset_kernel_stats(qs_handle h) {
  if (!h) return fail(QS_EINVAL, "null handle");
  collect_stats(h);
  h->stats.clear();
  return QS_OK;
}

qs_status qs_reset(qs_handle h) {
  if (!h) return fail(QS_EINVAL, "null handle");
  for (int q = 0; q < h->n; q++) h->sigma[q] = q;
  CUDA_TRY(timed(h, "init", (double)h->bytes, [&] { return launch_init_zero(h->psi, h->n, h->store_bytes, h->stream); }),
           "init");
  return QS_OK;
}

qs_status qs_get_info(qs_handle h, int* n, qs_dtype* dtype, void** device_ptr, size_t* bytes) {
  if (!h) return fail(QS_EINVAL, "null handle");
  if (n) *n = h->n;
  if (dtype) *dtype = h->dtype;
  if (device_ptr) *device_ptr = h->psi;
  if (bytes) *bytes = h->bytes;
  return QS_OK;
}

qs_status qs_sync(qs_handle h) {
  if (!h) return fail(QS_EINVAL, "null handle");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "sync");
  return check_status(h);
}

static qs_status apply_op(qs_handle h, const qs_op& op, const double* mats, size_t nmats) {
  HGate g;
  std::string err;
  if (!make_hgate(h->n, op, mats, nmats, &g, &err)) return fail(QS_EINVAL, err);
  return apply_hgate(h, g);
}

qs_status qs_apply_1q(qs_handle h, const double* U, int q) {
  if (!h || !U) return fail(QS_EINVAL, "null argument");
  qs_op op{};
  op.kind = QS_OP_U1;
  op.nq = 1;
  op.q[0] = q;
  op.mat = 0;
  return apply_op(h, op, U, 8);
}

qs_status qs_apply_2q(qs_handle h, const double* U, int q0, int q1) {
  if (!h || !U) return fail(QS_EINVAL, "null argument");
  qs_op op{};
  op.kind = QS_OP_U2;
  op.nq = 2;
  op.q[0] = q0;
  op.q[1] = q1;
  op.mat = 0;
  return apply_op(h, op, U, 32);
}

qs_status qs_apply_controlled(qs_handle h, const double* U, int c, int t) {
  if (!h || !U) return fail(QS_EINVAL, "null argument");
  qs_op op{};
  op.kind = QS_OP_CU;
  op.nq = 2;
  op.q[0] = c;
  op.q[1] = t;
  op.mat = 0;
  return apply_op(h, op, U, 8);
}

qs_status qs_set_dense_path(qs_handle h, int path) {
  if (!h) return fail(QS_EINVAL, "null handle");
  if (path < QS_DENSE_AUTO || path > QS_DENSE_TENSOR) return fail(QS_EINVAL, "unknown dense path");
  h->dense_path = path;
  return QS_OK;
}

qs_status qs_apply_dense(qs_handle h, const double* U, int k, const int* qubits) {
  if (!h || !U || !qubits) return fail(QS_EINVAL, "null argument");
  if (k < 1 || k > kMaxDenseK) return fail(QS_EINVAL, "k must be in [1, 6]");
  for (int t = 0; t < k; t++) {
    if (qubits[t] < 0 || qubits[t] >= h->n) return fail(QS_EINVAL, "qubit out of range");
    for (int u = 0; u < t; u++)
      if (qubits[u] == qubits[t]) return fail(QS_EINVAL, "repeated qubit");
  }
  bool low = true;   // qubits already on storage bits 0..k-1 (any order)
  for (int t = 0; t < k; t++) low &= h->sigma[qubits[t]] < k;
  const bool tensor_ok = h->dtype == QS_C64 && h->n >= dense_mma_min_qubits();
  bool use_tensor = false;
  if (h->dense_path == QS_DENSE_TENSOR) {
    if (!tensor_ok) return fail(QS_EINVAL, "tensor-core dense path needs complex64 and n >= 12");
    use_tensor = true;
  } else if (h->dense_path == QS_DENSE_AUTO) {
    use_tensor = tensor_ok && dense_auto_tensor(k, low);
  }
  if (use_tensor) return apply_dense_tensor(h, U, k, qubits, low);
  qs_op op{};
  op.kind = QS_OP_UK;
  op.nq = k;
  for (int t = 0; t < k; t++) op.q[t] = qubits[t];
  op.mat = 0;
  return apply_op(h, op, U, (size_t)2 << (2 * k));
}

qs_status qs_permute(qs_handle h, const int* perm) {
  if (!h || !perm) return fail(QS_EINVAL, "null argument");
  if (!valid_perm(h->n, perm)) return fail(QS_EINVAL, "perm is not a permutation of 0..n-1");
  std::vector<int> ns(perm, perm + h->n);
  if (ns == h->sigma) return QS_OK;
  std::vector<int> src_of(h->n);
  for (int q = 0; q < h->n; q++) src_of[ns[q]] = h->sigma[q];
  return do_permute(h, src_of, ns, 2.0 * (double)h->bytes);
}

qs_status qs_get_permutation(qs_handle h, int* perm_out) {
  if (!h || !perm_out) return fail(QS_EINVAL, "null argument");
  for (int q = 0; q < h->n; q++) perm_out[q] = h->sigma[q];
  return QS_OK;
}

qs_status qs_compile(int n, const qs_op* ops, size_t nops, const double* mats, size_t nmats, const int* sigma0,
                     const qs_compile_opts* opts, qs_plan_t* out) {
  if (!out) return fail(QS_EINVAL, "null output plan");
  *out = nullptr;
  if (n < 1 || n > kMaxQubits) return fail(QS_EINVAL, "n must be in [1, 36]");
  if (nops > 0 && !ops) return fail(QS_EINVAL, "null ops");
  reap_deferred();
  qs_compile_opts o{};
  o.mode = QS_MODE_TILE;
  o.dtype = QS_C128;
  if (opts) o = *opts;
  std::string err;
  if (!normalize_compile_opts(n, &o, &err)) return fail(QS_EINVAL, err);
  std::vector<int> s0(n);
  if (sigma0) {
    if (!valid_perm(n, sigma0)) return fail(QS_EINVAL, "sigma0 is not a permutation");
    s0.assign(sigma0, sigma0 + n);
  } else {
    for (int q = 0; q < n; q++) s0[q] = q;
  }
  std::vector<HGate> gates(nops);
  for (size_t i = 0; i < nops; i++)
    if (!make_hgate(n, ops[i], mats, nmats, &gates[i], &err)) return fail(QS_EINVAL, "op " + std::to_string(i) + ": " + err);
  qs_plan* p = new qs_plan();
  p->n = n;
  p->dtype = o.dtype;
  p->pol = policy_for((qs_dtype)o.dtype, (qs_arith)o.arith);
  p->sigma0 = s0;
  if (!compile_circuit(n, std::move(gates), s0, o, &p->cr, &err)) {
    delete p;
    return fail(QS_EINVAL, err);
  }
  // device copies are made on first execution, so compiling needs no GPU
  *out = p;
  return QS_OK;
}

qs_status qs_default_cost_model(qs_dtype dtype, qs_arith arith, qs_cost_model* out) {
  if (!out) return fail(QS_EINVAL, "null output");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "unknown dtype");
  if (arith != QS_ARITH_AUTO && arith != QS_ARITH_DF && arith != QS_ARITH_F64) return fail(QS_EINVAL, "unknown arith");
  *out = default_cost_model(policy_for(dtype, arith));
  return QS_OK;
}

qs_status qs_plan_destroy(qs_plan_t p) {
  if (!p) return QS_OK;
  reap_deferred();
  DeferredFree d;
  d.native = p->native_alloc;
  if (p->uploaded) {
    d.bufs = {{p->ops_dev, p->ops_bytes}, {p->rops_dev, p->rops_bytes}, {p->stages_dev, p->stages_bytes},
              {p->pool_dev, p->pool_bytes}, {p->dense_w_dev, p->dense_w_bytes}};
  }
  for (auto& u : p->uses) d.events.push_back(u.second);
  if (p->upload_event) d.events.push_back(p->upload_event);
  if (events_done(d.events)) {
    release_deferred(d);
  } else {   // still in use on some stream: released by a later reap, without waiting here
    std::lock_guard<std::mutex> lk(g_deferred_mu);
    g_deferred.push_back(std::move(d));
  }
  delete p;
  return QS_OK;
}

qs_status qs_plan_get_stats(qs_plan_t p, qs_plan_stats* out) {
  if (!p || !out) return fail(QS_EINVAL, "null argument");
  *out = p->cr.stats;
  return QS_OK;
}

qs_status qs_plan_final_permutation(qs_plan_t p, int* perm_out) {
  if (!p || !perm_out) return fail(QS_EINVAL, "null argument");
  for (int q = 0; q < p->n; q++) perm_out[q] = p->cr.sigma_final[q];
  return QS_OK;
}

qs_status qs_plan_get_trace(qs_plan_t p, int32_t* kinds, int32_t* values, size_t max, size_t* count) {
  if (!p || !count) return fail(QS_EINVAL, "null argument");
  const size_t k = std::min(max, p->cr.trace.size());
  for (size_t i = 0; i < k; i++) {
    if (kinds) kinds[i] = p->cr.trace[i].first;
    if (values) values[i] = p->cr.trace[i].second;
  }
  *count = p->cr.trace.size();
  return QS_OK;
}

// Device copies of a plan, made on first execution on the executing stream (stream-ordered
// allocation and copies); an execution on another stream waits for them through an event.
static qs_status plan_upload(qs_plan* p, cudaStream_t s) {
  if (p->uploaded) {
    if (s != p->upload_stream) CUDA_TRY(cudaStreamWaitEvent(s, p->upload_event, 0), "plan upload wait");
    return QS_OK;
  }
  p->ops_bytes = p->cr.tile_ops.size() * sizeof(DevOp);
  p->rops_bytes = p->cr.reg_ops.size() * sizeof(RegOp);
  p->stages_bytes = p->cr.stages.size() * sizeof(StageRec);
  std::vector<unsigned char> ser = p->cr.pool.serialise(p->pol);
  p->pool_bytes = ser.size();
  p->dense_w_bytes = p->cr.dense_w.size() * sizeof(float);
  if (p->dense_w_bytes) p->dense_w_dev = (float*)dev_alloc(p->dense_w_bytes, s);
  if (p->ops_bytes) p->ops_dev = (DevOp*)dev_alloc(p->ops_bytes, s);
  if (p->rops_bytes) p->rops_dev = (RegOp*)dev_alloc(p->rops_bytes, s);
  if (p->stages_bytes) p->stages_dev = (StageRec*)dev_alloc(p->stages_bytes, s);
  if (p->pool_bytes) p->pool_dev = dev_alloc(p->pool_bytes, s);
  p->uploaded = true;   // whatever was allocated is released with the plan
  p->native_alloc = dev_alloc_native();
  p->upload_stream = s;
  if ((p->ops_bytes && !p->ops_dev) || (p->pool_bytes && !p->pool_dev) || (p->rops_bytes && !p->rops_dev) ||
      (p->stages_bytes && !p->stages_dev) || (p->dense_w_bytes && !p->dense_w_dev))
    return fail(QS_ENOMEM, "plan upload allocation failed");
  // pageable sources: each copy has read its source when the call returns
  cudaError_t e = cudaSuccess;
  if (p->ops_bytes) e = cudaMemcpyAsync(p->ops_dev, p->cr.tile_ops.data(), p->ops_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && p->rops_bytes)
    e = cudaMemcpyAsync(p->rops_dev, p->cr.reg_ops.data(), p->rops_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && p->stages_bytes)
    e = cudaMemcpyAsync(p->stages_dev, p->cr.stages.data(), p->stages_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && p->pool_bytes) e = cudaMemcpyAsync(p->pool_dev, ser.data(), p->pool_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && p->dense_w_bytes)
    e = cudaMemcpyAsync(p->dense_w_dev, p->cr.dense_w.data(), p->dense_w_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->upload_event, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(p->upload_event, s);
  if (e != cudaSuccess) return cuda_fail(e, "plan upload");
  return QS_OK;
}

static qs_status execute_steps(qs_handle h, qs_plan_t p) {
  for (const Step& s : p->cr.steps) {
    const char* name = step_name(s, p->pol);
    if (s.kind == ST_PASS) {
      // a PermuteQubits fused into the pass's store writes the permuted vector to the other
      // buffer (out of place), which then becomes the state
      const bool fused = s.pass.swap_a != s.pass.swap_b;
      if (fused) {
        qs_status st = ensure_scratch(h);
        if (st != QS_OK) return st;
      }
      void* dst = fused ? h->scratch : h->psi;
      CUDA_TRY(timed(h, name, s.bytes,
                     [&] {
                       return launch_tile_pass(p->pol, h->psi, dst, s.pass, p->stages_dev, p->rops_dev, p->ops_dev,
                                               p->pool_dev, h->status_dev, h->stream);
                     }, s.alu),
               "tile pass launch");
      if (fused) {
        std::swap(h->psi, h->scratch);
        h->sigma = s.perm;
      }
    } else if (s.kind == ST_GATE) {
      CUDA_TRY(timed(h, name, s.bytes, [&] { return launch_gate(p->pol, h->psi, h->n, s.op, p->pool_dev, h->stream); },
                     s.alu),
               "gate launch");
    } else if (s.kind == ST_RENORM) {
      qs_status st = renormalize(h);
      if (st != QS_OK) return st;
    } else if (s.kind == ST_DENSE) {
      if (!h->num_sms) {
        int dev = 0;
        CUDA_TRY(cudaGetDevice(&dev), "device query");
        CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
      }
      const float* w = p->dense_w_dev + (size_t)s.dense_idx * kDenseWFloats;
      CUDA_TRY(timed(h, name, s.bytes, [&] { return launch_dense_mma(h->psi, h->n, w, h->status_dev, h->num_sms, h->stream); }),
               "dense block launch");
    } else {
      qs_status st = do_permute(h, s.src_of, s.perm, s.bytes);
      if (st != QS_OK) return st;
    }
  }
  h->sigma = p->cr.sigma_final;
  return QS_OK;
}

qs_status qs_execute(qs_handle h, qs_plan_t p) {
  if (!h || !p) return fail(QS_EINVAL, "null argument");
  if (h->n != p->n) return fail(QS_EINVAL, "plan and state have different n");
  if ((int)h->dtype != p->dtype) return fail(QS_EINVAL, "plan and state have different dtype");
  if (h->sigma != p->sigma0) return fail(QS_EINVAL, "state permutation differs from the plan's start permutation");
  {
    qs_status ust = plan_upload(p, h->stream);
    if (ust != QS_OK) {
      note_plan_use(p, h->stream);   // copies may have been enqueued
      return ust;
    }
  }
  const qs_status st = execute_steps(h, p);
  // whatever was enqueued keeps the plan's buffers alive until it has run
  const qs_status su = note_plan_use(p, h->stream);
  return st != QS_OK ? st : su;
}

qs_status qs_run(qs_handle h, const qs_op* ops, size_t nops, const double* mats, size_t nmats,
                 const qs_compile_opts* opts) {
  if (!h) return fail(QS_EINVAL, "null handle");
  qs_compile_opts o{};
  o.mode = QS_MODE_TILE;
  if (opts) o = *opts;
  o.dtype = h->dtype;
  if (!opts) o.arith = h->arith;
  qs_plan_t p = nullptr;
  qs_status st = qs_compile(h->n, ops, nops, mats, nmats, h->sigma.data(), &o, &p);
  if (st != QS_OK) return st;
  st = qs_execute(h, p);
  // the plan's device buffers are released once the stream has consumed them
  qs_plan_destroy(p);
  return st;
}

qs_status qs_probabilities(qs_handle h, double* out, int order) {
  if (!h || !out) return fail(QS_EINVAL, "null argument");
  if (order != QS_ORDER_LOGICAL && order != QS_ORDER_STORAGE) return fail(QS_EINVAL, "unknown order");
  const size_t N = (size_t)1 << h->n;
  double* d = (double*)dev_alloc(N * sizeof(double), h->stream);
  if (!d) return fail(QS_ENOMEM, "probability buffer allocation failed");
  cudaError_t e = launch_probabilities(h->psi, h->n, h->dtype == QS_C128, d, h->sigma.data(),
                                       order == QS_ORDER_LOGICAL, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(d, N * sizeof(double), h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "probabilities");
  return check_status(h);
}

qs_status qs_get_amplitudes(qs_handle h, void* out, uint64_t first, uint64_t count, int order) {
  if (!h || (!out && count)) return fail(QS_EINVAL, "null argument");
  if (order != QS_ORDER_LOGICAL && order != QS_ORDER_STORAGE) return fail(QS_EINVAL, "unknown order");
  const uint64_t N = 1ull << h->n;
  if (first > N || count > N - first) return fail(QS_EINVAL, "amplitude range out of bounds");
  if (count == 0) return QS_OK;
  const size_t bytes = (size_t)count * h->store_bytes;
  void* d = dev_alloc(bytes, h->stream);
  if (!d) return fail(QS_ENOMEM, "amplitude buffer allocation failed");
  cudaError_t e = launch_gather_amplitudes(h->psi, h->n, h->store_bytes, d, first, count, h->sigma.data(),
                                           order == QS_ORDER_LOGICAL, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(d, bytes, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get amplitudes");
  return check_status(h);
}

qs_status qs_set_amplitudes(qs_handle h, const void* in) {
  if (!h || !in) return fail(QS_EINVAL, "null argument");
  CUDA_TRY(cudaMemcpyAsync(h->psi, in, h->bytes, cudaMemcpyHostToDevice, h->stream), "set amplitudes");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "set amplitudes sync");
  return QS_OK;
}

qs_status qs_copy_range_device(qs_handle h, void* dev, uint64_t first, uint64_t count, int to_state) {
  if (!h || (!dev && count)) return fail(QS_EINVAL, "null argument");
  const uint64_t N = 1ull << h->n;
  if (first > N || count > N - first) return fail(QS_EINVAL, "range out of bounds");
  if (count == 0) return QS_OK;
  char* st = (char*)h->psi + first * h->store_bytes;
  const size_t bytes = (size_t)count * h->store_bytes;
  CUDA_TRY(cudaMemcpyAsync(to_state ? (void*)st : dev, to_state ? (const void*)dev : (const void*)st, bytes,
                           cudaMemcpyDeviceToDevice, h->stream),
           "range copy");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "range copy sync");
  return QS_OK;
}

qs_status qs_gate_matrix(int n, const qs_op* op, const double* mats, size_t nmats, double* U_out, int* k_out) {
  if (!op || !U_out || !k_out) return fail(QS_EINVAL, "null argument");
  if (n < 1 || n > kMaxQubits) return fail(QS_EINVAL, "n must be in [1, 36]");
  HGate g;
  std::string err;
  if (!make_hgate(n, *op, mats, nmats, &g, &err)) return fail(QS_EINVAL, err);
  for (size_t i = 0; i < g.U.size(); i++) {
    U_out[2 * i] = g.U[i].real();
    U_out[2 * i + 1] = g.U[i].imag();
  }
  *k_out = g.nq;
  return QS_OK;
}

qs_status qs_norm(qs_handle h, double* out) {
  if (!h || !out) return fail(QS_EINVAL, "null argument");
  const int np = norm_num_partials();
  CUDA_TRY(timed(h, "norm", (double)h->bytes,
                 [&] { return launch_norm_partials(h->psi, h->n, h->dtype == QS_C128, h->norm_buf, np, h->stream); }),
           "norm partials");
  CUDA_TRY(launch_norm_final(h->norm_buf, np, h->norm_buf + np, h->stream), "norm final");
  CUDA_TRY(cudaMemcpyAsync(out, h->norm_buf + np, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "norm read");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "norm sync");
  return check_status(h);
}

qs_status qs_renormalize(qs_handle h, double* norm_out) {
  if (!h) return fail(QS_EINVAL, "null handle");
  qs_status st = renormalize(h);
  if (st != QS_OK) return st;
  if (!norm_out) return QS_OK;
  CUDA_TRY(cudaMemcpyAsync(norm_out, h->norm_buf + norm_num_partials(), sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream),
           "norm read");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "renormalize sync");
  return check_status(h);
}

qs_status qs_inner(qs_handle a, qs_handle b, double* out) {
  if (!a || !b || !out) return fail(QS_EINVAL, "null argument");
  if (a->n != b->n) return fail(QS_EINVAL, "states have different n");
  if (a->sigma != b->sigma) return fail(QS_EINVAL, "states have different permutations (qs_permute one of them first)");
  if (a != b && a->stream != b->stream) {   // a's stream waits for b's work up to now
    cudaEvent_t ev;
    CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
    cudaError_t e = cudaEventRecord(ev, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(a->stream, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
  }
  const int np = inner_num_partials();
  const size_t nb = sizeof(double) * 2 * (np + 1);
  double* d = (double*)dev_alloc(nb, a->stream);
  if (!d) return fail(QS_ENOMEM, "inner-product buffer allocation failed");
  cudaError_t e = cudaSuccess;
  timed(a, "inner", (double)(a->bytes + b->bytes), [&] {
    e = launch_inner(a->psi, a->dtype == QS_C128, b->psi, b->dtype == QS_C128, a->n, d, d + 2 * np, a->stream);
    return e;
  });
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + 2 * np, 2 * sizeof(double), cudaMemcpyDeviceToHost, a->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(a->stream);
  dev_free(d, nb, a->stream);
  if (e != cudaSuccess) return cuda_fail(e, "inner product");
  return check_status(a);
}

}  // extern "C"
