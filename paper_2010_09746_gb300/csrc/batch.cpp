// Batches of independent circuits: one state buffer, one compiled plan per circuit, and
// "waves" of tile passes -- wave w runs pass w of every circuit that has one -- each wave a
// single persistent launch over all its passes' blocks.  After a first eager run the whole
// sequence (init, waves, per-circuit norms) is captured into a CUDA graph and replayed.
// A circuit's tile passes are compiled exactly as qs_compile compiles them and run through
// the same per-block code, so every amplitude is bitwise the value a solo qs_execute gives.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <atomic>
#include <thread>
#include <vector>

#include "runtime.h"

using namespace qs;

namespace qs {
cudaError_t launch_batch_init(void* psi, int store_bytes, const uint64_t* offs, int count, size_t total_elems,
                              cudaStream_t s);
cudaError_t launch_batch_norms(const void* psi, int is_c128, const uint64_t* offs, const int* ns, int count,
                               double* out, cudaStream_t s);
}  // namespace qs

namespace {

template <class T>
T* upload(qs_batch* b, const std::vector<T>& v, cudaError_t* e) {
  if (v.empty() || *e != cudaSuccess) return nullptr;
  const size_t bytes = v.size() * sizeof(T);
  void* p = dev_alloc_as(bytes, b->stream, b->native_alloc);
  if (!p) {
    *e = cudaErrorMemoryAllocation;
    return nullptr;
  }
  b->allocs.push_back({p, bytes});
  // pageable source: read by the time the call returns; the vector lives in the batch anyway
  *e = cudaMemcpyAsync(p, v.data(), bytes, cudaMemcpyHostToDevice, b->stream);
  return (T*)p;
}

qs_status bfail(qs_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

cudaError_t enqueue(qs_batch* b) {
  cudaError_t e = launch_batch_init(b->psi, b->store_bytes, b->off_d, b->count, b->total_elems, b->stream);
  for (const auto& w : b->waves) {
    if (e != cudaSuccess) break;
    e = launch_tile_batched(b->pol, b->K, b->psi, b->passes_d + w.pass_off, b->prefix_d + w.prefix_off,
                            (int)w.passes.size(), w.prefix.back(), w.maxL, w.minc, b->stages_d, b->rops_d, b->dops_d,
                            b->pool_d, b->status_d, b->stream);
  }
  if (e == cudaSuccess)
    e = launch_batch_norms(b->psi, b->dtype == QS_C128, b->off_d, b->n_d, b->count, b->norms_d, b->stream);
  return e;
}

}  // namespace

namespace qs {

qs_status batch_from_plans(const std::vector<const qs_plan*>& plans, qs_dtype dtype, cudaStream_t stream,
                           qs_batch** out) {
  *out = nullptr;
  const int count = (int)plans.size();
  if (count < 1) return bfail(QS_EINVAL, "empty batch");
  qs_batch* b = new qs_batch();
  b->stream = stream;
  b->native_alloc = dev_alloc_native();
  b->count = count;
  b->dtype = dtype;
  b->store_bytes = dtype == QS_C128 ? 16 : 8;
  b->off.resize(count);
  size_t elems = 0;
  std::vector<std::vector<BatchPass>> per_circuit(count);
  for (int i = 0; i < count; i++) {
    const qs_plan* p = plans[i];
    if (p->dtype != (int)dtype || p->n < 1 || p->n > 30) {
      delete b;
      return bfail(QS_EINVAL, "batch plan " + std::to_string(i) + " has another dtype or n outside [1, 30]");
    }
    b->n.push_back(p->n);
    b->off[i] = elems;
    elems += ((size_t)1 << p->n);
    elems = (elems + 31) & ~(size_t)31;   // 256-byte aligned starts
  }
  // offsets of each plan's stages, register ops, tile ops and pool entries in the
  // concatenation (every circuit's entries start 16-byte aligned, so that its tables stay
  // aligned), and its passes
  std::vector<int> sbase(count), rbase(count), dbase(count);
  std::vector<size_t> pbase(count);
  size_t ns = 0, nr = 0, nd = 0, np = 0;
  for (int i = 0; i < count; i++) {
    const CompileResult& cr = plans[i]->cr;
    b->pol = cr.pol;
    sbase[i] = (int)ns;
    rbase[i] = (int)nr;
    dbase[i] = (int)nd;
    pbase[i] = np;
    ns += cr.stages.size();
    nr += cr.reg_ops.size();
    nd += cr.tile_ops.size();
    np += cr.pool.entries();
    np += np & 1;
    for (const Step& s : cr.steps) {
      if (s.kind != ST_PASS) {
        delete b;
        return bfail(QS_EUNSUPPORTED, "batch plans must consist of tile passes only");
      }
      BatchPass bp;
      bp.tp = s.pass;
      bp.tp.st0 += sbase[i];
      bp.psi_off = b->off[i];
      if (b->K == 0) b->K = bp.tp.K;
      if (bp.tp.K != b->K) {
        delete b;
        return bfail(QS_EUNSUPPORTED, "all circuits of a batch need the same register bits (n too small)");
      }
      per_circuit[i].push_back(bp);
      b->stats.hbm_bytes += s.bytes;
      b->stats.alu_instr += s.alu;
    }
    b->stats.n_gates += cr.stats.n_gates;
    b->stats.n_passes += cr.stats.n_passes;
  }
  if (np == 0) np = 1;
  // the concatenation itself, and the pool in the device format, spread over the host's
  // cores (for thousands of circuits these are hundreds of megabytes)
  b->stages.resize(ns);
  b->rops.resize(nr);
  b->dops.resize(nd);
  const size_t eb = Pool::entry_bytes(b->pol);
  std::vector<unsigned char> ser(np * eb, 0);
  {
    std::atomic<int> next(0);
    auto worker = [&] {
      for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
        const CompileResult& cr = plans[i]->cr;
        const int pb = (int)pbase[i];
        for (size_t k = 0; k < cr.stages.size(); k++) {
          StageRec st = cr.stages[k];
          st.op0 += (st.kind == 0) ? rbase[i] : dbase[i];
          b->stages[sbase[i] + k] = st;
        }
        for (size_t k = 0; k < cr.reg_ops.size(); k++) {
          RegOp r = cr.reg_ops[k];
          if (r.mat >= 0) r.mat += pb;
          b->rops[rbase[i] + k] = r;
        }
        for (size_t k = 0; k < cr.tile_ops.size(); k++) {
          DevOp d = cr.tile_ops[k];
          if (d.mat >= 0) d.mat += pb;
          b->dops[dbase[i] + k] = d;
        }
        if (cr.pool.entries()) cr.pool.serialise_into(b->pol, ser.data() + pbase[i] * eb);
      }
    };
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::max(1u, std::min(nt, 64u));
    if ((int)nt > count) nt = (unsigned)count;
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; t++) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
  }
  b->total_elems = elems;
  size_t maxw = 0;
  for (auto& v : per_circuit) maxw = std::max(maxw, v.size());
  for (size_t w = 0; w < maxw; w++) {
    qs_batch::Wave wave;
    wave.prefix.push_back(0);
    for (int i = 0; i < count; i++) {
      if (w >= per_circuit[i].size()) continue;
      const BatchPass& bp = per_circuit[i][w];
      wave.passes.push_back(bp);
      wave.prefix.push_back(wave.prefix.back() + (1ull << (bp.tp.n - bp.tp.L)));
      wave.maxL = std::max(wave.maxL, bp.tp.L);
      wave.minc = std::min(wave.minc, bp.tp.c);
    }
    b->waves.push_back(std::move(wave));
  }
  b->stats.n_circuits = count;
  b->stats.n_waves = (int64_t)b->waves.size();
  b->stats.state_bytes = (double)elems * b->store_bytes;
  // device copies
  std::vector<BatchPass> all_passes;
  std::vector<uint64_t> all_prefix;
  for (auto& w : b->waves) {
    w.pass_off = all_passes.size();
    w.prefix_off = all_prefix.size();
    all_passes.insert(all_passes.end(), w.passes.begin(), w.passes.end());
    all_prefix.insert(all_prefix.end(), w.prefix.begin(), w.prefix.end());
  }
  cudaError_t e = cudaSuccess;
  b->psi = dev_alloc_as(elems * b->store_bytes, stream, b->native_alloc);
  if (b->psi) b->allocs.push_back({b->psi, elems * b->store_bytes});
  else e = cudaErrorMemoryAllocation;
  b->stages_d = upload(b, b->stages, &e);
  b->rops_d = upload(b, b->rops, &e);
  b->dops_d = upload(b, b->dops, &e);
  b->pool_d = upload(b, ser, &e);
  b->passes_d = upload(b, all_passes, &e);
  b->prefix_d = upload(b, all_prefix, &e);
  b->off_d = upload(b, b->off, &e);
  b->n_d = upload(b, b->n, &e);
  std::vector<double> zeros(count, 0.0);
  b->norms_d = upload(b, zeros, &e);
  std::vector<int> st(64, 0);
  b->status_d = upload(b, st, &e);
  if (e != cudaSuccess) {
    qs_batch_destroy(b);
    set_last_error(std::string("batch upload: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA;
  }
  *out = b;
  return QS_OK;
}

}  // namespace qs


extern "C" {

qs_status qs_batch_create(int count, const int* n, const qs_op* ops, const int64_t* op_offsets, const double* mats,
                          size_t nmats, const qs_compile_opts* opts, qs_batch_t* out) {
  if (!out) return bfail(QS_EINVAL, "null output batch");
  *out = nullptr;
  if (count < 1 || !n || !op_offsets) return bfail(QS_EINVAL, "empty batch");
  qs_compile_opts o{};
  o.mode = QS_MODE_TILE;
  o.dtype = QS_C64;
  if (opts) o = *opts;
  if (o.mode != QS_MODE_TILE) return bfail(QS_EINVAL, "batches run tile-mode plans only");
  if (o.dtype != QS_C64 && o.dtype != QS_C128) return bfail(QS_EINVAL, "unknown dtype");
  if ((o.flags & ~(QS_FLAG_FULL_RX | QS_FLAG_NO_DENSE | QS_FLAG_NO_FUSE)) || o.reg_bits < 0 || o.reg_bits > 5)
    return bfail(QS_EINVAL, "bad options");
  if (o.renorm_every != 0) return bfail(QS_EINVAL, "periodic renormalisation is not available in batches");
  o.flags |= QS_FLAG_NO_DENSE;   // a batch runs tile passes only
  auto t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < count; i++) {
    if (n[i] < 1 || n[i] > 30) return bfail(QS_EINVAL, "circuit " + std::to_string(i) + ": n must be in [1, 30] in a batch");
    if (op_offsets[i + 1] < op_offsets[i]) return bfail(QS_EINVAL, "op_offsets must be non-decreasing");
  }
  // the circuits compile independently (each exactly as qs_compile compiles it): spread them
  // over the host's cores, then concatenate the programs in circuit order
  std::vector<qs_plan_t> plans(count, nullptr);
  std::vector<std::string> errs(count);
  std::vector<qs_status> sts(count, QS_OK);
  {
    std::atomic<int> next(0);
    auto worker = [&] {
      for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
        sts[i] = qs_compile(n[i], ops + op_offsets[i], (size_t)(op_offsets[i + 1] - op_offsets[i]), mats, nmats, nullptr,
                            &o, &plans[i]);
        if (sts[i] != QS_OK) errs[i] = "circuit " + std::to_string(i) + ": " + qs_last_error();
      }
    };
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::max(1u, std::min(nt, 64u));
    if ((int)nt > count) nt = (unsigned)count;
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; t++) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
  }
  qs_status st = QS_OK;
  std::string err;
  for (int i = 0; i < count && st == QS_OK; i++)
    if (sts[i] != QS_OK) {
      st = sts[i];
      err = errs[i];
    }
  qs_batch* b = nullptr;
  if (st == QS_OK) {
    std::vector<const qs_plan*> cp(plans.begin(), plans.end());
    st = batch_from_plans(cp, (qs_dtype)o.dtype, nullptr, &b);
    if (st != QS_OK) err = qs_last_error();
  }
  for (qs_plan_t p : plans) qs_plan_destroy(p);   // never uploaded: nothing on the device
  if (st != QS_OK) return bfail(st, err);
  if (cudaStreamSynchronize(nullptr) != cudaSuccess) {   // uploads done before the stream may change
    qs_batch_destroy(b);
    return bfail(QS_ECUDA, "batch upload");
  }
  b->stats.compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = b;
  return QS_OK;
}

qs_status qs_batch_set_stream(qs_batch_t b, void* stream) {
  if (!b) return bfail(QS_EINVAL, "null batch");
  cudaStreamSynchronize(b->stream);
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->stream = (cudaStream_t)stream;
  return QS_OK;
}

qs_status qs_batch_set_graph(qs_batch_t b, int on) {
  if (!b) return bfail(QS_EINVAL, "null batch");
  b->use_graph = on != 0;
  return QS_OK;
}

qs_status qs_batch_run(qs_batch_t b) {
  if (!b) return bfail(QS_EINVAL, "null batch");
  cudaError_t e;
  if (!b->use_graph || b->runs == 0 || b->stream == nullptr) {
    // eager (the first run also configures the kernels outside any capture)
    e = enqueue(b);
  } else {
    if (!b->graph) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e2 = enqueue(b);
        e = cudaStreamEndCapture(b->stream, &g);
        if (e2 != cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return bfail(QS_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphLaunch(b->graph, b->stream);
  }
  if (e != cudaSuccess) return bfail(QS_ECUDA, std::string("batch run: ") + cudaGetErrorString(e));
  b->runs++;
  return QS_OK;
}

qs_status qs_batch_sync(qs_batch_t b) {
  if (!b) return bfail(QS_EINVAL, "null batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(QS_ECUDA, std::string("batch sync: ") + cudaGetErrorString(e));
  int st = 0;
  cudaMemcpyAsync(&st, b->status_d, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  cudaStreamSynchronize(b->stream);
  if (st != 0) {
    cudaMemsetAsync(b->status_d, 0, sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
    return bfail(QS_ETIMEOUT, "a device-side wait timed out");
  }
  return QS_OK;
}

qs_status qs_batch_norms(qs_batch_t b, double* out) {
  if (!b || !out) return bfail(QS_EINVAL, "null argument");
  qs_status s = qs_batch_sync(b);
  if (s != QS_OK) return s;
  cudaError_t e = cudaMemcpyAsync(out, b->norms_d, sizeof(double) * b->count, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(QS_ECUDA, std::string("batch norms: ") + cudaGetErrorString(e));
  return QS_OK;
}

qs_status qs_batch_get_amplitudes(qs_batch_t b, int i, void* out, uint64_t first, uint64_t count) {
  if (!b || !out) return bfail(QS_EINVAL, "null argument");
  if (i < 0 || i >= b->count) return bfail(QS_EINVAL, "circuit index out of range");
  const uint64_t N = 1ull << b->n[i];
  if (first > N || count > N - first) return bfail(QS_EINVAL, "amplitude range out of bounds");
  qs_status s = qs_batch_sync(b);
  if (s != QS_OK) return s;
  cudaError_t e = cudaMemcpyAsync(out, (char*)b->psi + (b->off[i] + first) * b->store_bytes, count * b->store_bytes,
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(QS_ECUDA, std::string("batch amplitudes: ") + cudaGetErrorString(e));
  return QS_OK;
}

qs_status qs_batch_get_stats(qs_batch_t b, qs_batch_stats* out) {
  if (!b || !out) return bfail(QS_EINVAL, "null argument");
  *out = b->stats;
  return QS_OK;
}

qs_status qs_batch_destroy(qs_batch_t b) {
  if (!b) return QS_OK;
  // the batch's own stream finishes first (the caller may read results right up to here);
  // the buffers then go back in stream order, without waiting for the whole device
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& a : b->allocs) dev_free_as(a.first, a.second, b->stream, b->native_alloc);
  delete b;
  return QS_OK;
}

}  // extern "C"
