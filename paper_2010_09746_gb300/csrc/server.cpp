// Serving loop (no counterpart in the paper): continuous batching of independent circuits.
//
// Requests arrive through qs_server_submit at any time.  A pool of host threads compiles
// each request's plan as soon as it arrives (QS_MODE_TILE, the request's dtype), so that
// compilation never holds up admission.  One admission thread owns the device side: it
// starts a compiled request as soon as one of the server's slots (a CUDA stream) and the
// bytes of its state within the memory budget are free -- it never waits for requests
// already on the GPU -- enqueues state preparation, the plan and the read-out (the FP64 norm
// and the first amplitudes, copied into pinned host memory) on the slot's stream, and
// records an event.  Requests whose states are small (n <= batch_small_n) and that are
// ready together share one slot as one batch: their tile passes run as persistent launches
// over all of their states (the same per-tile code as a solo run, so each result is
// bitwise the solo one).  Completion is found by polling the events; the state is released
// in stream order and the slot goes back to the pool.  Results wait in host memory until the
// caller fetches them (qs_server_poll, qs_server_take).
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "runtime.h"

using namespace qs;

static_assert(sizeof(qs_server_opts) == 48, "qs_server_opts layout");
static_assert(sizeof(qs_server_result) == 192, "qs_server_result layout");
static_assert(sizeof(qs_server_stats) == 80, "qs_server_stats layout");

namespace {

qs_status sfail(qs_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

// one request through its whole life
enum Phase { PH_QUEUED, PH_COMPILING, PH_READY, PH_RUNNING, PH_DONE };
struct Req {
  int64_t id = 0;
  Phase phase = PH_QUEUED;
  bool cancel = false;       // asked to cancel while compiling
  int n = 0;
  qs_dtype dtype = QS_C64;
  std::vector<qs_op> ops;
  std::vector<double> mats;
  qs_plan_t plan = nullptr;
  int K = 0;                 // register bits of the plan's passes (batch grouping key)
  bool batchable = false;    // tile passes only
  double work = 0;           // estimated device work (admission order "least work first")
  double t_submit = 0, t_admit = 0, t_done = 0;
  qs_status status = QS_OK;
  std::string error;
  double norm = 0;
  int batched = 0;
  std::vector<unsigned char> amps;   // first min(2^n, readout) amplitudes, the request's dtype
};

// work on one slot: a solo state or a batch of small states
struct Flight {
  int slot = -1;
  std::vector<std::shared_ptr<Req>> reqs;
  qs_state* state = nullptr;
  qs_batch* batch = nullptr;
  size_t bytes = 0;
  cudaEvent_t done = nullptr;
};

struct Slot {
  cudaStream_t stream = nullptr;
  bool busy = false;
  // pinned staging for the read-outs: norms, then each request's amplitudes
  unsigned char* host = nullptr;
  size_t host_bytes = 0;
};

}  // namespace

struct qs_server {
  qs_server_opts o{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::vector<Slot> slots;
  std::mutex mu;                       // everything below
  std::condition_variable cv_compile;  // compile queue non-empty or stopping
  std::condition_variable cv_loop;     // something for the admission thread
  std::condition_variable cv_done;     // a result finished
  std::deque<std::shared_ptr<Req>> compile_q;
  std::vector<std::shared_ptr<Req>> ready;           // compiled, waiting for a slot
  std::map<int64_t, std::shared_ptr<Req>> finished;  // results not yet taken
  std::map<int64_t, std::shared_ptr<Req>> live;      // submitted, not finished
  std::deque<int64_t> unreported;                    // finished ids not yet returned by poll
  std::vector<Flight> flights;                       // owned by the admission thread
  int64_t next_id = 1;
  int compiling = 0;                                 // requests a compile thread holds
  bool stop = false;
  size_t mem_used = 0;
  qs_server_stats stats{};
  std::vector<std::thread> compilers;
  std::thread loop;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  // one amplitude vector per request: the server compiles tile-mode plans only, whose steps
  // (tile passes, dense blocks, renormalisations) all run in place, so no request ever
  // allocates the permutation buffer (the compile worker refuses a plan that would)
  size_t state_bytes(const Req& r) const { return (size_t)(r.dtype == QS_C128 ? 16 : 8) << r.n; }
  size_t readout_count(const Req& r) const {
    return (size_t)std::min<uint64_t>(1ull << r.n, (uint64_t)o.readout);
  }
};

namespace {

// (caller holds the lock)
void finish_request(qs_server* s, const std::shared_ptr<Req>& r, double t) {
  r->t_done = t;
  r->phase = PH_DONE;
  if (r->plan) {
    qs_plan_destroy(r->plan);   // released once its executions are done (they are)
    r->plan = nullptr;
  }
  s->live.erase(r->id);
  s->finished[r->id] = r;
  s->unreported.push_back(r->id);
  s->stats.completed++;
}

void compile_worker(qs_server* s) {
  cudaSetDevice(s->device);
  set_thread_native_alloc(true);
  for (;;) {
    std::shared_ptr<Req> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_compile.wait(lk, [&] { return s->stop || !s->compile_q.empty(); });
      if (s->compile_q.empty()) return;   // stopping
      r = s->compile_q.front();
      s->compile_q.pop_front();
      s->compiling++;
      r->phase = PH_COMPILING;
    }
    qs_compile_opts co{};
    co.mode = QS_MODE_TILE;
    co.dtype = r->dtype;
    co.tile_bits = s->o.tile_bits;
    qs_plan_t p = nullptr;
    const qs_status st = qs_compile(r->n, r->ops.data(), r->ops.size(), r->mats.data(), r->mats.size(), nullptr, &co, &p);
    const std::string cerr = st != QS_OK ? std::string(qs_last_error()) : std::string();
    std::lock_guard<std::mutex> lk(s->mu);
    s->compiling--;
    if (st != QS_OK || r->cancel) {
      if (st == QS_OK) qs_plan_destroy(p);
      r->status = r->cancel ? QS_ECANCELED : st;
      r->error = r->cancel ? "cancelled" : cerr;
      finish_request(s, r, s->now());
      s->cv_done.notify_all();
      continue;
    }
    bool in_place = true;
    for (const Step& stp : p->cr.steps)
      if (stp.kind == ST_PERMUTE || (stp.kind == ST_PASS && stp.pass.swap_a != stp.pass.swap_b)) in_place = false;
    if (!in_place) {   // the memory admission counts one vector per request
      qs_plan_destroy(p);
      r->status = QS_EUNSUPPORTED;
      r->error = "served plans must run in place (no permutation buffer)";
      finish_request(s, r, s->now());
      s->cv_done.notify_all();
      continue;
    }
    r->plan = p;
    r->batchable = true;
    for (const Step& stp : p->cr.steps) {
      if (stp.kind != ST_PASS) r->batchable = false;
      else if (!r->K) r->K = stp.pass.K;
      else if (r->K != stp.pass.K) r->batchable = false;
    }
    // device work: arithmetic-bound tile passes cost about their counted instructions, with
    // the HBM bytes as a floor for light circuits
    r->work = std::max(p->cr.stats.alu_instr / 40e12, p->cr.stats.hbm_bytes / 6e12) + 5e-6;
    r->phase = PH_READY;
    s->ready.push_back(r);
    s->cv_loop.notify_one();
  }
}

// the device status word (bounded waits) is copied into the last 16 bytes of the slot's pinned
// buffer, which the read-outs never reach
int* status_slot(Slot& sl) { return reinterpret_cast<int*>(sl.host + sl.host_bytes - 16); }

// enqueue the read-out of a finished solo run: FP64 norm and the first amplitudes into the
// slot's pinned buffer (norm at offset 0, amplitudes from offset 16)
cudaError_t enqueue_solo_readout(qs_server* s, Slot& sl, Flight& f) {
  qs_state* h = f.state;
  Req& r = *f.reqs[0];
  const int np = norm_num_partials();
  cudaError_t e = launch_norm_partials(h->psi, h->n, h->dtype == QS_C128, h->norm_buf, np, sl.stream);
  if (e == cudaSuccess) e = launch_norm_final(h->norm_buf, np, h->norm_buf + np, sl.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.host, h->norm_buf + np, sizeof(double), cudaMemcpyDeviceToHost, sl.stream);
  // tile-mode plans end in the identity permutation: the first storage elements are the
  // first logical amplitudes
  const size_t cnt = s->readout_count(r);
  if (e == cudaSuccess && cnt)
    e = cudaMemcpyAsync(sl.host + 16, h->psi, cnt * h->store_bytes, cudaMemcpyDeviceToHost, sl.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status_slot(sl), h->status_dev, sizeof(int), cudaMemcpyDeviceToHost, sl.stream);
  return e;
}

cudaError_t enqueue_batch_readout(qs_server* s, Slot& sl, Flight& f) {
  qs_batch* b = f.batch;
  cudaError_t e = cudaMemcpyAsync(sl.host, b->norms_d, sizeof(double) * b->count, cudaMemcpyDeviceToHost, sl.stream);
  size_t off = ((sizeof(double) * b->count + 15) / 16) * 16;
  for (int i = 0; i < b->count && e == cudaSuccess; i++) {
    const size_t cnt = s->readout_count(*f.reqs[i]);
    if (cnt)
      e = cudaMemcpyAsync(sl.host + off, (char*)b->psi + b->off[i] * b->store_bytes, cnt * b->store_bytes,
                          cudaMemcpyDeviceToHost, sl.stream);
    off += ((cnt * b->store_bytes + 15) / 16) * 16;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(status_slot(sl), b->status_d, sizeof(int), cudaMemcpyDeviceToHost, sl.stream);
  return e;
}

// the index in `ready` to admit next (caller holds the lock; ready is not empty)
size_t pick_next(qs_server* s, double now) {
  size_t oldest = 0;
  for (size_t i = 1; i < s->ready.size(); i++)
    if (s->ready[i]->t_submit < s->ready[oldest]->t_submit) oldest = i;
  if (s->o.order == 0 || now - s->ready[oldest]->t_submit >= s->o.max_wait_ms * 1e-3) return oldest;
  size_t best = 0;
  for (size_t i = 1; i < s->ready.size(); i++)
    if (s->ready[i]->work < s->ready[best]->work ||
        (s->ready[i]->work == s->ready[best]->work && s->ready[i]->t_submit < s->ready[best]->t_submit))
      best = i;
  return best;
}

// admit as many ready requests as slots and memory allow; returns how many started
int admit(qs_server* s) {
  int started = 0;
  for (;;) {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->ready.empty()) return started;
    int slot = -1;
    for (size_t i = 0; i < s->slots.size(); i++)
      if (!s->slots[i].busy) {
        slot = (int)i;
        break;
      }
    if (slot < 0) return started;
    const double now = s->now();
    const size_t k = pick_next(s, now);
    std::shared_ptr<Req> head = s->ready[k];
    const size_t need = s->state_bytes(*head);
    if (s->mem_used + need > (size_t)s->o.mem_budget) return started;
    // group: ready small requests of the same dtype and register bits, oldest first
    std::vector<std::shared_ptr<Req>> group{head};
    size_t mem = need;
    if (head->batchable && head->n <= s->o.batch_small_n && s->o.batch_max > 1) {
      std::vector<size_t> idx;
      for (size_t i = 0; i < s->ready.size(); i++)
        if (i != k) idx.push_back(i);
      std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return s->ready[a]->t_submit < s->ready[b]->t_submit; });
      for (size_t i : idx) {
        const auto& r = s->ready[i];
        if ((int)group.size() >= s->o.batch_max) break;
        const size_t b2 = s->state_bytes(*r);
        if (r->batchable && r->n <= s->o.batch_small_n && r->dtype == head->dtype && r->K == head->K &&
            s->mem_used + mem + b2 <= (size_t)s->o.mem_budget) {
          group.push_back(r);
          mem += b2;
        }
      }
    }
    // the read-outs must fit the slot's pinned buffer
    size_t host_need = 16 * (group.size() + 1) + sizeof(double) * group.size();
    for (auto& r : group) host_need += ((s->readout_count(*r) * (r->dtype == QS_C128 ? 16 : 8) + 15) / 16) * 16;
    while (group.size() > 1 && host_need > s->slots[slot].host_bytes) {
      host_need -= ((s->readout_count(*group.back()) * (group.back()->dtype == QS_C128 ? 16 : 8) + 15) / 16) * 16;
      mem -= s->state_bytes(*group.back());
      group.pop_back();
    }
    // take them off the ready list
    std::vector<std::shared_ptr<Req>> keep;
    for (auto& r : s->ready)
      if (std::find(group.begin(), group.end(), r) == group.end()) keep.push_back(r);
    s->ready.swap(keep);
    Slot& sl = s->slots[slot];
    sl.busy = true;
    s->mem_used += mem;
    s->stats.peak_mem_bytes = std::max(s->stats.peak_mem_bytes, (double)s->mem_used);
    for (auto& r : group) {
      r->t_admit = now;
      r->phase = PH_RUNNING;
    }
    lk.unlock();

    // ---- device work, outside the lock
    Flight f;
    f.slot = slot;
    f.reqs = group;
    f.bytes = mem;
    qs_status st = QS_OK;
    std::string err;
    cudaError_t e = cudaSuccess;
    if (group.size() == 1) {
      Req& r = *group[0];
      st = state_create_on(r.n, r.dtype, sl.stream, &f.state);
      if (st == QS_OK) st = qs_execute(f.state, r.plan);
      if (st == QS_OK) e = enqueue_solo_readout(s, sl, f);
      if (st != QS_OK) err = qs_last_error();
    } else {
      std::vector<const qs_plan*> plans;
      for (auto& r : group) plans.push_back(r->plan);
      st = batch_from_plans(plans, head->dtype, sl.stream, &f.batch);
      if (st == QS_OK) {
        f.batch->use_graph = false;
        st = qs_batch_run(f.batch);
        if (st == QS_OK) {
          // the plans' data now lives in the batch: they can go (never uploaded)
          for (auto& r : group) {
            qs_plan_destroy(r->plan);
            r->plan = nullptr;
            r->batched = 1;
          }
          e = enqueue_batch_readout(s, sl, f);
        }
      }
      if (st != QS_OK) err = qs_last_error();
    }
    if (st == QS_OK && e != cudaSuccess) {
      st = QS_ECUDA;
      err = std::string("serving read-out: ") + cudaGetErrorString(e);
    }
    if (st == QS_OK) {
      e = cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(f.done, sl.stream);
      if (e != cudaSuccess) {
        st = QS_ECUDA;
        err = std::string("serving event: ") + cudaGetErrorString(e);
      }
    }
    if (st != QS_OK) {   // the request(s) fail; the slot's stream drains before reuse
      cudaStreamSynchronize(sl.stream);
      if (f.state) qs_destroy(f.state);
      if (f.batch) qs_batch_destroy(f.batch);
      if (f.done) cudaEventDestroy(f.done);
      std::lock_guard<std::mutex> lk2(s->mu);
      for (auto& r : group) {
        r->status = st;
        r->error = err;
        finish_request(s, r, s->now());
      }
      sl.busy = false;
      s->mem_used -= mem;
      s->cv_done.notify_all();
      continue;
    }
    {
      std::lock_guard<std::mutex> lk2(s->mu);
      s->flights.push_back(std::move(f));
      s->stats.in_flight += (int64_t)group.size();
      s->stats.peak_in_flight = std::max(s->stats.peak_in_flight, s->stats.in_flight);
      if (group.size() > 1) {
        s->stats.batches++;
        s->stats.batched_requests += (int64_t)group.size();
      }
    }
    started += (int)group.size();
  }
}

// collect finished flights; returns how many requests completed
int reap(qs_server* s) {
  std::vector<Flight> done;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<Flight> keep;
    for (Flight& f : s->flights) {
      const cudaError_t q = cudaEventQuery(f.done);
      if (q == cudaErrorNotReady) keep.push_back(std::move(f));
      else done.push_back(std::move(f));
    }
    s->flights.swap(keep);
  }
  int n = 0;
  for (Flight& f : done) {
    Slot& sl = s->slots[f.slot];
    const cudaError_t q = cudaEventQuery(f.done);
    qs_status st = (q == cudaSuccess) ? QS_OK : QS_ECUDA;
    std::string err = (q == cudaSuccess) ? "" : std::string("serving: ") + cudaGetErrorString(q);
    // a bounded device-side wait that gave up leaves its status word set (copied with the
    // read-out, before the event)
    const int dev_status = *status_slot(sl);
    if (st == QS_OK && dev_status != 0) {
      st = (qs_status)dev_status;
      err = "a device-side wait timed out";
    }
    const double t = s->now();
    size_t off = f.batch ? ((sizeof(double) * f.reqs.size() + 15) / 16) * 16 : 16;
    for (size_t i = 0; i < f.reqs.size(); i++) {
      Req& r = *f.reqs[i];
      r.status = st;
      r.error = err;
      double nv = 0;
      memcpy(&nv, sl.host + (f.batch ? sizeof(double) * i : 0), sizeof(double));
      r.norm = nv;
      const size_t bytes = s->readout_count(r) * (r.dtype == QS_C128 ? 16 : 8);
      r.amps.assign(sl.host + off, sl.host + off + bytes);
      off += ((bytes + 15) / 16) * 16;
    }
    if (f.state) qs_destroy(f.state);   // stream-ordered release
    if (f.batch) {
      for (auto& a : f.batch->allocs) dev_free_as(a.first, a.second, sl.stream, f.batch->native_alloc);
      f.batch->allocs.clear();
      delete f.batch;
    }
    cudaEventDestroy(f.done);
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& r : f.reqs) finish_request(s, r, t);
    s->stats.in_flight -= (int64_t)f.reqs.size();
    sl.busy = false;
    s->mem_used -= f.bytes;
    n += (int)f.reqs.size();
  }
  if (n) s->cv_done.notify_all();
  return n;
}

void loop_main(qs_server* s) {
  cudaSetDevice(s->device);
  set_thread_native_alloc(true);
  for (;;) {
    const int done = reap(s);
    const int started = admit(s);
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop && s->flights.empty() && s->compile_q.empty() && s->compiling == 0 && s->ready.empty()) return;
    if (!done && !started) {
      // nothing moved: wait for a submission, a compiled plan or a short while (flights
      // are polled, their events cannot wake this thread)
      s->cv_loop.wait_for(lk, std::chrono::microseconds(s->flights.empty() ? 2000 : 100));
    }
  }
}

}  // namespace

extern "C" {

qs_status qs_server_create(const qs_server_opts* opts, qs_server_t* out) {
  if (!out) return sfail(QS_EINVAL, "null output server");
  *out = nullptr;
  qs_server_opts o{};
  if (opts) o = *opts;
  if (o.slots == 0) o.slots = 8;
  if (o.compile_threads == 0) o.compile_threads = 4;
  if (o.readout == 0) o.readout = 256;
  if (o.batch_small_n == 0) o.batch_small_n = 16;
  if (o.batch_max == 0) o.batch_max = 64;
  if (o.max_wait_ms == 0) o.max_wait_ms = 1000;
  if (o.slots < 1 || o.slots > 256 || o.compile_threads < 1 || o.compile_threads > 256 || o.readout < 0 ||
      o.batch_max < 1 || o.order < 0 || o.order > 1 || o.max_wait_ms < 0 || o.mem_budget < 0 || o.readout > (1 << 24) ||
      o.tile_bits < 0 || o.tile_bits > kMaxTileBits || o.reserved != 0)
    return sfail(QS_EINVAL, "invalid server options");
  qs_server* s = new qs_server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return sfail(QS_ECUDA, "no current device");
  }
  if (o.mem_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return sfail(QS_ECUDA, "cudaMemGetInfo failed");
    }
    o.mem_budget = (int64_t)(fr / 4 * 3);
  }
  s->o = o;
  s->t0 = std::chrono::steady_clock::now();
  s->slots.resize(o.slots);
  const size_t per_amp = 16;
  for (Slot& sl : s->slots) {
    // room for one request's read-out, and for a full batch's up to 64 MiB (admission trims
    // a batch to what fits)
    const size_t per_req = ((size_t)o.readout * per_amp + 15) / 16 * 16 + 32;
    sl.host_bytes = std::max(per_req + 64, std::min<size_t>((size_t)o.batch_max * per_req + 64, (size_t)64 << 20));
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.host, sl.host_bytes);
    if (e != cudaSuccess) {
      for (Slot& x : s->slots) {
        if (x.stream) cudaStreamDestroy(x.stream);
        if (x.host) cudaFreeHost(x.host);
      }
      delete s;
      return sfail(QS_ECUDA, std::string("server slot setup: ") + cudaGetErrorString(e));
    }
  }
  for (int i = 0; i < o.compile_threads; i++) s->compilers.emplace_back(compile_worker, s);
  s->loop = std::thread(loop_main, s);
  *out = s;
  return QS_OK;
}

qs_status qs_server_submit(qs_server_t s, int n, qs_dtype dtype, const qs_op* ops, size_t nops, const double* mats,
                           size_t nmats, int64_t* id_out) {
  if (!s || !id_out || (nops && !ops)) return sfail(QS_EINVAL, "null argument");
  if (n < 1 || n > 30) return sfail(QS_EINVAL, "served requests need 1 <= n <= 30");
  if (dtype != QS_C64 && dtype != QS_C128) return sfail(QS_EINVAL, "unknown dtype");
  auto r = std::make_shared<Req>();
  r->n = n;
  r->dtype = dtype;
  if ((size_t)(dtype == QS_C128 ? 16 : 8) << n > (size_t)s->o.mem_budget)
    return sfail(QS_EINVAL, "request needs more device memory than the server's whole budget");
  r->ops.assign(ops, ops + nops);
  if (nmats) r->mats.assign(mats, mats + nmats);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return sfail(QS_EBUSY, "server is stopping");
  r->id = s->next_id++;
  r->t_submit = s->now();
  s->compile_q.push_back(r);
  s->live[r->id] = r;
  s->stats.submitted++;
  *id_out = r->id;
  s->cv_compile.notify_one();
  s->cv_loop.notify_one();
  return QS_OK;
}

qs_status qs_server_poll(qs_server_t s, qs_server_result* out, int max, int* count, int timeout_ms) {
  if (!s || !count || (max > 0 && !out)) return sfail(QS_EINVAL, "null argument");
  *count = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->unreported.empty() && timeout_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->unreported.empty(); });
  while (*count < max && !s->unreported.empty()) {
    const int64_t id = s->unreported.front();
    s->unreported.pop_front();
    auto it = s->finished.find(id);
    if (it == s->finished.end()) continue;
    const Req& r = *it->second;
    qs_server_result& x = out[(*count)++];
    memset(&x, 0, sizeof(x));
    x.id = r.id;
    x.status = r.status;
    x.n = r.n;
    x.dtype = r.dtype;
    x.batched = r.batched;
    x.norm = r.norm;
    x.t_submit_s = r.t_submit;
    x.t_admit_s = r.t_admit;
    x.t_done_s = r.t_done;
    x.amplitudes = r.amps.size() / (r.dtype == QS_C128 ? 16 : 8);
    strncpy(x.error, r.error.c_str(), sizeof(x.error) - 1);
  }
  return QS_OK;
}

qs_status qs_server_take(qs_server_t s, int64_t id, void* amps, uint64_t count) {
  if (!s) return sfail(QS_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->finished.find(id);
  if (it == s->finished.end()) return sfail(QS_EINVAL, "no finished request with this id (or already taken)");
  const Req& r = *it->second;
  const size_t eb = r.dtype == QS_C128 ? 16 : 8;
  if (count > r.amps.size() / eb) return sfail(QS_EINVAL, "more amplitudes requested than the result holds");
  if (count && !amps) return sfail(QS_EINVAL, "null amplitude buffer");
  if (count) memcpy(amps, r.amps.data(), count * eb);
  s->finished.erase(it);
  return QS_OK;
}

qs_status qs_server_cancel(qs_server_t s, int64_t id) {
  if (!s) return sfail(QS_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->live.find(id);
  if (it == s->live.end()) {
    if (id >= 1 && id < s->next_id) return sfail(QS_EBUSY, "request already finished");
    return sfail(QS_EINVAL, "no request with this id");
  }
  std::shared_ptr<Req> r = it->second;
  switch (r->phase) {
    case PH_QUEUED:
      for (auto q = s->compile_q.begin(); q != s->compile_q.end(); ++q)
        if (*q == r) {
          s->compile_q.erase(q);
          break;
        }
      break;
    case PH_READY:
      s->ready.erase(std::find(s->ready.begin(), s->ready.end(), r));
      break;
    case PH_COMPILING:   // the compile thread drops it when it is done
      r->cancel = true;
      return QS_OK;
    default:
      return sfail(QS_EBUSY, "request already on the GPU");
  }
  r->status = QS_ECANCELED;
  r->error = "cancelled";
  finish_request(s, r, s->now());
  s->cv_done.notify_all();
  return QS_OK;
}

qs_status qs_server_get_stats(qs_server_t s, qs_server_stats* out) {
  if (!s || !out) return sfail(QS_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->waiting = (int64_t)(s->compile_q.size() + s->ready.size());
  out->mem_used_bytes = (double)s->mem_used;
  out->now_s = s->now();
  return QS_OK;
}

qs_status qs_server_destroy(qs_server_t s) {
  if (!s) return QS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_compile.notify_all();
  s->cv_loop.notify_all();
  for (auto& t : s->compilers) t.join();
  // the admission thread finishes every request already submitted, then returns
  s->loop.join();
  for (auto& kv : s->finished)
    if (kv.second->plan) qs_plan_destroy(kv.second->plan);
  for (Slot& sl : s->slots) {
    cudaStreamSynchronize(sl.stream);
    cudaStreamDestroy(sl.stream);
    cudaFreeHost(sl.host);
  }
  delete s;
  return QS_OK;
}

}  // extern "C"
