// Runtime objects behind the C ABI handles (states, plans, batches) and the host helpers that
// the ABI files share.  Internal: not part of include/qs.h.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "qs_internal.h"

struct KernelRecord {
  std::string name;
  cudaEvent_t e0, e1;
  double bytes;
  double alu;
};

constexpr size_t kDenseWBytes = 2 * 128 * 128 * sizeof(float);

struct qs_state {
  int n = 0;
  qs_dtype dtype = QS_C128;
  qs_arith arith = QS_ARITH_AUTO;
  int store_bytes = 16;
  size_t bytes = 0;
  void* psi = nullptr;
  void* scratch = nullptr;        // permutation target, allocated on first use
  std::vector<int> sigma;
  cudaStream_t stream = nullptr;
  int* status_dev = nullptr;      // device status word (bounded waits)
  double* norm_buf = nullptr;     // norm partials + result
  void* gate_pool = nullptr;      // matrix entries of qs_apply_* calls
  size_t gate_pool_bytes = 0;
  int dense_path = QS_DENSE_AUTO; // qs_apply_dense engine (qs_set_dense_path)
  float* dense_w = nullptr;       // 2 x 128 x 128 floats: W^T split for the tensor-core kernel
  int num_sms = 0;
  bool profiling = false;
  std::vector<KernelRecord> pending;
  std::vector<cudaEvent_t> free_events;
  std::vector<qs_kernel_stat> stats;
  bool native_alloc = true;       // buffers come from cudaMallocAsync (else the installed allocator)
};

struct qs_plan {
  int n = 0;
  int dtype = QS_C128;
  qs::Policy pol = qs::POL_DF;
  std::vector<int> sigma0;
  qs::CompileResult cr;
  qs::DevOp* ops_dev = nullptr;
  size_t ops_bytes = 0;
  qs::RegOp* rops_dev = nullptr;
  size_t rops_bytes = 0;
  qs::StageRec* stages_dev = nullptr;
  size_t stages_bytes = 0;
  void* pool_dev = nullptr;
  size_t pool_bytes = 0;
  float* dense_w_dev = nullptr;           // ST_DENSE operands
  size_t dense_w_bytes = 0;
  bool uploaded = false;
  bool native_alloc = true;
  cudaStream_t upload_stream = nullptr;   // the device copies were enqueued here ...
  cudaEvent_t upload_event = nullptr;     // ... and are complete once this has completed
  // one event per stream the plan was executed on, recorded after its last launch there:
  // the device buffers are released once all of them have completed
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
};

struct qs_batch {
  int count = 0;
  qs_dtype dtype = QS_C64;
  qs::Policy pol = qs::POL_F32;
  int K = 0;
  int store_bytes = 8;
  std::vector<int> n;
  std::vector<uint64_t> off;       // element offset of each state
  size_t total_elems = 0;
  // concatenated plan data
  std::vector<qs::StageRec> stages;
  std::vector<qs::RegOp> rops;
  std::vector<qs::DevOp> dops;
  struct Wave {
    std::vector<qs::BatchPass> passes;
    std::vector<uint64_t> prefix;
    int maxL = 0, minc = 64;
    size_t pass_off = 0, prefix_off = 0;   // into the device arrays
  };
  std::vector<Wave> waves;
  qs_batch_stats stats{};
  // device
  void* psi = nullptr;
  qs::StageRec* stages_d = nullptr;
  qs::RegOp* rops_d = nullptr;
  qs::DevOp* dops_d = nullptr;
  void* pool_d = nullptr;
  qs::BatchPass* passes_d = nullptr;
  uint64_t* prefix_d = nullptr;
  uint64_t* off_d = nullptr;
  int* n_d = nullptr;
  double* norms_d = nullptr;
  int* status_d = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;   // device buffers (from dev_alloc on `stream`)
  bool native_alloc = true;
  cudaStream_t stream = nullptr;
  bool use_graph = true;
  int runs = 0;
  cudaGraphExec_t graph = nullptr;
};

namespace qs {

// Device memory through the allocator installed with qs_set_allocator, else
// cudaMallocAsync / cudaFreeAsync on stream s (stream-ordered).
void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, size_t bytes, cudaStream_t s);
void* dev_alloc_as(size_t bytes, cudaStream_t s, bool native);
// the same for memory whose allocator kind was recorded at allocation (native = cudaMallocAsync)
void dev_free_as(void* p, size_t bytes, cudaStream_t s, bool native);
// whether this thread's allocations bypass the installed allocator (or none is installed)
bool dev_alloc_native();
// make this thread's allocations use cudaMallocAsync even when an allocator is installed
// (the serving threads: callbacks into a host runtime from them could stall on its locks)
void set_thread_native_alloc(bool on);
Policy policy_for(qs_dtype dt, qs_arith a);

// A state of n qubits allocated and set to |0...0> on `stream`, without synchronising.
qs_status state_create_on(int n, qs_dtype dtype, cudaStream_t stream, qs_state** out);
// Record that plan p has just been enqueued on stream s (its buffers outlive that work).
qs_status note_plan_use(qs_plan* p, cudaStream_t s);

// A batch built from plans compiled in QS_MODE_TILE (one per circuit, in order; every plan
// consists of tile passes with the same register bits), its device buffers allocated and
// uploaded on `stream`, which becomes the batch's stream.  On failure *out stays NULL and
// the status says why.
qs_status batch_from_plans(const std::vector<const qs_plan*>& plans, qs_dtype dtype, cudaStream_t stream,
                           qs_batch** out);

}  // namespace qs
