// The opaque handle behind ibfem_t (runtime side only).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "../../include/ibfem.h"
#include "host_setup.h"
#include "internal.h"

namespace ibfem {

constexpr int kGraphSteps = 32;   // steps per captured graph (even: parity preserved)
constexpr int kPowerChunk = 32;   // power iterations between host convergence checks

// Device arrays of one discretisation that its clones share: cell classes, cut-cell
// indices and matrices (FP64 and FP32 pairs), K_ref and its tensor-core image, and
// 1/sqrt(M_L).  Freed when the last handle using them is destroyed.
struct DeviceShared {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  int device = 0;
  void (*dev_free)(void*, void*) = nullptr;
  void* alloc_ctx = nullptr;
  ~DeviceShared();
};

struct Handle {
  Handle() = default;
  explicit Handle(std::shared_ptr<Setup> s) : setup_p(std::move(s)) {}
  ibfem_options opt{};
  SetupInput input;
  std::shared_ptr<Setup> setup_p = std::make_shared<Setup>();   // host discretisation (shared by clones)
  Setup& setup = *setup_p;
  std::shared_ptr<DeviceShared> shared;   // device arrays shared with clones
  bool to_shared = false;                 // dalloc places new arrays in `shared`
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevProblem dev{};
  int tile[3] = {1, 1, 1};
  int n_blocks = 0;
  double* U[2] = {nullptr, nullptr};  // U[cur] = u^k, U[1 - cur] = u^{k-1}
  int cur = 0;
  double* W = nullptr;                 // work vector (power iteration, apply)
  double* scratch = nullptr;
  double* d_minv = nullptr;
  float* d_minv32 = nullptr;
  int tc_tile[3] = {1, 1, 1};
  int tc_variant = 0;          // tile shape of the tensor-core kernel (0 full, 1 small)
  int tc_ctas = 0;             // resident CTAs per SM of the exact kernel (0: as many as fit)
  bool tune_cached = false;    // the last ibfem_autotune took its choice from the cache
  void build_tc_tiles();
  void upload_tc_sources();
  void set_tc_variant(int v);
  // tensor-core scheme: 0 exact digit slices, 1 bf16 three-pass, 2 bf16 one pass, 3 FP64-grade
  int tc_scheme() const {
    return opt.precision == IBFEM_EXACT_TC ? 0 : opt.precision == IBFEM_BF16X3_TC ? 1 : opt.precision == IBFEM_EXACT64_TC ? 3 : 2;
  }
  // IMEX (Algorithm 2): host partition/factor and their device copies
  bool imex = false;
  bool consistent = false;      // IBFEM_CDM_CONSISTENT: the IMEX machinery with beta = 0
  double beta = 0.25;
  double* pw[2] = {nullptr, nullptr};   // work vectors of the consistent-mass power iteration
  void prepare_consistent();
  ImexData imex_host;
  ImexDev imex_dev{};
  size_t imex_nnz_alloc = 0;
  std::vector<std::pair<int64_t, double>> src_host;  // merged (lattice dof, value) of the load
  double src_fe = 0.0;
  void imex_upload_factor();
  double* partials = nullptr;
  double* scalars = nullptr;
  double* lam_hist = nullptr;
  double* obs_out = nullptr;
  unsigned long long* counters = nullptr;
  cudaGraphExec_t graphs[2] = {nullptr, nullptr};
  std::vector<void*> allocs;
  size_t device_bytes = 0;
  // K_ref image as uploaded (batched launches share equal images between members)
  std::vector<uint16_t> tc_img_host;
  std::vector<int> tc_frow_host;
  void* batch = nullptr;   // the batch this handle is a member of (its steps run there)
  // device bytes build_device allocates (sources, observers and the IMEX factor excluded)
  size_t planned_device_bytes() const;
  bool have_dt = false, have_init = false;
  double dt = 0.0;
  int64_t step = 0, ring_start = 0;

  void* dalloc(size_t bytes);
  void dfree_all();
  template <typename T>
  T* upload(const std::vector<T>& v);
  void to_lattice(const double* kept, std::vector<double>& lat) const;
  void from_lattice(const std::vector<double>& lat, double* kept) const;
  void build_device();
  void build_clone(const Handle& src);
  void invalidate_graphs();
  // optional per-kernel timing: when `timing` is set, enqueue_step records an event
  // pair around every launch and accumulates into slot_ms after a synchronise
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_slot;
  size_t ev_used = 0;
  std::vector<size_t> step_first_ev, step_last_ev;
  double slot_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int n_slots = 1;
  const char* slot_name[8] = {"step", "", "", "", "", "", "", ""};
  void timed_begin(int slot);
  void timed_end();
  void timed_collect();
  void enqueue_step(int cur);
  void run_steps(int64_t n);
};

// Remove a member from its batch (batch.cu): waits for the batch's queued work first.
void batch_forget(Handle* h);

}  // namespace ibfem

struct ibfem_s : ibfem::Handle {
  using Handle::Handle;
};
