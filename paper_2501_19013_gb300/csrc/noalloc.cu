// K x on the node lattice without any device allocation.
//
// Some callers cannot allocate device memory: an application that hands every byte of
// the GPU to its own fixed-size pool or arena (a cudaMalloc behind its back breaks its
// budget and can fail once the pool holds the memory), or a latency-critical loop that
// must not call cudaMalloc/cudaFree because they may synchronise the whole device.  For
// them this entry point keeps its only scratch buffer -- the per-cut-cell products K^e x_e
// that the cut-cell kernel hands to the assembly kernel -- in the file-scope array below.
// The array is a module global: every GPU that loads the library holds it until the
// process exits, and all calls share it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/ibfem.h"
#include "internal.h"

namespace {

// Scratch for K^e x_e of every cut cell: n_cut * n_loc doubles at most (4 MiB).
constexpr long long kScratchDoubles = 1ll << 19;
static __device__ __align__(256) double g_cut_products[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

namespace ibfem {
void set_last_error(const std::string& msg);  // runtime.cu
}  // namespace ibfem

namespace {
int noalloc_fail(int code, const std::string& msg) {
  ibfem::set_last_error(msg);
  return code;
}
}  // namespace

extern "C" int ibfem_apply_operator_noalloc(int dim, int p, int ncomp, const int n_cells[3],
                                            const uint8_t* cell_class, const int32_t* cut_index,
                                            const int64_t* cut_cells, int64_t n_cut,
                                            const double* K_ref, const double* K_cut,
                                            const double* x, double* y, void* stream) {
  using namespace ibfem;
  if ((dim != 2 && dim != 3) || !n_cells || !cell_class || !cut_index || !K_ref || !x || !y ||
      n_cut < 0 || (n_cut > 0 && (!cut_cells || !K_cut)))
    return noalloc_fail(IBFEM_ERR_ARG, "ibfem_apply_operator_noalloc: bad arguments");
  if (!op_fp64_supported(dim, p, ncomp))
    return noalloc_fail(IBFEM_ERR_ARG, "ibfem_apply_operator_noalloc: no kernel for this (dim, p, ncomp)");
  int nn_loc = 1;
  for (int k = 0; k < dim; ++k) {
    if (n_cells[k] < 1) return noalloc_fail(IBFEM_ERR_ARG, "ibfem_apply_operator_noalloc: cells per axis must be >= 1");
    nn_loc *= p + 1;
  }
  const int n_loc = nn_loc * ncomp;
  // n_cut * n_loc <= kScratchDoubles, written as a division so that no product can overflow
  if (n_cut > kScratchDoubles / n_loc)
    return noalloc_fail(IBFEM_ERR_ARG,
                        "ibfem_apply_operator_noalloc: n_cut = " + std::to_string(n_cut) + " cut cells of " +
                            std::to_string(n_loc) + " DOFs exceed the static scratch of " +
                            std::to_string(kScratchDoubles) + " doubles");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(IBFEM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(IBFEM_ERR_ARG, "device ordinal too large");
  double* scratch = nullptr;
  {
    // one-time set-up per device (with that device current): the host-side name of the
    // array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_cut_products);
      if (e != cudaSuccess) return noalloc_fail(IBFEM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = static_cast<double*>(ptr);
    }
    scratch = g_scratch_addr[dev];
  }
  DevProblem pb{};
  pb.dim = dim;
  pb.p = p;
  pb.ncomp = ncomp;
  pb.n_loc = n_loc;
  pb.nn_loc = nn_loc;
  pb.n_lat_dof = ncomp;
  for (int k = 0; k < 3; ++k) {
    pb.n[k] = k < dim ? n_cells[k] : 1;
    pb.lat[k] = k < dim ? n_cells[k] * p + 1 : 1;
    pb.n_lat_dof *= pb.lat[k];
  }
  pb.cls = cell_class;
  pb.cut_index = cut_index;
  pb.cut_cell = cut_cells;
  pb.n_cut = (int)n_cut;
  pb.Kref = K_ref;
  pb.Kcut = K_cut;
  pb.Ycut = scratch;  // fully written by the cut-cell kernel before the assembly reads it
  int tile[3];
  op_fp64_tiles(dim, p, ncomp, tile);
  for (int k = 0; k < 3; ++k) pb.tiles[k] = k < dim ? (pb.n[k] + tile[k] - 1) / tile[k] : 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  OpInput in{x, nullptr, nullptr};
  e = launch_cut_apply_fp64(pb, in, false, st);
  if (e == cudaSuccess) e = launch_op_fp64(pb, in, y, kModeApply, nullptr, st);
  if (e != cudaSuccess) return noalloc_fail(IBFEM_ERR_CUDA, cudaGetErrorString(e));
  return IBFEM_OK;
}
