// Internal device-side types shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace ibfem {

// Per-lattice-DOF arrays use the node lattice (n_k p + 1 nodes per axis, x fastest) with
// the ncomp components of a node interleaved.  Dead lattice nodes (not in any kept cell)
// carry zero mass and are never written.
struct DevProblem {
  int dim, p, ncomp, n_loc, nn_loc;
  int n[3];          // cells per axis
  int lat[3];        // lattice nodes per axis
  int64_t n_lat_dof;
  const uint8_t* cls;       // per cell: 0 outside, 1 cut, 2 uncut
  const int32_t* cut_index; // per cell
  const int64_t* cut_cell;  // cut index -> cell
  const int32_t* cut_mat;   // cut index -> matrix index of Kcut / Kcut32 (null: the same index)
  int n_cut;
  const double* Kref;       // n_loc^2 (symmetric)
  const double* Kcut;       // per cut matrix n_loc^2 (symmetric, row-major)
  const float* Kcut32;      // per cut matrix: n_loc^2 interleaved FP32 (hi, lo) pairs
  double* Ycut;             // n_cut * n_loc: K^e x_e of the cut cells for the current step
  const double* minv;       // dt^2 / M_L per lattice DOF (0 = dead); -(c + 1) marks IMEX c-DOF c
  const double* sinv;       // 1 / sqrt(M_L) per lattice DOF (0 = dead or IMEX c-DOF)
  // source: per tile CSR of (lattice dof, value)
  const int32_t* src_ptr;   // n_tiles + 1, or null
  const int64_t* src_dof;
  const double* src_val;
  double f_e;               // Ricker centre frequency (0 = no source)
  double dt;
  // observers
  int n_obs_rows;           // observers x ncomp
  int obs_nodes;            // nn_loc
  const int64_t* obs_dof;   // n_obs_rows * nn_loc lattice dofs
  const double* obs_w;      // n_obs_rows * nn_loc weights
  double* ring;             // capacity * n_obs_rows
  int64_t ring_cap;
  // counters
  unsigned long long* step; // device step counter
  unsigned int* done;       // block-completion counter for the step increment
  int* tile_counter;        // persistent tensor-core kernel: next tile to take (reset by the last block)
  int* flags;               // bit 0: non-finite state
  int tiles[3];             // tile grid of the fused kernel
  // mixed-precision tensor-core path
  int tc_tiles[3];          // tile grid of the tensor-core kernel
  const uint16_t* tc_bimg;  // K_ref as UMMA B operand: four BF16 slices (digits or hi/lo)
  const int* tc_frow;       // exact scheme: unbiased exponent F_i of each K_ref row
  int tc_gexp;              // FP64-grade scheme: unbiased exponent G of K_ref's largest entry
  const int32_t* tc_order;  // tensor-core tiles in processing order (costliest first), or null
  const float* minv32;      // dt^2 / M_L as two FP32 slices: hi[n_lat_dof] then lo[n_lat_dof]
  const int32_t* tsrc_ptr;  // source CSR over the tensor-core tile grid
  const int64_t* tsrc_dof;
  const double* tsrc_val;
  // IMEX: c-DOF velocity / acceleration (c-index order) and predictor coefficients
  double* imex_vc;
  double* imex_ac;
  double imex_c1;           // (1/2 - beta) dt^2
  double imex_c2;           // (1 - gamma) dt
};

// One problem of a batched tensor-core launch: its descriptor, its two state buffers and
// the step at which it stops.  The state u^k lives in Ua for even k and in Ub for odd k,
// so that a member's buffers do not depend on when it joined the batch.
struct BatchMember {
  DevProblem pb;
  double* Ua;
  double* Ub;
  unsigned long long step_end;   // tiles of a member with step >= step_end are skipped
};

// Launch-wide counters of a batched launch (reset by its last CTA).
struct BatchCtl {
  int tile_counter;
  unsigned int done;
};

// Device view of the IMEX partition and factor (kernels_imex.cu).
// One CTA of a sweep of the block solve: its supernode sn (first row st, wd rows, dense
// block at doff), the threads per row of its off-block sums, its share c of the g CTAs of the
// supernode, for g > 1 the supernode's first partial sum (32 per CTA; pbase / 32 is the
// supernode's arrival counter), and the supernodes it waits for (dep[dep_beg, dep_beg +
// dep_n) of its direction).
struct __align__(16) LevelTask {
  int32_t st;
  int32_t wd_tpr;            // wd | tpr << 16
  int32_t c, g;
  int64_t doff, pbase;
  int32_t sn, dep_beg, dep_n, pad;
};

// One direction's sweep (CTAs in the order they take tickets).
struct ImexSplitDev {
  const LevelTask* task;
  const int32_t* dep;
  unsigned int* done;        // per supernode: the epoch of the sweep that finished it
  int n_tasks;
};

// Sweep control in device memory: the ticket counters of the two sweeps and the epoch of
// the current solve (the kernel before a solve resets the tickets and advances the epoch).
struct SweepCtl {
  unsigned int tick[2];
  unsigned int epoch;
  unsigned int pad;
};

struct ImexDev {
  int n_cells;               // cells touching the c-set
  const int64_t* cells;
  double* Y;                 // n_cells * n_loc products K^e x_e
  int64_t n_rows;            // c-DOFs (rows of S, permuted order)
  const int64_t* g_ptr;      // residual gather per permuted row
  const int32_t* g_idx;
  const double* Fc;          // spatial load on the c-DOFs (permuted rows), or null
  double* work;              // n_c
  const int32_t* Li;         // L by rows, diagonal last (column indices)
  const double* Lx;
  const int32_t* Ui;         // L^T by rows, diagonal first
  const double* Ux;
  // block triangular solves: supernodes (contiguous permuted rows of at most 32) with the
  // dense diagonal block of L (row-major w x w at the task's doff, 1 / L_jj on the
  // diagonal) and its transpose DT; per row the range of its off-block entries in L
  // (forward) and in L^T (backward); per direction the CTAs of its sweep, the partial sums
  // of split supernodes and one arrival counter per split supernode
  const double* D;
  const double* DT;
  const int2* row_fdesc;     // {Lp[r], end of the off-block entries of row r}
  const int2* row_bdesc;     // {start of the off-block entries of row r of L^T, Up[r + 1]}
  ImexSplitDev fs, bs;       // forward, backward
  double* part;
  unsigned int* cnt;         // per split supernode; zero between launches (its last CTA resets it)
  SweepCtl* ctl;
  int* flags;                // bit 1: a bounded wait gave up
  const int64_t* perm;       // permuted row -> c index
  const int64_t* c_dof;      // c index -> lattice DOF
  double* vc;
  double* ac;
  double beta_dt2, gamma_dt;
};

// Input transform of the operator kernels: x_i = in[i] * (vec ? vec[i] : 1) * (scal ? *scal : 1)
struct OpInput {
  const double* in;
  const double* vec;
  const double* scal;
};

enum OpMode : int {
  kModeCDM = 0,       // out <- 2u - out + minv (F_k - K u), u = the input
  kModeStartup = 1,   // out <- u - dt * out + 0.5 minv (F_0 - K u)  (out holds v0)
  kModeApply = 2,     // out <- K x
  kModePower = 3,     // out <- sinv * K x, partial sums of x_in * out and out * out
  kModeImex = 4,      // d-DOFs: CDM update; c-DOFs: Newmark predictor (no step advance)
};

// Launchers (kernels_fp64.cu)
cudaError_t launch_cut_apply_fp64(const DevProblem& pb, OpInput x, bool sample, cudaStream_t st,
                                  bool do_cut = true);
// Launchers (kernels_imex.cu)
cudaError_t launch_imex_cell_apply(const DevProblem& pb, const ImexDev& im, const double* x, cudaStream_t st);
cudaError_t launch_imex_solve(const DevProblem& pb, const ImexDev& im, double* out, cudaStream_t st);
cudaError_t launch_imex_tri(const ImexDev& im, const double* in, const double* scal, double* out, bool backward,
                            cudaStream_t st);
cudaError_t launch_scale_vec(int64_t n, const double* s, const double* in, const double* scal, double* out,
                             cudaStream_t st);
cudaError_t launch_dot2(int64_t n, const double* a, const double* scal, const double* b, double* partials,
                        int nblocks, cudaStream_t st);
cudaError_t launch_op_fp64(const DevProblem& pb, OpInput x, double* out, int mode,
                           double* partials, cudaStream_t st);
cudaError_t launch_reduce_power(const double* partials, int nblocks, double* lam_hist,
                                double* inv_norm, int iter, cudaStream_t st);
cudaError_t launch_sample_now(const DevProblem& pb, const double* u, double* out, cudaStream_t st);
int op_fp64_blocks(const DevProblem& pb);
// L2 eviction before a timed step: memset of the first half of buf, read of the second half
cudaError_t launch_l2_evict(void* buf, size_t bytes, cudaStream_t st);
// Launchers (kernels_tc.cu)
// scheme: 0 exact digit slices, 1 bf16 hi/lo three-pass, 2 bf16 one pass
// variant: tile shape (0 full MMA tile, 1 small tile; 1 only with scheme 0); ctas_per_sm:
// cap on the resident CTAs per SM of the persistent launch (0: as many as fit)
cudaError_t launch_op_tc(const DevProblem& pb, const double* u, double* out, int mode, int scheme, int variant,
                         cudaStream_t st, int ctas_per_sm = 0);
// Batched launch (exact scheme, CDM): every member advances one step; members[m] owns the
// global tiles [tile_start[m], tile_start[m + 1]).
cudaError_t launch_op_tc_batch(int dim, int p, int ncomp, int variant, const BatchMember* members,
                               const int* tile_start, int n_members, int total_tiles, BatchCtl* ctl,
                               cudaStream_t st);
// Launchers (kernels_tc64.cu): the FP64-grade tensor-core operator (CDM, start-up or apply
// mode); pb.Ycut must hold this input's cut-cell products (launch_cut_apply_fp64 first).
// Its tile shape is variant op_tc64_variant(dim) of op_tc_tiles.
cudaError_t launch_op_tc64(const DevProblem& pb, const double* u, double* out, int mode, cudaStream_t st);
int op_tc64_variant(int dim);
// One bounded mbarrier wait that runs out (nothing arrives): sets bit 1 of *flags.
cudaError_t launch_bounded_wait_probe(int* flags, int polls, cudaStream_t st);
bool op_tc_supported(int dim, int p, int ncomp);
void op_tc_tiles(int dim, int p, int ncomp, int variant, int* tile);
void op_tc_dims(int dim, int p, int ncomp, int* kp, int* np);
int op_tc_core_offset(int kp, int row, int k);
bool op_fp64_supported(int dim, int p, int ncomp);
void op_fp64_tiles(int dim, int p, int ncomp, int* tile);

}  // namespace ibfem
