// Newmark IMEX step on the GPU (Algorithm 2 of Buerchner et al., arXiv 2501.19013).
//
// Per step, after the fused kernel has advanced the d-DOFs explicitly (Eq. cdm) and
// written the c-DOF predictor Psi_pred^c = Psi^c + dt Psi'^c + (1/2 - beta) dt^2 Psi''^c
// (and Psi'_pred^c) into the new state buffer:
//   * imex_cell_apply : y_e = K^e x_e for every cell touching a c-DOF (one warp per cell,
//                       FP64), x = [Psi_{k+1}^d ; Psi_pred^c];
//   * imex_solve      : the forward and backward solves with the host Cholesky factor of
//                       S = M^cc + beta dt^2 K^cc by supernode blocks, one dependency-
//                       driven launch per sweep; the forward sweep forms the residual
//                       r = F^c_{k+1} - K^c Psi_pred of its rows (gathered in a fixed
//                       order), the backward sweep applies the Newmark correction
//                       Psi''^c = S^{-1} r, Psi'^c = Psi'_pred^c + gamma dt Psi''^c,
//                       Psi^c = Psi_pred^c + beta dt^2 Psi''^c to its rows and advances the
//                       step counter.
#include <algorithm>

#include "internal.h"

namespace ibfem {

__device__ __forceinline__ double ricker_imex(double t, double f_e) {
  const double pi = 3.141592653589793238462643383279502884;
  double ts = 2.0 * sqrt(6.0) / (pi * f_e);
  double q = pi * f_e * (t - ts);
  return (1.0 - 2.0 * q * q) * exp(-q * q);
}

// A new solve: both sweeps' tickets from zero, done flags of earlier solves stale.
__device__ __forceinline__ void sweep_begin(SweepCtl* ctl) {
  ctl->tick[0] = 0u;
  ctl->tick[1] = 0u;
  ctl->epoch += 1u;
}

template <int DIM, int P, int NC>
__global__ void __launch_bounds__(256) imex_cell_apply_kernel(DevProblem pb, ImexDev im, const double* __restrict__ x) {
  constexpr int NN1 = P + 1;
  constexpr int NL = (DIM == 2 ? NN1 * NN1 : NN1 * NN1 * NN1) * NC;
  __shared__ double xs[8][NL];
  if (blockIdx.x == 0 && threadIdx.x == 0) sweep_begin(im.ctl);   // the solve follows
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int slot = blockIdx.x * 8 + warp;
  if (slot >= im.n_cells) return;
  int64_t cell = im.cells[slot];
  int cx = (int)(cell % pb.n[0]);
  int cy = (int)((cell / pb.n[0]) % pb.n[1]);
  int cz = DIM == 3 ? (int)(cell / ((int64_t)pb.n[0] * pb.n[1])) : 0;
  for (int j = lane; j < NL; j += 32) {
    int node = j / NC, comp = j % NC;
    int a = node % NN1, b = (node / NN1) % NN1, c = DIM == 3 ? node / (NN1 * NN1) : 0;
    int64_t g = ((int64_t)(cz * P + c) * pb.lat[1] + (cy * P + b)) * pb.lat[0] + cx * P + a;
    xs[warp][j] = x[g * NC + comp];
  }
  __syncwarp();
  const int32_t ci = pb.cls[cell] == 1 ? pb.cut_index[cell] : 0;
  const double* K = pb.cls[cell] == 1 ? pb.Kcut + (size_t)(pb.cut_mat ? pb.cut_mat[ci] : ci) * NL * NL : pb.Kref;
  for (int i = lane; i < NL; i += 32) {
    double acc = 0.0;
    for (int j = 0; j < NL; ++j) acc = fma(K[(size_t)j * NL + i], xs[warp][j], acc);
    im.Y[(size_t)slot * NL + i] = acc;
  }
}

// Block triangular solves over the supernodes of the nested-dissection order (each leaf
// block and each separator, a contiguous run of at most 32 rows).  One launch per sweep:
// every CTA takes a ticket and with it the next task of a topological order of the
// supernodes (by height of the dissection tree where that order is topological); it loads
// what does not depend on other supernodes (its dense diagonal block, its rows' right-hand
// sides and its share of the factor's entries), then waits, with bounded polls, for the
// done flags of the supernodes its rows depend on (edges of the elimination tree between
// supernodes, all taken by lower tickets: CTAs already running, so every wait ends), and:
//   (1) sums its share of its rows' entries outside the diagonal block (forward: columns
//       before it; backward, rows of L^T: columns after it): the g CTAs of a supernode each
//       take the same fraction of every row, tpr threads per row with at most
//       kImexThreadEntries entries each (g fixed on the host), so that one round of
//       gathers of the solution follows the wait;
//   (2) with g > 1 stores its 32 partial sums and counts itself in; the last CTA to arrive
//       adds the partials in a fixed order (it does not depend on the arrival order) and
//       resets the counter;
//   (3) that CTA solves t_i = w_i - sum_i with the dense diagonal block by substitution in
//       registers, writes the block's rows back and releases the supernode's done flag
//       with the epoch of this solve.
// The solution vector is read through L2 only (ld.global.cg): rows become final while the
// kernel runs, and an L1 line could still hold a neighbour's earlier value.
// FWD: L y = b; else L^T x = y.
constexpr int kSnMax = 32;           // rows of a supernode (the host splits longer runs)
constexpr int kLevelThreads = 256;   // threads of a sweep CTA
constexpr int kSweepK = 8;           // entries per thread and row share (kImexThreadEntries)
constexpr int kSweepPolls = 1 << 21; // polls of one wait before it gives up (about 1 s)

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// atomic add with release (this CTA's partial sums, ordered before it by the block barrier)
// and acquire (the other CTAs' partial sums, for the last to arrive) semantics
__device__ __forceinline__ unsigned int atom_add_acq_rel_u32(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// STEP: the sweeps of an IMEX step: the forward sweep forms its rows' right-hand sides, the
// residual r = F^c_{k+1} - K^c Psi_pred (a fixed order per row), and the backward sweep
// applies the Newmark correction to its rows (and advances the step counter once); else
// the right-hand side is the work vector and the solution stays there.
template <bool FWD, bool STEP>
__global__ void __launch_bounds__(kLevelThreads) imex_sweep_kernel(DevProblem pb, ImexDev im, double* __restrict__ out) {
  __shared__ double S[kSnMax * kSnMax];
  __shared__ double T[kSnMax];
  __shared__ int ticket, last;
  const ImexSplitDev& sp = FWD ? im.fs : im.bs;
  if (threadIdx.x == 0) ticket = (int)atomicAdd(&im.ctl->tick[FWD ? 0 : 1], 1u);
  __syncthreads();
  if (ticket >= sp.n_tasks) {   // the tickets were not reset before this sweep
    if (threadIdx.x == 0) atomicOr(im.flags, 2);
    return;
  }
  const LevelTask tk = sp.task[ticket];
  const unsigned int ep = *((volatile unsigned int*)&im.ctl->epoch);
  const int st = tk.st, wd = tk.wd_tpr & 0xffff, tpr = tk.wd_tpr >> 16, c = tk.c, g = tk.g;
  double* __restrict__ w = im.work;
  // independent of other supernodes: the dense block (forward reads column j as row j of
  // DT, backward row j of D), the rows' right-hand sides (only this supernode writes them)
  // and the first round of this thread's entries
  const double* __restrict__ M = (FWD ? im.DT : im.D) + tk.doff;
  for (int e = threadIdx.x; e < wd * wd; e += kLevelThreads) S[e] = M[e];
  double rhs = 0.0;
  if (threadIdx.x < wd) {
    if (STEP && FWD) {
      const int64_t r = st + threadIdx.x;
      const unsigned long long k = *((volatile unsigned long long*)pb.step);
      const double fk1 = pb.f_e > 0.0 && im.Fc ? ricker_imex((double)(k + 1) * pb.dt, pb.f_e) : 0.0;
      double acc = im.Fc ? im.Fc[r] * fk1 : 0.0;
      for (int64_t e = im.g_ptr[r]; e < im.g_ptr[r + 1]; ++e) acc -= im.Y[im.g_idx[e]];
      rhs = acc;
    } else {
      rhs = __ldcg(w + st + threadIdx.x);
    }
  }
  if (STEP && !FWD && ticket == 0 && threadIdx.x == 0) *pb.step += 1ull;
  const int32_t* __restrict__ I = FWD ? im.Li : im.Ui;
  const double* __restrict__ X = FWD ? im.Lx : im.Ux;
  const int row = threadIdx.x / tpr, sub = threadIdx.x & (tpr - 1);
  int e0 = 0, e1 = 0;   // this thread's row share: entries [e0, e1)
  if (row < wd) {
    const int2 d = (FWD ? im.row_fdesc : im.row_bdesc)[st + row];
    const int len = d.y - d.x;
    e0 = d.x + (int)((int64_t)len * c / g);
    e1 = d.x + (int)((int64_t)len * (c + 1) / g);
  }
  double xv[kSweepK];
  int iv[kSweepK];
#pragma unroll
  for (int k = 0; k < kSweepK; ++k) {
    const int p = e0 + sub + k * tpr;
    xv[k] = p < e1 ? X[p] : 0.0;
    iv[k] = p < e1 ? I[p] : -1;
  }
  // the supernodes this one reads: relaxed polls, one acquire fence once they are done
  bool waited = false;
  for (int k = threadIdx.x; k < tk.dep_n; k += kLevelThreads) {
    const unsigned int* f = sp.done + sp.dep[tk.dep_beg + k];
    int it = 0;
    while (ld_relaxed_u32(f) != ep) {
      if (++it >= kSweepPolls) {
        atomicOr(im.flags, 2);
        break;
      }
      __nanosleep(32);
    }
    waited = true;
  }
  if (waited) fence_acq_rel_gpu();
  __syncthreads();
  // (1) this CTA's share of the off-block sums
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kSweepK; ++k)
    if (iv[k] >= 0) acc = fma(xv[k], __ldcg(w + iv[k]), acc);
  for (int p = e0 + sub + kSweepK * tpr; p < e1; p += tpr) acc = fma(X[p], __ldcg(w + I[p]), acc);
  for (int o = tpr >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, tpr);
  if (g == 1) {
    if (sub == 0 && row < wd) T[row] = acc;
  } else {
    // (2) partial sums; the last CTA of the supernode takes over
    if (sub == 0 && row < wd) im.part[tk.pbase + (int64_t)c * kSnMax + row] = acc;
    __syncthreads();
    unsigned int* cnt = im.cnt + (tk.pbase >> 5);
    if (threadIdx.x == 0) last = atom_add_acq_rel_u32(cnt, 1u) == (unsigned)(g - 1);
    __syncthreads();
    if (!last) return;
    // 8 threads per row, each over every 8th share in order, then a fixed shuffle tree
    const int r8 = threadIdx.x >> 3, q8 = threadIdx.x & 7;
    double s8 = 0.0;
    if (r8 < wd)
      for (int k = q8; k < g; k += 8) s8 += __ldcg(im.part + tk.pbase + (int64_t)k * kSnMax + r8);
    for (int o = 4; o > 0; o >>= 1) s8 += __shfl_down_sync(0xffffffffu, s8, o, 8);
    if (q8 == 0 && r8 < wd) T[r8] = s8;
    if (threadIdx.x == 0) *cnt = 0u;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  // (3) substitution with the block in registers: lane l holds row l; at step j lane j's
  // value is final, x_j = t_j / L_jj goes to every lane by a shuffle and the lanes below
  // (forward) or above (backward) subtract L_lj x_j (S[j wd + l]; S[l wd + l] = 1 / L_ll)
  const int lane = threadIdx.x;
  double t = lane < wd ? rhs - T[lane] : 0.0;
  const double dl = lane < wd ? S[lane * wd + lane] : 0.0;
  for (int jj = 0; jj < wd; ++jj) {
    const int j = FWD ? jj : wd - 1 - jj;
    const double a = S[j * wd + lane];   // in bounds: j wd + 31 < 32 x 32
    const double xj = __shfl_sync(0xffffffffu, t * dl, j);
    if (FWD ? (lane > j && lane < wd) : (lane < j)) t = fma(-a, xj, t);
  }
  const double x = t * dl;
  if (lane < wd) w[st + lane] = x;
  if (STEP && !FWD && lane < wd) {
    // Newmark correction of Algorithm 2 on this row: Psi''^c = x, Psi'^c += gamma dt x,
    // Psi^c = Psi_pred^c + beta dt^2 x
    const int64_t ci = im.perm[st + lane];
    im.ac[ci] = x;
    im.vc[ci] = fma(im.gamma_dt, x, im.vc[ci]);
    const int64_t dof = im.c_dof[ci];
    const double nv = fma(im.beta_dt2, x, out[dof]);
    out[dof] = nv;
    if (!isfinite(nv)) atomicOr(pb.flags, 1);
  }
  __syncwarp();
  if (lane == 0) st_release_u32(sp.done + tk.sn, ep);
}

// gather b[r] = in[c_dof[perm[r]]] * scal into work, or scatter out[c_dof[perm[r]]] = work[r]
__global__ void __launch_bounds__(256) imex_gather_kernel(ImexDev im, const double* __restrict__ in,
                                                          const double* __restrict__ scal) {
  const double sc = scal ? *scal : 1.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) sweep_begin(im.ctl);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < im.n_rows; r += (int64_t)gridDim.x * blockDim.x)
    im.work[r] = in[im.c_dof[im.perm[r]]] * sc;
}

__global__ void __launch_bounds__(256) imex_scatter_kernel(ImexDev im, double* __restrict__ out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < im.n_rows; r += (int64_t)gridDim.x * blockDim.x)
    out[im.c_dof[im.perm[r]]] = im.work[r];
}

static int rows_grid(const ImexDev& im) { return (int)std::min<int64_t>((im.n_rows + 255) / 256, 4096); }

// one sweep: one CTA per task
template <bool STEP>
static cudaError_t launch_sweep(const DevProblem* pb, const ImexDev& im, double* out, bool fwd, cudaStream_t st) {
  const int n = (fwd ? im.fs : im.bs).n_tasks;
  if (n <= 0) return cudaSuccess;
  const DevProblem none{};
  const DevProblem& p = pb ? *pb : none;
  if (fwd)
    imex_sweep_kernel<true, STEP><<<n, kLevelThreads, 0, st>>>(p, im, out);
  else
    imex_sweep_kernel<false, STEP><<<n, kLevelThreads, 0, st>>>(p, im, out);
  return cudaGetLastError();
}

// One triangular solve with the Cholesky factor L of S (permuted order), for the power
// iteration of the consistent-mass CDM (S = M^cc there): the right-hand side is
// b[r] = in[c_dof[perm[r]]] * scal, the solution of L w = b (forward) or of L^T w = b
// (backward) is written to out[c_dof[perm[r]]].
cudaError_t launch_imex_tri(const ImexDev& im, const double* in, const double* scal, double* out, bool backward,
                            cudaStream_t st) {
  if (im.n_rows == 0) return cudaSuccess;
  imex_gather_kernel<<<rows_grid(im), 256, 0, st>>>(im, in, scal);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_sweep<false>(nullptr, im, nullptr, !backward, st);
  if (e != cudaSuccess) return e;
  imex_scatter_kernel<<<rows_grid(im), 256, 0, st>>>(im, out);
  return cudaGetLastError();
}

#define IBFEM_IMEX_SHAPES(X) \
  X(2, 1, 1) X(2, 2, 1) X(2, 3, 1) X(2, 4, 1) X(2, 5, 1) X(2, 6, 1) \
  X(2, 1, 2) X(2, 2, 2) X(2, 3, 2) X(2, 4, 2) X(3, 1, 1) X(3, 2, 1) X(3, 3, 1)

cudaError_t launch_imex_cell_apply(const DevProblem& pb, const ImexDev& im, const double* x, cudaStream_t st) {
  if (im.n_cells == 0) return cudaSuccess;
  int blocks = (im.n_cells + 7) / 8;
#define X(D, P, N)                                                                   \
  if (pb.dim == D && pb.p == P && pb.ncomp == N) {                                   \
    imex_cell_apply_kernel<D, P, N><<<blocks, 256, 0, st>>>(pb, im, x);              \
    return cudaGetLastError();                                                       \
  }
  IBFEM_IMEX_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_imex_solve(const DevProblem& pb, const ImexDev& im, double* out, cudaStream_t st) {
  if (im.n_rows == 0) return cudaSuccess;
  cudaError_t e = launch_sweep<true>(&pb, im, out, true, st);
  if (e == cudaSuccess) e = launch_sweep<true>(&pb, im, out, false, st);
  return e;
}

}  // namespace ibfem
