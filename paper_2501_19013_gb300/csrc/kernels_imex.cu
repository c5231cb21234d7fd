// Newmark IMEX step on the GPU (Algorithm 2 of Buerchner et al., arXiv 2501.19013).
//
// Per step, after the fused kernel has advanced the d-DOFs explicitly (Eq. cdm) and
// written the c-DOF predictor Psi_pred^c = Psi^c + dt Psi'^c + (1/2 - beta) dt^2 Psi''^c
// (and Psi'_pred^c) into the new state buffer:
//   * imex_cell_apply : y_e = K^e x_e for every cell touching a c-DOF (one warp per cell,
//                       FP64), x = [Psi_{k+1}^d ; Psi_pred^c];
//   * imex_solve      : the residual r = F^c_{k+1} - K^c Psi_pred gathered in a fixed
//                       order, the forward and backward solves with the host Cholesky
//                       factor of S = M^cc + beta dt^2 K^cc by supernode blocks (one launch
//                       per height of the dissection tree), and the Newmark correction
//                       Psi''^c = S^{-1} r, Psi'^c = Psi'_pred^c + gamma dt Psi''^c,
//                       Psi^c = Psi_pred^c + beta dt^2 Psi''^c, which advances the step
//                       counter.
#include <algorithm>

#include "internal.h"

namespace ibfem {

__device__ __forceinline__ double ricker_imex(double t, double f_e) {
  const double pi = 3.141592653589793238462643383279502884;
  double ts = 2.0 * sqrt(6.0) / (pi * f_e);
  double q = pi * f_e * (t - ts);
  return (1.0 - 2.0 * q * q) * exp(-q * q);
}

template <int DIM, int P, int NC>
__global__ void __launch_bounds__(256) imex_cell_apply_kernel(DevProblem pb, ImexDev im, const double* __restrict__ x) {
  constexpr int NN1 = P + 1;
  constexpr int NL = (DIM == 2 ? NN1 * NN1 : NN1 * NN1 * NN1) * NC;
  __shared__ double xs[8][NL];
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
// block and each separator, a contiguous run of at most 32 rows, depends only on the
// supernodes below it in the dissection tree).  One launch per tree height, over every
// component: the launches of lower (forward) or higher (backward) heights have completed,
// so every row a supernode reads is final.  For each supernode:
//   (1) its rows' entries outside the diagonal block (forward: columns before it; backward,
//       rows of L^T: columns after it) are summed by g CTAs, each taking the same fraction
//       of every row, with 4, 8 or 32 lanes on a row (g and the lanes fixed on the host by
//       the entry counts: the separators near the top of the tree reach far back and get
//       many CTAs);
//   (2) with g > 1 each CTA stores its 32 partial sums and counts itself in; the last CTA
//       to arrive adds the partials in share order (the sum does not depend on the arrival
//       order) and resets the counter;
//   (3) that CTA solves t_i = w_i - sum_i with the dense diagonal block by substitution in
//       shared memory (walking its columns forward, its rows backward, lanes over the other
//       rows) and writes the block's rows back.
// FWD: L y = b; else L^T x = y.  No CTA waits on another.
constexpr int kSnMax = 32;          // rows of a supernode (the host splits longer runs)
constexpr int kLevelThreads = 256;  // threads of a level CTA

template <bool FWD>
__global__ void __launch_bounds__(kLevelThreads) imex_level_kernel(ImexDev im, int c0) {
  __shared__ double S[kSnMax * kSnMax];
  __shared__ double T[kSnMax];
  __shared__ int last;
  const ImexSplitDev& sp = FWD ? im.fs : im.bs;
  const int2 task = sp.cta[c0 + blockIdx.x];
  const int sn = task.x, c = task.y;
  const int g = sp.g[sn];
  const int64_t st = im.sn_start[sn];
  const int wd = im.sn_w[sn];
  double* __restrict__ w = im.work;
  const double* __restrict__ M = (FWD ? im.DT : im.D) + im.sn_doff[sn];
  // the dense block (forward reads column j as row j of DT, backward row j of D)
  if (g == 1)
    for (int e = threadIdx.x; e < wd * wd; e += kLevelThreads) S[e] = M[e];
  // (1) this CTA's share of the off-block sums
  const int64_t* __restrict__ I = FWD ? im.Li : im.Ui;
  const double* __restrict__ X = FWD ? im.Lx : im.Ux;
  const int2* __restrict__ desc = FWD ? im.row_fdesc : im.row_bdesc;
  const int lpr = sp.lpr[sn];
  const int slots = kLevelThreads / lpr, slot = threadIdx.x / lpr, sub = threadIdx.x & (lpr - 1);
  double* __restrict__ part = im.part + (g > 1 ? sp.pbase[sn] + (int64_t)c * kSnMax : 0);
  for (int i0 = 0; i0 < wd; i0 += slots) {
    const int i = i0 + slot;
    double acc = 0.0;
    if (i < wd) {
      const int2 d = desc[st + i];
      const int len = d.y - d.x;
      const int pb = d.x + (int)((int64_t)len * c / g), pe = d.x + (int)((int64_t)len * (c + 1) / g);
#pragma unroll 4
      for (int p = pb + sub; p < pe; p += lpr) acc = fma(X[p], w[I[p]], acc);
    }
    for (int o = lpr >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, lpr);
    if (sub == 0 && i < wd) {
      if (g == 1)
        T[i] = w[st + i] - acc;
      else
        part[i] = acc;
    }
  }
  if (g > 1) {
    // (2) the last CTA of the supernode takes over
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&im.cnt[sn], 1u) == (unsigned)(g - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int e = threadIdx.x; e < wd * wd; e += kLevelThreads) S[e] = M[e];
    const double* __restrict__ p0 = im.part + sp.pbase[sn];
    if (threadIdx.x < wd) {
      double acc = 0.0;
      for (int k = 0; k < g; ++k) acc += __ldcg(p0 + (int64_t)k * kSnMax + threadIdx.x);
      T[threadIdx.x] = w[st + threadIdx.x] - acc;
    }
    if (threadIdx.x == 0) im.cnt[sn] = 0u;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  // (3) substitution with the block (Sj[j] holds 1 / L_jj)
  const int lane = threadIdx.x;
  for (int jj = 0; jj < wd; ++jj) {
    const int j = FWD ? jj : wd - 1 - jj;
    const double* Sj = S + j * wd;
    const double xj = T[j] * Sj[j];
    __syncwarp();
    if (lane == 0) T[j] = xj;
    if (FWD ? (lane > j && lane < wd) : (lane < j)) T[lane] = fma(-Sj[lane], xj, T[lane]);
    __syncwarp();
  }
  if (lane < wd) w[st + lane] = T[lane];
}

// r = F^c_{k+1} - K^c Psi_pred on the permuted rows (a fixed summation order per row)
__global__ void __launch_bounds__(256) imex_residual_kernel(DevProblem pb, ImexDev im) {
  const unsigned long long k = *((volatile unsigned long long*)pb.step);
  double fk1 = 0.0;
  if (pb.f_e > 0.0 && im.Fc) fk1 = ricker_imex((double)(k + 1) * pb.dt, pb.f_e);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < im.n_rows; r += (int64_t)gridDim.x * blockDim.x) {
    double acc = im.Fc ? im.Fc[r] * fk1 : 0.0;
    for (int64_t e = im.g_ptr[r]; e < im.g_ptr[r + 1]; ++e) acc -= im.Y[im.g_idx[e]];
    im.work[r] = acc;
  }
}

// Newmark correction on the c-DOFs: Psi''^c = S^{-1} r (in work), Psi'^c += gamma dt Psi''^c,
// Psi^c = Psi_pred^c + beta dt^2 Psi''^c; one thread advances the step counter
__global__ void __launch_bounds__(256) imex_correct_kernel(DevProblem pb, ImexDev im, double* __restrict__ out) {
  bool bad = false;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < im.n_rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ci = im.perm[r];
    const double a = im.work[r];
    im.ac[ci] = a;
    im.vc[ci] = fma(im.gamma_dt, a, im.vc[ci]);
    const int64_t dof = im.c_dof[ci];
    const double nv = fma(im.beta_dt2, a, out[dof]);
    out[dof] = nv;
    if (!isfinite(nv)) bad = true;
  }
  if (bad) atomicOr(pb.flags, 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) *pb.step += 1ull;
}

// gather b[r] = in[c_dof[perm[r]]] * scal into work, or scatter out[c_dof[perm[r]]] = work[r]
__global__ void __launch_bounds__(256) imex_gather_kernel(ImexDev im, const double* __restrict__ in,
                                                          const double* __restrict__ scal) {
  const double sc = scal ? *scal : 1.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < im.n_rows; r += (int64_t)gridDim.x * blockDim.x)
    im.work[r] = in[im.c_dof[im.perm[r]]] * sc;
}

__global__ void __launch_bounds__(256) imex_scatter_kernel(ImexDev im, double* __restrict__ out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < im.n_rows; r += (int64_t)gridDim.x * blockDim.x)
    out[im.c_dof[im.perm[r]]] = im.work[r];
}

static int rows_grid(const ImexDev& im) { return (int)std::min<int64_t>((im.n_rows + 255) / 256, 4096); }

// the launches of one triangular solve, height by height (the CTA ranges live on the host)
static cudaError_t launch_levels(const ImexDev& im, bool fwd, cudaStream_t st) {
  const int32_t* ptr = fwd ? im.fs.cta_ptr_host : im.bs.cta_ptr_host;
  for (int hh = 0; hh < im.n_heights; ++hh) {
    const int h = fwd ? hh : im.n_heights - 1 - hh;
    const int c0 = ptr[h], n = ptr[h + 1] - ptr[h];
    if (n <= 0) continue;
    if (fwd)
      imex_level_kernel<true><<<n, kLevelThreads, 0, st>>>(im, c0);
    else
      imex_level_kernel<false><<<n, kLevelThreads, 0, st>>>(im, c0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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
  if (e == cudaSuccess) e = launch_levels(im, !backward, st);
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
  imex_residual_kernel<<<rows_grid(im), 256, 0, st>>>(pb, im);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_levels(im, true, st);
  if (e == cudaSuccess) e = launch_levels(im, false, st);
  if (e != cudaSuccess) return e;
  imex_correct_kernel<<<rows_grid(im), 256, 0, st>>>(pb, im, out);
  return cudaGetLastError();
}

}  // namespace ibfem
