// Newmark IMEX step on the GPU (Algorithm 2 of Buerchner et al., arXiv 2501.19013).
//
// Per step, after the fused kernel has advanced the d-DOFs explicitly (Eq. cdm) and
// written the c-DOF predictor Psi_pred^c = Psi^c + dt Psi'^c + (1/2 - beta) dt^2 Psi''^c
// (and Psi'_pred^c) into the new state buffer:
//   * imex_cell_apply : y_e = K^e x_e for every cell touching a c-DOF (one warp per cell,
//                       FP64), x = [Psi_{k+1}^d ; Psi_pred^c];
//   * imex_solve      : one CTA per connected component of the c-set: the residual
//                       r = F^c_{k+1} - K^c Psi_pred gathered in a fixed order, the
//                       level-scheduled forward and backward solves with the host Cholesky
//                       factor of S = M^cc + beta dt^2 K^cc, and the Newmark correction
//                       Psi''^c = S^{-1} r, Psi'^c = Psi'_pred^c + gamma dt Psi''^c,
//                       Psi^c = Psi_pred^c + beta dt^2 Psi''^c.  The last CTA advances the
//                       step counter.
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

// Level-scheduled triangular solve of one component (rows of a level are independent, one
// warp per row, a block barrier between levels).  FWD: L y = b with the diagonal stored last
// in each CSR row of L; else L^T x = y with the CSR rows of L^T, diagonal first.  The first
// row of every warp in the next level -- its column indices, values (first 32) and 1/L_rr --
// is fetched before the current level is solved, so after a barrier only the gathers of w
// (shared memory when the component fits) remain on the critical path.
template <bool FWD>
__device__ __forceinline__ void level_solve(int l0, int l1, const int4* __restrict__ sched,
                                            const int32_t* __restrict__ lvl, const int32_t* __restrict__ rows,
                                            const int64_t* __restrict__ P, const int64_t* __restrict__ I,
                                            const double* __restrict__ X, const double* __restrict__ dinv,
                                            double* w, int lane, int warp, int nwarps) {
  // sched[lv * 32 + warp] = {row, first entry, end, rows in the level} of the warp's first row
  // of level lv (row -1: none).  Software pipeline: the schedule entry of level lv + 2 and
  // the entries (first 128) and 1/L_rr of level lv + 1 are loaded while level lv is solved,
  // so after a barrier only the gathers of w (shared memory) wait.
  constexpr int PF = 4;
  const int4 none = make_int4(-1, 0, 0, 0);
  int li[PF], li_n[PF];
  double lx[PF], lx_n[PF], dv = 0.0, dv_n = 0.0;
  auto load_row = [&](const int4 e, int* L, double* V, double& d) {
    if (e.x < 0) return;
#pragma unroll
    for (int c = 0; c < PF; ++c) {
      const int p = e.y + lane + 32 * c;
      if (p < e.z) {
        L[c] = (int)I[p];
        V[c] = X[p];
      }
    }
    d = dinv[e.x];
  };
  int4 sA = l0 < l1 ? sched[(size_t)l0 * 32 + warp] : none;
  int4 sB = l0 + 1 < l1 ? sched[(size_t)(l0 + 1) * 32 + warp] : none;
  load_row(sA, li, lx, dv);
  for (int lv = l0; lv < l1; ++lv) {
    const int4 sC = lv + 2 < l1 ? sched[(size_t)(lv + 2) * 32 + warp] : none;
    load_row(sB, li_n, lx_n, dv_n);
    if (sA.x >= 0) {
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < PF; ++c)
        if (sA.y + lane + 32 * c < sA.z) acc = fma(lx[c], w[li[c]], acc);
      for (int p = sA.y + lane + 32 * PF; p < sA.z; p += 32) acc = fma(X[p], w[I[p]], acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) w[sA.x] = (w[sA.x] - acc) * dv;
    }
    if (sA.w > nwarps) {   // levels wider than the warps: the other rows, fetched on demand
      const int q0 = lvl[lv], q1 = lvl[lv + 1];
      for (int q = q0 + warp + nwarps; q < q1; q += nwarps) {
        const int rr = rows[q];
        const int64_t a0 = FWD ? P[rr] : P[rr] + 1, a1 = FWD ? P[rr + 1] - 1 : P[rr + 1];
        double acc = 0.0;
        for (int64_t p = a0 + lane; p < a1; p += 32) acc = fma(X[p], w[I[p]], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) w[rr] = (w[rr] - acc) * dinv[rr];
      }
    }
    __syncthreads();
    sA = sB;
    sB = sC;
#pragma unroll
    for (int c = 0; c < PF; ++c) {
      li[c] = li_n[c];
      lx[c] = lx_n[c];
    }
    dv = dv_n;
  }
}

// A component's rows only couple to rows of the same component, so its vector can live in
// shared memory, indexed by the permuted row (w = smem - r0).
extern __shared__ double imex_smem[];

__global__ void __launch_bounds__(1024) imex_solve_kernel(DevProblem pb, ImexDev im, double* __restrict__ out,
                                                          int in_smem) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int r0 = im.comp_ptr[b], r1 = im.comp_ptr[b + 1];
  const unsigned long long k = *((volatile unsigned long long*)pb.step);
  double fk1 = 0.0;
  if (pb.f_e > 0.0 && im.Fc) fk1 = ricker_imex((double)(k + 1) * pb.dt, pb.f_e);
  double* w = in_smem ? imex_smem - r0 : im.work;
  // residual r = F_{k+1}^c - K^c Psi_pred (fixed summation order)
  for (int r = r0 + tid; r < r1; r += blockDim.x) {
    double acc = im.Fc ? im.Fc[r] * fk1 : 0.0;
    for (int64_t e = im.g_ptr[r]; e < im.g_ptr[r + 1]; ++e) acc -= im.Y[im.g_idx[e]];
    w[r] = acc;
  }
  __syncthreads();
  // L y = r, then L^T x = y, level by level
  level_solve<true>(im.comp_flvl[b], im.comp_flvl[b + 1], im.f_sched, im.f_lvl, im.f_rows, im.Lp, im.Li, im.Lx,
                    im.dinv, w, lane, warp, nwarps);
  level_solve<false>(im.comp_blvl[b], im.comp_blvl[b + 1], im.b_sched, im.b_lvl, im.b_rows, im.Up, im.Ui, im.Ux,
                     im.dinv, w, lane, warp, nwarps);
  // Newmark correction on the c-DOFs
  bool bad = false;
  for (int r = r0 + tid; r < r1; r += blockDim.x) {
    int64_t ci = im.perm[r];
    double a = w[r];
    im.ac[ci] = a;
    im.vc[ci] = fma(im.gamma_dt, a, im.vc[ci]);
    int64_t dof = im.c_dof[ci];
    double nv = fma(im.beta_dt2, a, out[dof]);
    out[dof] = nv;
    if (!isfinite(nv)) bad = true;
  }
  if (bad) atomicOr(pb.flags, 1);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    unsigned prev = atomicAdd(pb.done, 1u);
    if (prev == gridDim.x - 1) {
      *pb.step = k + 1;
      *pb.done = 0u;
      __threadfence();
    }
  }
}

// One triangular solve with the Cholesky factor L of S (permuted order), for the power
// iteration of the consistent-mass CDM (S = M^cc there): one CTA per component; the right-
// hand side is b[r] = in[c_dof[perm[r]]] * scal, the solution of L w = b (forward) or of
// L^T w = b (backward) is written to out[c_dof[perm[r]]].
__global__ void __launch_bounds__(1024, 1) imex_tri_kernel(ImexDev im, const double* __restrict__ in,
                                                        const double* __restrict__ scal,
                                                        double* __restrict__ out, int backward, int in_smem) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int r0 = im.comp_ptr[b], r1 = im.comp_ptr[b + 1];
  const double sc = scal ? *scal : 1.0;
  double* w = in_smem ? imex_smem - r0 : im.work;
  for (int r = r0 + tid; r < r1; r += blockDim.x) w[r] = in[im.c_dof[im.perm[r]]] * sc;
  __syncthreads();
  if (!backward)
    level_solve<true>(im.comp_flvl[b], im.comp_flvl[b + 1], im.f_sched, im.f_lvl, im.f_rows, im.Lp, im.Li, im.Lx,
                      im.dinv, w, lane, warp, nwarps);
  else
    level_solve<false>(im.comp_blvl[b], im.comp_blvl[b + 1], im.b_sched, im.b_lvl, im.b_rows, im.Up, im.Ui, im.Ux,
                       im.dinv, w, lane, warp, nwarps);
  for (int r = r0 + tid; r < r1; r += blockDim.x) out[im.c_dof[im.perm[r]]] = w[r];
}

// dynamic shared memory for the largest component's vector (0: the global work vector)
static size_t imex_smem_bytes(const ImexDev& im) {
  const size_t bytes = (size_t)im.max_comp * sizeof(double);
  return bytes <= (size_t)200 * 1024 ? bytes : 0;
}

template <typename KernelT>
static cudaError_t imex_smem_config(KernelT kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_imex_tri(const ImexDev& im, const double* in, const double* scal, double* out, bool backward,
                            cudaStream_t st) {
  if (im.n_comp == 0) return cudaSuccess;
  static const cudaError_t cfg = imex_smem_config(imex_tri_kernel);
  if (cfg != cudaSuccess) return cfg;
  const size_t sm = imex_smem_bytes(im);
  imex_tri_kernel<<<im.n_comp, 1024, sm, st>>>(im, in, scal, out, backward ? 1 : 0, sm > 0 ? 1 : 0);
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
  if (im.n_comp == 0) return cudaSuccess;
  static const cudaError_t cfg = imex_smem_config(imex_solve_kernel);
  if (cfg != cudaSuccess) return cfg;
  const size_t sm = imex_smem_bytes(im);
  imex_solve_kernel<<<im.n_comp, 1024, sm, st>>>(pb, im, out, sm > 0 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace ibfem
