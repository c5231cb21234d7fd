// Newmark IMEX step on the GPU (Algorithm 2 of Buerchner et al., arXiv 2501.19013).
//
// Per step, after the fused kernel has advanced the d-DOFs explicitly (Eq. cdm) and
// written the c-DOF predictor Psi_pred^c = Psi^c + dt Psi'^c + (1/2 - beta) dt^2 Psi''^c
// (and Psi'_pred^c) into the new state buffer:
//   * imex_cell_apply : y_e = K^e x_e for every cell touching a c-DOF (one warp per cell,
//                       FP64), x = [Psi_{k+1}^d ; Psi_pred^c];
//   * imex_solve      : one CTA per connected component of the c-set: the residual
//                       r = F^c_{k+1} - K^c Psi_pred gathered in a fixed order, the
//                       forward and backward solves with the host Cholesky factor of
//                       S = M^cc + beta dt^2 K^cc by supernode blocks, and the Newmark correction
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

// Block triangular solve of one component over the supernodes of its nested-dissection
// order, one height group at a time (a supernode depends only on the supernodes below it in
// the dissection tree, all in lower groups).  Per group: (1) every row with entries outside
// its supernode subtracts them, w_r -= sum_j L_rj w_j (forward: columns j before the
// supernode; backward, with L^T: rows j after it), 4, 8 or 32 lanes per row; (2) every supernode
// (at most 32 rows) solves with its dense diagonal block of L by substitution, one warp per
// supernode: the block is first copied to the warp's 32 x 32 shared-memory area with
// independent coalesced loads, then the warp walks its columns (forward) or rows
// (backward) while the lanes update the other rows; a block barrier after each part.
// FWD: L y = b; else L^T x = y.
constexpr int kSnMax = 32;   // rows of a supernode (the host splits longer runs)

template <bool FWD>
__device__ __forceinline__ void block_solve(const ImexDev& im, int g0, int g1, double* w, double* scratch,
                                            int lane, int warp, int nwarps) {
  const int64_t* __restrict__ I = FWD ? im.Li : im.Ui;
  const double* __restrict__ X = FWD ? im.Lx : im.Ux;
  double* const S = scratch + warp * kSnMax * kSnMax;
  for (int gi = 0; gi < g1 - g0; ++gi) {
    const int g = FWD ? g0 + gi : g1 - 1 - gi;
    const int4* __restrict__ desc = FWD ? im.hg_fdesc : im.hg_bdesc;
    const int q0 = FWD ? im.hg_frow_ptr[g] : im.hg_brow_ptr[g];
    const int q1 = FWD ? im.hg_frow_ptr[g + 1] : im.hg_brow_ptr[g + 1];
    // lpr lanes per row, 32 / lpr rows per warp at a time (the host picks lpr by the
    // group's longest row); a row's entries are strided over its lanes, four loads in flight
    const int lpr = FWD ? im.hg_flpr[g] : im.hg_blpr[g];
    const int rpw = 32 / lpr, sub = lane & (lpr - 1), slot = lane / lpr;
    for (int qb = q0 + warp * rpw; qb < q1; qb += nwarps * rpw) {
      const int q = qb + slot;
      double acc = 0.0;
      int r = -1;
      if (q < q1) {
        const int4 dq = desc[q];
        r = dq.x;
#pragma unroll 4
        for (int p = dq.y + sub; p < dq.z; p += lpr) acc = fma(X[p], w[I[p]], acc);
      }
      for (int o = lpr >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, lpr);
      if (sub == 0 && r >= 0) w[r] -= acc;
    }
    __syncthreads();
    for (int q = im.hg_sn_ptr[g] + warp; q < im.hg_sn_ptr[g + 1]; q += nwarps) {
      const int sn = im.hg_sn[q];
      double* __restrict__ ws = w + im.sn_start[sn];
      const int wd = im.sn_w[sn];
      // forward: column j of the block is row j of DT; backward: row j of L_ss is row j of D
      const double* __restrict__ M = (FWD ? im.DT : im.D) + im.sn_doff[sn];
      for (int e = lane; e < wd * wd; e += 32) S[e] = M[e];
      __syncwarp();
      for (int jj = 0; jj < wd; ++jj) {
        const int j = FWD ? jj : wd - 1 - jj;
        const double* Sj = S + j * wd;
        const double xj = ws[j] * Sj[j];   // Sj[j] = 1 / L_jj
        __syncwarp();
        if (lane == 0) ws[j] = xj;
        const int i = lane;
        if (FWD ? (i > j && i < wd) : (i < j)) ws[i] = fma(-Sj[i], xj, ws[i]);
        __syncwarp();
      }
      __syncwarp();   // the scratch is reused by the warp's next supernode
    }
    __syncthreads();
  }
}

// A component's rows only couple to rows of the same component, so its vector can live in
// shared memory, indexed by the permuted row (w = smem - r0).
// The first kImexWarps * 32 * 32 doubles of the dynamic shared memory are the warps'
// supernode scratch areas, the component's vector (when it fits) follows.
extern __shared__ double imex_smem[];
constexpr int kImexThreads = 512;
constexpr int kImexScratch = kImexThreads / 32 * kSnMax * kSnMax;

__global__ void __launch_bounds__(kImexThreads, 1) imex_solve_kernel(DevProblem pb, ImexDev im, double* __restrict__ out,
                                                                  int in_smem) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int r0 = im.comp_ptr[b], r1 = im.comp_ptr[b + 1];
  const unsigned long long k = *((volatile unsigned long long*)pb.step);
  double fk1 = 0.0;
  if (pb.f_e > 0.0 && im.Fc) fk1 = ricker_imex((double)(k + 1) * pb.dt, pb.f_e);
  double* w = in_smem ? imex_smem + kImexScratch - r0 : im.work;
  // residual r = F_{k+1}^c - K^c Psi_pred (fixed summation order)
  for (int r = r0 + tid; r < r1; r += blockDim.x) {
    double acc = im.Fc ? im.Fc[r] * fk1 : 0.0;
    for (int64_t e = im.g_ptr[r]; e < im.g_ptr[r + 1]; ++e) acc -= im.Y[im.g_idx[e]];
    w[r] = acc;
  }
  __syncthreads();
  // L y = r, then L^T x = y, by supernode height groups
  block_solve<true>(im, im.comp_hg[b], im.comp_hg[b + 1], w, imex_smem, lane, warp, nwarps);
  block_solve<false>(im, im.comp_hg[b], im.comp_hg[b + 1], w, imex_smem, lane, warp, nwarps);
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
__global__ void __launch_bounds__(kImexThreads) imex_tri_kernel(ImexDev im, const double* __restrict__ in,
                                                        const double* __restrict__ scal,
                                                        double* __restrict__ out, int backward, int in_smem) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int r0 = im.comp_ptr[b], r1 = im.comp_ptr[b + 1];
  const double sc = scal ? *scal : 1.0;
  double* w = in_smem ? imex_smem + kImexScratch - r0 : im.work;
  for (int r = r0 + tid; r < r1; r += blockDim.x) w[r] = in[im.c_dof[im.perm[r]]] * sc;
  __syncthreads();
  if (!backward)
    block_solve<true>(im, im.comp_hg[b], im.comp_hg[b + 1], w, imex_smem, lane, warp, nwarps);
  else
    block_solve<false>(im, im.comp_hg[b], im.comp_hg[b + 1], w, imex_smem, lane, warp, nwarps);
  for (int r = r0 + tid; r < r1; r += blockDim.x) out[im.c_dof[im.perm[r]]] = w[r];
}

// dynamic shared memory: the warps' scratch, then the largest component's vector if it fits
// (else the vector stays in the global work array)
static size_t imex_vec_bytes(const ImexDev& im) {
  const size_t bytes = (size_t)im.max_comp * sizeof(double);
  return bytes + kImexScratch * sizeof(double) <= (size_t)220 * 1024 ? bytes : 0;
}

template <typename KernelT>
static cudaError_t imex_smem_config(KernelT kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

cudaError_t launch_imex_tri(const ImexDev& im, const double* in, const double* scal, double* out, bool backward,
                            cudaStream_t st) {
  if (im.n_comp == 0) return cudaSuccess;
  static const cudaError_t cfg = imex_smem_config(imex_tri_kernel);
  if (cfg != cudaSuccess) return cfg;
  const size_t vb = imex_vec_bytes(im);
  imex_tri_kernel<<<im.n_comp, kImexThreads, kImexScratch * sizeof(double) + vb, st>>>(im, in, scal, out,
                                                                                     backward ? 1 : 0, vb > 0 ? 1 : 0);
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
  const size_t vb = imex_vec_bytes(im);
  imex_solve_kernel<<<im.n_comp, kImexThreads, kImexScratch * sizeof(double) + vb, st>>>(pb, im, out, vb > 0 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace ibfem
