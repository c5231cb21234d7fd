// FP64 element-by-element operator and fused central-difference update (CUDA cores).
//
// One time step of Eq. cdm, u^{k+1} = 2u^k - u^{k-1} + dt^2 M_L^{-1} (F^k - K u^k), with
// K u = sum_e P_e^T K^e P_e u applied cell by cell (Sec. 2.2; Sec. 3.3 "right-hand side
// computation"):
//   * cut_apply  : y_e = K^e x_e for every cut cell (one warp per cell, K^e symmetric so
//                  lane i reads row j of K^e contiguously while forming (K^e x)_i);
//                  extra blocks record the observer readings Psi(x_i, t_k) (Sec. 3.2).
//   * op_fused   : one CTA per tile of cells; the CTA owns the lattice nodes of its tile
//                  and recomputes the one-cell halo, so every node's sum over its cells
//                  is formed by exactly one CTA in a fixed order (deterministic, no
//                  atomics); uncut cells contract the shared reference matrix K_ref held
//                  in shared memory; the epilogue applies the load, M_L^{-1} and the CDM
//                  update in place over u^{k-1}.
// The same fused kernel also provides K x (apply) and the power-iteration product
// M_L^{-1/2} K M_L^{-1/2} w with deterministic per-CTA partial sums (Sec. 2.3).
#include <cstdio>

#include <algorithm>

#include "internal.h"

namespace ibfem {

__device__ __forceinline__ double ricker_dev(double t, double f_e) {
  const double pi = 3.141592653589793238462643383279502884;
  double ts = 2.0 * sqrt(6.0) / (pi * f_e);
  double q = pi * f_e * (t - ts);
  return (1.0 - 2.0 * q * q) * exp(-q * q);
}

__device__ __forceinline__ double load_in(const OpInput& x, int64_t dof, double scal) {
  double v = x.in[dof];
  if (x.vec) v *= x.vec[dof];
  return v * scal;
}

template <int DIM, int P, int NC>
struct Shape {
  static constexpr int NN1 = P + 1;
  static constexpr int NNL = DIM == 2 ? NN1 * NN1 : NN1 * NN1 * NN1;
  static constexpr int NL = NNL * NC;
};

// Tile edge (cells) of the fused kernel per instantiation.
__host__ __device__ constexpr int tile_edge(int dim, int p, int nc) {
  return dim == 3 ? 4 : (p * nc >= 6 ? 8 : (p * nc >= 3 ? 12 : 16));
}

// ------------------------------------------------------------------ cut cells
template <int DIM, int P, int NC>
__global__ void __launch_bounds__(256) cut_apply_fp64_kernel(DevProblem pb, OpInput x,
                                                             int n_cut_blocks, int sample) {
  using S = Shape<DIM, P, NC>;
  constexpr int NL = S::NL, NN1 = S::NN1;
  __shared__ double xs[8][NL];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double scal = x.scal ? *x.scal : 1.0;
  if ((int)blockIdx.x < n_cut_blocks) {
    int ce = blockIdx.x * 8 + warp;
    if (ce >= pb.n_cut) return;
    int64_t cell = pb.cut_cell[ce];
    int cx = (int)(cell % pb.n[0]);
    int cy = (int)((cell / pb.n[0]) % pb.n[1]);
    int cz = DIM == 3 ? (int)(cell / ((int64_t)pb.n[0] * pb.n[1])) : 0;
    for (int j = lane; j < NL; j += 32) {
      int node = j / NC, comp = j % NC;
      int a = node % NN1, b = (node / NN1) % NN1, c = DIM == 3 ? node / (NN1 * NN1) : 0;
      int64_t g = ((int64_t)(cz * P + c) * pb.lat[1] + (cy * P + b)) * pb.lat[0] + cx * P + a;
      xs[warp][j] = load_in(x, g * NC + comp, scal);
    }
    __syncwarp();
    const double* K = pb.Kcut + (size_t)(pb.cut_mat ? pb.cut_mat[ce] : ce) * NL * NL;
    for (int i0 = 0; i0 < NL; i0 += 32) {
      int i = i0 + lane;
      if (i < NL) {
        double acc = 0.0;
#pragma unroll 4
        for (int j = 0; j < NL; ++j) acc = fma(K[(size_t)j * NL + i], xs[warp][j], acc);
        pb.Ycut[(size_t)ce * NL + i] = acc;
      }
    }
    return;
  }
  if (!sample || pb.n_obs_rows == 0 || pb.ring_cap == 0) return;
  int r = (blockIdx.x - n_cut_blocks) * blockDim.x + threadIdx.x;
  if (r >= pb.n_obs_rows) return;
  unsigned long long k = *((volatile unsigned long long*)pb.step);
  double acc = 0.0;
  for (int j = 0; j < pb.obs_nodes; ++j) {
    int64_t d = pb.obs_dof[(size_t)r * pb.obs_nodes + j];
    acc += pb.obs_w[(size_t)r * pb.obs_nodes + j] * x.in[d];
  }
  pb.ring[(size_t)(k % (unsigned long long)pb.ring_cap) * pb.n_obs_rows + r] = acc;
}

__global__ void sample_now_kernel(DevProblem pb, const double* u, double* out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= pb.n_obs_rows) return;
  double acc = 0.0;
  for (int j = 0; j < pb.obs_nodes; ++j) {
    int64_t d = pb.obs_dof[(size_t)r * pb.obs_nodes + j];
    acc += pb.obs_w[(size_t)r * pb.obs_nodes + j] * u[d];
  }
  out[r] = acc;
}

// ------------------------------------------------------------------ fused tile kernel
template <int DIM, int P, int NC>
struct FusedCfg {
  using S = Shape<DIM, P, NC>;
  static constexpr int T = tile_edge(DIM, P, NC);
  static constexpr int EX = T + 1, EY = T + 1, EZ = DIM == 3 ? T + 1 : 1;
  static constexpr int PX = EX * P + 1, PY = EY * P + 1, PZ = DIM == 3 ? EZ * P + 1 : 1;
  static constexpr int NE = EX * EY * EZ;
  static constexpr int PATCH = PX * PY * PZ * NC;
  static constexpr size_t SMEM = sizeof(double) * ((size_t)PATCH + (size_t)NE * S::NL +
                                                   (size_t)S::NL * S::NL) +
                                 sizeof(int) * S::NL + 64;
};

template <int DIM, int P, int NC>
__global__ void __launch_bounds__(256) op_fp64_kernel(DevProblem pb, OpInput x, double* __restrict__ out,
                                                      int mode, double* partials) {
  using S = Shape<DIM, P, NC>;
  using C = FusedCfg<DIM, P, NC>;
  constexpr int NL = S::NL, NN1 = S::NN1, T = C::T;
  constexpr int EX = C::EX, EY = C::EY, EZ = C::EZ, PX = C::PX, PY = C::PY, PZ = C::PZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* patch = reinterpret_cast<double*>(smem_raw);
  double* ybuf = patch + C::PATCH;
  double* kref = ybuf + (size_t)C::NE * NL;
  int* off = reinterpret_cast<int*>(kref + NL * NL);

  const int tid = threadIdx.x, nth = blockDim.x;
  const int tile = blockIdx.x;
  const int bx = tile % pb.tiles[0];
  const int by = (tile / pb.tiles[0]) % pb.tiles[1];
  const int bz = DIM == 3 ? tile / (pb.tiles[0] * pb.tiles[1]) : 0;
  const int X0 = bx * T, Y0 = by * T, Z0 = bz * T;
  const int X1 = min(X0 + T, pb.n[0]), Y1 = min(Y0 + T, pb.n[1]);
  const int Z1 = DIM == 3 ? min(Z0 + T, pb.n[2]) : 1;
  const int ox0 = X0 * P, ox1 = X1 * P + (X1 == pb.n[0] ? 1 : 0);
  const int oy0 = Y0 * P, oy1 = Y1 * P + (Y1 == pb.n[1] ? 1 : 0);
  const int oz0 = DIM == 3 ? Z0 * P : 0;
  const int oz1 = DIM == 3 ? Z1 * P + (Z1 == pb.n[2] ? 1 : 0) : 1;
  const int gx0 = (X0 - 1) * P, gy0 = (Y0 - 1) * P, gz0 = DIM == 3 ? (Z0 - 1) * P : 0;
  const double scal = x.scal ? *x.scal : 1.0;

  for (int i = tid; i < NL * NL; i += nth) kref[i] = pb.Kref[i];
  for (int j = tid; j < NL; j += nth) {
    int node = j / NC, comp = j % NC;
    int a = node % NN1, b = (node / NN1) % NN1, c = DIM == 3 ? node / (NN1 * NN1) : 0;
    off[j] = ((c * PY + b) * PX + a) * NC + comp;
  }
  for (int i = tid; i < C::PATCH; i += nth) {
    int comp = i % NC, node = i / NC;
    int px = node % PX, py = (node / PX) % PY, pz = node / (PX * PY);
    int gx = gx0 + px, gy = gy0 + py, gz = gz0 + pz;
    double v = 0.0;
    if (gx >= 0 && gx < pb.lat[0] && gy >= 0 && gy < pb.lat[1] && gz >= 0 && gz < pb.lat[2]) {
      int64_t dof = (((int64_t)gz * pb.lat[1] + gy) * pb.lat[0] + gx) * NC + comp;
      v = load_in(x, dof, scal);
    }
    patch[i] = v;
  }
  __syncthreads();

  // element contributions of the cells touching owned nodes (rows of owned nodes only)
  for (int w = tid; w < C::NE * NL; w += nth) {
    int el = w / NL, row = w - el * NL;
    int elx = el % EX, ely = (el / EX) % EY, elz = el / (EX * EY);
    int ex = X0 - 1 + elx, ey = Y0 - 1 + ely, ez = DIM == 3 ? Z0 - 1 + elz : 0;
    double y = 0.0;
    bool in_dom = ex >= 0 && ex < pb.n[0] && ey >= 0 && ey < pb.n[1] && (DIM == 2 || (ez >= 0 && ez < pb.n[2]));
    if (in_dom) {
      int rn = row / NC;
      int a = rn % NN1, b = (rn / NN1) % NN1, c = DIM == 3 ? rn / (NN1 * NN1) : 0;
      int gx = ex * P + a, gy = ey * P + b, gz = ez * P + c;
      bool owned = gx >= ox0 && gx < ox1 && gy >= oy0 && gy < oy1 && gz >= oz0 && gz < oz1;
      if (owned) {
        int64_t cell = ((int64_t)ez * pb.n[1] + ey) * pb.n[0] + ex;
        uint8_t cl = pb.cls[cell];
        if (cl == 2) {
          const double* xe = patch + ((elz * P * PY + ely * P) * PX + elx * P) * NC;
          const double* kr = kref + row * NL;
          double acc = 0.0;
#pragma unroll 5
          for (int j = 0; j < NL; ++j) acc = fma(kr[j], xe[off[j]], acc);
          y = acc;
        } else if (cl == 1) {
          y = pb.Ycut[(size_t)pb.cut_index[cell] * NL + row];
        }
      }
    }
    ybuf[w] = y;
  }
  __syncthreads();

  // node-centric assembly + epilogue
  const int nox = ox1 - ox0, noy = oy1 - oy0, noz = oz1 - oz0;
  const int n_own = nox * noy * noz * NC;
  double part_wz = 0.0, part_zz = 0.0;
  bool bad = false;
  double fk = 0.0;
  unsigned long long k = 0;
  int src_lo = 0, src_hi = 0;
  if (mode == kModeCDM || mode == kModeStartup || mode == kModeImex) {
    k = *((volatile unsigned long long*)pb.step);
    if (pb.src_ptr && pb.f_e > 0.0) {
      src_lo = pb.src_ptr[tile];
      src_hi = pb.src_ptr[tile + 1];
      if (src_hi > src_lo) fk = ricker_dev((double)k * pb.dt, pb.f_e);
    }
  }
  for (int i = tid; i < n_own; i += nth) {
    int comp = i % NC, node = i / NC;
    int gx = ox0 + node % nox, gy = oy0 + (node / nox) % noy, gz = oz0 + node / (nox * noy);
    double ku = 0.0;
    int exs[2], eys[2], ezs[2], nxe = 0, nye = 0, nze = 0;
    int qx = gx / P, qy = gy / P, qz = gz / P;
    if (DIM == 3) {
      if (gz % P == 0 && qz - 1 >= 0) ezs[nze++] = qz - 1;
      if (qz < pb.n[2]) ezs[nze++] = qz;
    } else {
      ezs[nze++] = 0;
    }
    if (gy % P == 0 && qy - 1 >= 0) eys[nye++] = qy - 1;
    if (qy < pb.n[1]) eys[nye++] = qy;
    if (gx % P == 0 && qx - 1 >= 0) exs[nxe++] = qx - 1;
    if (qx < pb.n[0]) exs[nxe++] = qx;
    for (int iz = 0; iz < nze; ++iz)
      for (int iy = 0; iy < nye; ++iy)
        for (int ix = 0; ix < nxe; ++ix) {
          int ex = exs[ix], ey = eys[iy], ez = ezs[iz];
          int el = ((DIM == 3 ? ez - (Z0 - 1) : 0) * EY + (ey - (Y0 - 1))) * EX + (ex - (X0 - 1));
          int lr = (((gz - ez * P) * NN1 + (gy - ey * P)) * NN1 + (gx - ex * P)) * NC + comp;
          if (DIM == 2) lr = ((gy - ey * P) * NN1 + (gx - ex * P)) * NC + comp;
          ku += ybuf[el * NL + lr];
        }
    int64_t dof = (((int64_t)gz * pb.lat[1] + gy) * pb.lat[0] + gx) * NC + comp;
    double uval = patch[(((gz - gz0) * PY + (gy - gy0)) * PX + (gx - gx0)) * NC + comp];
    if (mode == kModeApply) {
      out[dof] = ku;
    } else if (mode == kModePower) {
      double z = pb.sinv[dof] * ku;
      out[dof] = z;
      double wv = x.in[dof] * scal;
      part_wz += wv * z;
      part_zz += z * z;
    } else {
      double m = pb.minv[dof];
      if (m > 0.0) {
        double f = 0.0;
        for (int s2 = src_lo; s2 < src_hi; ++s2)
          if (pb.src_dof[s2] == dof) f += pb.src_val[s2] * fk;
        double r = f - ku;
        double nv;
        if (mode == kModeStartup)
          nv = uval - pb.dt * out[dof] + 0.5 * m * r;
        else
          nv = fma(2.0, uval, -out[dof]) + m * r;
        out[dof] = nv;
        if (!isfinite(nv)) bad = true;
      } else if (m < 0.0 && mode == kModeImex) {
        // c-DOF: Newmark predictor of Algorithm 2 (beta = 1/4, gamma = 1/2)
        int64_t ci = (int64_t)(-m) - 1;
        double a = pb.imex_ac[ci], v = pb.imex_vc[ci];
        out[dof] = uval + pb.dt * v + pb.imex_c1 * a;
        pb.imex_vc[ci] = v + pb.imex_c2 * a;
      }
    }
  }
  if (bad) atomicOr(pb.flags, 1);
  if (mode == kModePower) {
    // deterministic block reduction
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
      part_wz += __shfl_down_sync(0xffffffffu, part_wz, o);
      part_zz += __shfl_down_sync(0xffffffffu, part_zz, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = part_wz;
      red[1][tid >> 5] = part_zz;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int wi = 0; wi < (nth + 31) / 32; ++wi) {
        a += red[0][wi];
        b += red[1][wi];
      }
      partials[2 * tile] = a;
      partials[2 * tile + 1] = b;
    }
  }
  if (mode == kModeCDM) {
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
}

__global__ void reduce_power_kernel(const double* partials, int nblocks, double* lam_hist,
                                     double* inv_norm, int iter) {
  __shared__ double sa[256], sb[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    lam_hist[iter] = sa[0];
    *inv_norm = sb[0] > 0.0 ? 1.0 / sqrt(sb[0]) : 0.0;
  }
}

// out = s .* in * (scal ? *scal : 1) over n entries
__global__ void scale_vec_kernel(int64_t n, const double* __restrict__ sv, const double* __restrict__ in,
                                 const double* __restrict__ scal, double* __restrict__ out) {
  const double sc = scal ? *scal : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = sv[i] * in[i] * sc;
}

// per-block partial sums (fixed order) of (a * scal) . b and b . b
__global__ void dot2_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ scal,
                            const double* __restrict__ b, double* __restrict__ partials) {
  __shared__ double sa[256], sb[256];
  const double sc = scal ? *scal : 1.0;
  double x = 0.0, y = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x = fma(a[i] * sc, b[i], x);
    y = fma(b[i], b[i], y);
  }
  sa[threadIdx.x] = x;
  sb[threadIdx.x] = y;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sa[0];
    partials[2 * blockIdx.x + 1] = sb[0];
  }
}

cudaError_t launch_scale_vec(int64_t n, const double* s, const double* in, const double* scal, double* out,
                             cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  scale_vec_kernel<<<blocks, 256, 0, st>>>(n, s, in, scal, out);
  return cudaGetLastError();
}

cudaError_t launch_dot2(int64_t n, const double* a, const double* scal, const double* b, double* partials,
                        int nblocks, cudaStream_t st) {
  dot2_kernel<<<nblocks, 256, 0, st>>>(n, a, scal, b, partials);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ dispatch
#define IBFEM_FOR_EACH_SHAPE(X) \
  X(2, 1, 1) X(2, 2, 1) X(2, 3, 1) X(2, 4, 1) X(2, 5, 1) X(2, 6, 1) \
  X(2, 1, 2) X(2, 2, 2) X(2, 3, 2) X(2, 4, 2) X(3, 1, 1) X(3, 2, 1) X(3, 3, 1)

bool op_fp64_supported(int dim, int p, int ncomp) {
#define X(D, P, N) if (dim == D && p == P && ncomp == N) return true;
  IBFEM_FOR_EACH_SHAPE(X)
#undef X
  return false;
}

void op_fp64_tiles(int dim, int p, int ncomp, int* t) {
  int e = tile_edge(dim, p, ncomp);
  t[0] = t[1] = e;
  t[2] = dim == 3 ? e : 1;
}

int op_fp64_blocks(const DevProblem& pb) { return pb.tiles[0] * pb.tiles[1] * pb.tiles[2]; }

template <int D, int P, int N>
static cudaError_t launch_op_t(const DevProblem& pb, OpInput x, double* out, int mode,
                               double* partials, cudaStream_t st) {
  using C = FusedCfg<D, P, N>;
  // thread-safe one-time configuration (function-local static initialisation)
  static const cudaError_t configured =
      cudaFuncSetAttribute(op_fp64_kernel<D, P, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (configured != cudaSuccess) return configured;
  op_fp64_kernel<D, P, N><<<op_fp64_blocks(pb), 256, C::SMEM, st>>>(pb, x, out, mode, partials);
  return cudaGetLastError();
}

template <int D, int P, int N>
static cudaError_t launch_cut_t(const DevProblem& pb, OpInput x, bool sample, cudaStream_t st, bool do_cut) {
  int ncb = do_cut ? (pb.n_cut + 7) / 8 : 0;
  int nsb = sample && pb.n_obs_rows > 0 ? (pb.n_obs_rows + 255) / 256 : 0;
  if (ncb + nsb == 0) return cudaSuccess;
  cut_apply_fp64_kernel<D, P, N><<<ncb + nsb, 256, 0, st>>>(pb, x, ncb, sample ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_op_fp64(const DevProblem& pb, OpInput x, double* out, int mode,
                           double* partials, cudaStream_t st) {
#define X(D, P, N) \
  if (pb.dim == D && pb.p == P && pb.ncomp == N) return launch_op_t<D, P, N>(pb, x, out, mode, partials, st);
  IBFEM_FOR_EACH_SHAPE(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_cut_apply_fp64(const DevProblem& pb, OpInput x, bool sample, cudaStream_t st, bool do_cut) {
#define X(D, P, N) \
  if (pb.dim == D && pb.p == P && pb.ncomp == N) return launch_cut_t<D, P, N>(pb, x, sample, st, do_cut);
  IBFEM_FOR_EACH_SHAPE(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_reduce_power(const double* partials, int nblocks, double* lam_hist,
                                double* inv_norm, int iter, cudaStream_t st) {
  reduce_power_kernel<<<1, 256, 0, st>>>(partials, nblocks, lam_hist, inv_norm, iter);
  return cudaGetLastError();
}

// Reads `n` 16-byte words (an L2 eviction: the lines it brings in are clean); a thread writes
// its xor to `sink` (a word of the flush buffer itself) only if it equals one arbitrary value,
// so that the loads cannot be dropped and almost nothing is written.
__global__ void l2_evict_read_kernel(const uint4* __restrict__ p, size_t n, unsigned* sink) {
  uint32_t acc = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint4 v = p[i];
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x9E3779B9u) *sink = acc;
}

cudaError_t launch_l2_evict(void* buf, size_t bytes, cudaStream_t st) {
  const size_t half = bytes / 2 / 16 * 16;
  if (half == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(buf, 0x5a, half, st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  l2_evict_read_kernel<<<sms * 4, 512, 0, st>>>(reinterpret_cast<const uint4*>(static_cast<char*>(buf) + half), half / 16,
                                              static_cast<unsigned*>(buf));
  return cudaGetLastError();
}

cudaError_t launch_sample_now(const DevProblem& pb, const double* u, double* out, cudaStream_t st) {
  if (pb.n_obs_rows == 0) return cudaSuccess;
  sample_now_kernel<<<(pb.n_obs_rows + 127) / 128, 128, 0, st>>>(pb, u, out);
  return cudaGetLastError();
}

}  // namespace ibfem
