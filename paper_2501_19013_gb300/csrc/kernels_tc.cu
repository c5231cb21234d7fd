// Mixed-precision element operator on the 5th-generation tensor cores, fused with the
// FP64 central-difference update (Eq. cdm of Buerchner et al., arXiv 2501.19013).
//
// One CTA per tile of cells; it owns the lattice nodes of its tile and recomputes the
// one-cell halo (as the FP64 kernel), so each node's sum over its cells is formed once, in
// a fixed order, without atomics.  Per CTA:
//   1. the FP64 node patch of u^k is read into shared memory;
//   2. the gathered element vectors X (one row per halo'd cell, M = 128 rows) are split
//      into TF32 hi/lo parts directly from the FP64 bit patterns (integer ops only) and
//      stored in the no-swizzle K-major core-matrix layout of a UMMA operand;
//   3. one thread issues tcgen05.mma kind::tf32: Y = X K_ref^T with the shared reference
//      matrix K_ref (hi/lo image prepared on the host) -- three passes hi*hi + hi*lo + lo*hi
//      for about FP32 accuracy, or one pass -- accumulating in TMEM (FP32);
//   4. four warps drain TMEM with tcgen05.ld into a shared FP32 buffer; cut cells replace
//      their rows with K^e x_e from their own FP32 matrices (CUDA cores);
//   5. per owned DOF: (K u)_i = sum of its cells' rows (FP32), delta = (dt^2/m_i)(F_i - (Ku)_i)
//      in FP32, widened to FP64 by bit manipulation, and u^{k+1} = (2 u^k - u^{k-1}) + delta
//      in FP64 -- two FP64 operations per DOF, the minimum for an FP64 state update.
// Block 0 also records the observer readings of u^k; the last block advances the step.
#include <cstdint>

#include "internal.h"

namespace ibfem {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// FP64 -> FP32 by truncating the significand (integer pipe only; values below the FP32
// normal range flush to zero, above it saturate to infinity).
__device__ __forceinline__ uint32_t f64_to_f32_bits(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  uint32_t sign = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7ffu) - 896;
  uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  if (e <= 0) return sign;
  if (e >= 255) return sign | 0x7f800000u;
  return sign | ((uint32_t)e << 23) | m;
}

// FP32 -> FP64 exactly by bit manipulation (subnormals flush to zero).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  uint32_t b = __float_as_uint(f);
  uint32_t sign = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  uint32_t hi, lo;
  if (e == 0) {
    hi = sign;
    lo = 0;
  } else if (e == 255) {
    hi = sign | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else {
    hi = sign | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double ricker_tc(double t, double f_e) {
  const double pi = 3.141592653589793238462643383279502884;
  double ts = 2.0 * sqrt(6.0) / (pi * f_e);
  double q = pi * f_e * (t - ts);
  return (1.0 - 2.0 * q * q) * exp(-q * q);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; base offset 0; no swizzle
  return d;
}

}  // namespace

// Tile geometry of the tensor-core kernel (halo'd cells <= 128 = M).
__host__ __device__ constexpr int tc_tile_x(int dim, int nl) { return dim == 3 ? 4 : (nl >= 32 ? 8 : 15); }
__host__ __device__ constexpr int tc_tile_y(int dim, int nl) { return dim == 3 ? 4 : (nl >= 32 ? 8 : 7); }
__host__ __device__ constexpr int tc_tile_z(int dim) { return dim == 3 ? 4 : 1; }

template <int DIM, int P, int NC>
struct TcCfg {
  static constexpr int NN1 = P + 1;
  static constexpr int NNL = DIM == 2 ? NN1 * NN1 : NN1 * NN1 * NN1;
  static constexpr int NL = NNL * NC;
  static constexpr int KP = (NL + 7) / 8 * 8;      // K padded to the tf32 MMA step
  static constexpr int NP = (NL + 15) / 16 * 16;   // N padded (M = 128 needs N % 16 == 0)
  static constexpr int TMEM_COLS = NP <= 32 ? 32 : (NP <= 64 ? 64 : (NP <= 128 ? 128 : 256));
  static constexpr int TX = tc_tile_x(DIM, NL), TY = tc_tile_y(DIM, NL), TZ = tc_tile_z(DIM);
  static constexpr int EX = TX + 1, EY = TY + 1, EZ = DIM == 3 ? TZ + 1 : 1;
  static constexpr int NE = EX * EY * EZ;
  static constexpr int PX = EX * P + 1, PY = EY * P + 1, PZ = DIM == 3 ? EZ * P + 1 : 1;
  static constexpr int PATCH = PX * PY * PZ * NC;
  static constexpr int LBO = 128;                   // bytes between K-adjacent core matrices
  static constexpr int SBO = (KP / 4) * 128;        // bytes between M/N-adjacent core matrices
  static constexpr int A_FLOATS = 128 * KP;
  static constexpr int B_FLOATS = NP * KP;
  static constexpr size_t OFF_A_HI = 0;
  static constexpr size_t OFF_A_LO = OFF_A_HI + 4 * (size_t)A_FLOATS;
  static constexpr size_t OFF_B_HI = OFF_A_LO + 4 * (size_t)A_FLOATS;
  static constexpr size_t OFF_B_LO = OFF_B_HI + 4 * (size_t)B_FLOATS;
  static constexpr size_t OFF_PATCH = (OFF_B_LO + 4 * (size_t)B_FLOATS + 15) / 16 * 16;
  static constexpr size_t OFF_OFF = OFF_PATCH + 8 * (size_t)PATCH;
  static constexpr size_t OFF_XS = (OFF_OFF + 4 * (size_t)NL + 15) / 16 * 16;   // 8 warps x NL f32
  static constexpr size_t OFF_BAR = (OFF_XS + 4 * (size_t)8 * NL + 15) / 16 * 16;
  static constexpr size_t SMEM = OFF_BAR + 32;
  static_assert(NE <= 128, "halo'd tile must fit one M = 128 MMA");
  static_assert((size_t)NE * NL <= (size_t)A_FLOATS, "element buffer aliases A_hi");
};

// core-matrix offset (in floats) of element (row, k) of a K-major operand with KP columns
template <int KP>
__host__ __device__ __forceinline__ int core_offset(int row, int k) {
  return (row >> 3) * (KP / 4) * 32 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

template <int DIM, int P, int NC>
__global__ void __launch_bounds__(256) op_tc_kernel(DevProblem pb, const double* __restrict__ u,
                                                    double* __restrict__ out, int mode, int passes) {
  using C = TcCfg<DIM, P, NC>;
  constexpr int NL = C::NL, NN1 = C::NN1, KP = C::KP, NP = C::NP;
  constexpr int EX = C::EX, EY = C::EY, PX = C::PX, PY = C::PY, PZ = C::PZ;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* A_hi = reinterpret_cast<float*>(smem + C::OFF_A_HI);
  float* A_lo = reinterpret_cast<float*>(smem + C::OFF_A_LO);
  float* B_hi = reinterpret_cast<float*>(smem + C::OFF_B_HI);
  float* B_lo = reinterpret_cast<float*>(smem + C::OFF_B_LO);
  double* patch = reinterpret_cast<double*>(smem + C::OFF_PATCH);
  int* off = reinterpret_cast<int*>(smem + C::OFF_OFF);
  float* xs = reinterpret_cast<float*>(smem + C::OFF_XS);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 8);
  float* ybuf = A_hi;  // reused once the MMAs have completed

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  const int bx = tile % pb.tc_tiles[0];
  const int by = (tile / pb.tc_tiles[0]) % pb.tc_tiles[1];
  const int bz = DIM == 3 ? tile / (pb.tc_tiles[0] * pb.tc_tiles[1]) : 0;
  const int X0 = bx * C::TX, Y0 = by * C::TY, Z0 = bz * C::TZ;
  const int X1 = min(X0 + C::TX, pb.n[0]), Y1 = min(Y0 + C::TY, pb.n[1]);
  const int Z1 = DIM == 3 ? min(Z0 + C::TZ, pb.n[2]) : 1;
  const int ox0 = X0 * P, ox1 = X1 * P + (X1 == pb.n[0] ? 1 : 0);
  const int oy0 = Y0 * P, oy1 = Y1 * P + (Y1 == pb.n[1] ? 1 : 0);
  const int oz0 = DIM == 3 ? Z0 * P : 0;
  const int oz1 = DIM == 3 ? Z1 * P + (Z1 == pb.n[2] ? 1 : 0) : 1;
  const int gx0 = (X0 - 1) * P, gy0 = (Y0 - 1) * P, gz0 = DIM == 3 ? (Z0 - 1) * P : 0;

  // ---- set-up: TMEM, barrier, observers, operands
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(C::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  unsigned long long k = 0;
  if (mode == kModeCDM) k = *((volatile unsigned long long*)pb.step);
  if (tile == 0 && mode == kModeCDM && pb.n_obs_rows > 0 && pb.ring_cap > 0) {
    for (int r = tid; r < pb.n_obs_rows; r += blockDim.x) {
      double acc = 0.0;
      for (int j = 0; j < pb.obs_nodes; ++j)
        acc += pb.obs_w[(size_t)r * pb.obs_nodes + j] * u[pb.obs_dof[(size_t)r * pb.obs_nodes + j]];
      pb.ring[(size_t)(k % (unsigned long long)pb.ring_cap) * pb.n_obs_rows + r] = acc;
    }
  }
  {
    const float4* bh = reinterpret_cast<const float4*>(pb.tc_bimg);
    const float4* bl = reinterpret_cast<const float4*>(pb.tc_bimg + C::B_FLOATS);
    float4* sh = reinterpret_cast<float4*>(B_hi);
    float4* sl = reinterpret_cast<float4*>(B_lo);
    for (int i = tid; i < C::B_FLOATS / 4; i += blockDim.x) {
      sh[i] = bh[i];
      sl[i] = bl[i];
    }
  }
  for (int j = tid; j < NL; j += blockDim.x) {
    int node = j / NC, comp = j % NC;
    int a = node % NN1, b = (node / NN1) % NN1, c = DIM == 3 ? node / (NN1 * NN1) : 0;
    off[j] = ((c * PY + b) * PX + a) * NC + comp;
  }
  for (int i = tid; i < C::PATCH; i += blockDim.x) {
    int comp = i % NC, node = i / NC;
    int px = node % PX, py = (node / PX) % PY, pz = node / (PX * PY);
    int gx = gx0 + px, gy = gy0 + py, gz = gz0 + pz;
    double v = 0.0;
    if (gx >= 0 && gx < pb.lat[0] && gy >= 0 && gy < pb.lat[1] && gz >= 0 && gz < pb.lat[2])
      v = u[(((int64_t)gz * pb.lat[1] + gy) * pb.lat[0] + gx) * NC + comp];
    patch[i] = v;
  }
  __syncthreads();

  // ---- gather X into the UMMA operand layout: a warp writes one 8 x 4 core matrix
  for (int idx = tid; idx < C::A_FLOATS; idx += blockDim.x) {
    int within = idx & 31, core = idx >> 5;
    int rg = core / (KP / 4), kg = core - rg * (KP / 4);
    int m = rg * 8 + (within >> 2), j = kg * 4 + (within & 3);
    uint32_t v = 0u;
    if (m < C::NE && j < NL) {
      int elx = m % EX, ely = (m / EX) % EY, elz = m / (EX * EY);
      const double* xe = patch + ((elz * P * PY + ely * P) * PX + elx * P) * NC;
      v = f64_to_f32_bits(xe[off[j]]);
    }
    uint32_t hi = v & 0xFFFFE000u;
    A_hi[idx] = __uint_as_float(hi);
    A_lo[idx] = __uint_as_float(v) - __uint_as_float(hi);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  // ---- MMA issue (one thread): Y[128 x NP] = X[128 x KP] K_ref^T
  if (tid == 0) {
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    const uint32_t a_op[3] = {smem_u32(A_hi), smem_u32(A_hi), smem_u32(A_lo)};
    const uint32_t b_op[3] = {smem_u32(B_hi), smem_u32(B_lo), smem_u32(B_hi)};
    int first = 1;
    for (int ps = 0; ps < passes; ++ps) {
      for (int kk = 0; kk < KP / 8; ++kk) {
        uint64_t da = umma_desc(a_op[ps] + kk * 2 * C::LBO, C::LBO, C::SBO);
        uint64_t db = umma_desc(b_op[ps] + kk * 2 * C::LBO, C::LBO, C::SBO);
        uint32_t acc = first ? 0u : 1u;
        first = 0;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(mbar)));
  }
  // bounded wait for the MMAs (phase 0)
  uint32_t ready = 0;
  for (int it = 0; it < (1 << 24) && !ready; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ready)
        : "r"(smem_u32(mbar)), "r"(0));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ready) {
    if (tid == 0) atomicOr(pb.flags, 2);  // timeout: report, skip the result
  } else if (warp < 4) {
    const int m = warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 16) {
      uint32_t r[16];
      uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < C::NE) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < NL) ybuf[m * NL + c0 + j] = __uint_as_float(r[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();

  // ---- cut and outside cells: replace their rows (one warp per cell)
  for (int m = warp; m < C::NE; m += 8) {
    int elx = m % EX, ely = (m / EX) % EY, elz = m / (EX * EY);
    int ex = X0 - 1 + elx, ey = Y0 - 1 + ely, ez = DIM == 3 ? Z0 - 1 + elz : 0;
    bool in_dom = ex >= 0 && ex < pb.n[0] && ey >= 0 && ey < pb.n[1] && (DIM == 2 || (ez >= 0 && ez < pb.n[2]));
    if (!in_dom) continue;
    int64_t cell = ((int64_t)ez * pb.n[1] + ey) * pb.n[0] + ex;
    uint8_t cl = pb.cls[cell];
    if (cl == 2) continue;
    if (cl == 0) {
      for (int i = lane; i < NL; i += 32) ybuf[m * NL + i] = 0.f;
      continue;
    }
    const double* xe = patch + ((elz * P * PY + ely * P) * PX + elx * P) * NC;
    float* xw = xs + warp * NL;
    for (int j = lane; j < NL; j += 32) xw[j] = __uint_as_float(f64_to_f32_bits(xe[off[j]]));
    __syncwarp();
    const float* K = pb.Kcut32 + (size_t)pb.cut_index[cell] * NL * NL;
    for (int i = lane; i < NL; i += 32) {
      float acc = 0.f;
#pragma unroll 4
      for (int j = 0; j < NL; ++j) acc = fmaf(K[(size_t)j * NL + i], xw[j], acc);
      ybuf[m * NL + i] = acc;
    }
    __syncwarp();
  }
  __syncthreads();

  // ---- node-centric assembly and the FP64 update
  const int nox = ox1 - ox0, noy = oy1 - oy0, noz = oz1 - oz0;
  const int n_own = nox * noy * noz * NC;
  double fk = 0.0;
  int src_lo = 0, src_hi = 0;
  if ((mode == kModeCDM || mode == kModeStartup) && pb.tsrc_ptr && pb.f_e > 0.0) {
    src_lo = pb.tsrc_ptr[tile];
    src_hi = pb.tsrc_ptr[tile + 1];
    if (src_hi > src_lo) fk = ricker_tc((double)k * pb.dt, pb.f_e);
  }
  bool bad = false;
  for (int i = tid; i < n_own; i += blockDim.x) {
    int comp = i % NC, node = i / NC;
    int gx = ox0 + node % nox, gy = oy0 + (node / nox) % noy, gz = oz0 + node / (nox * noy);
    int qx = gx / P, qy = gy / P, qz = gz / P;
    int exs[2], eys[2], ezs[2], nxe = 0, nye = 0, nze = 0;
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
    float ku = 0.f;
    for (int iz = 0; iz < nze; ++iz)
      for (int iy = 0; iy < nye; ++iy)
        for (int ix = 0; ix < nxe; ++ix) {
          int ex = exs[ix], ey = eys[iy], ez = ezs[iz];
          int el = ((DIM == 3 ? ez - (Z0 - 1) : 0) * EY + (ey - (Y0 - 1))) * EX + (ex - (X0 - 1));
          int lr = ((DIM == 3 ? (gz - ez * P) * NN1 : 0) + (gy - ey * P)) * NN1 + (gx - ex * P);
          ku += ybuf[el * NL + lr * NC + comp];
        }
    int64_t dof = (((int64_t)gz * pb.lat[1] + gy) * pb.lat[0] + gx) * NC + comp;
    if (mode == kModeApply) {
      out[dof] = f32_to_f64_bits(ku);
      continue;
    }
    float m32 = pb.minv32[dof];
    if (!(m32 > 0.f)) continue;
    float f = 0.f;
    for (int s2 = src_lo; s2 < src_hi; ++s2)
      if (pb.tsrc_dof[s2] == dof) f += (float)(pb.tsrc_val[s2] * fk);
    float d32 = m32 * (f - ku);
    if (!isfinite(d32)) bad = true;
    double delta = f32_to_f64_bits(d32);
    double uval = patch[(((gz - gz0) * PY + (gy - gy0)) * PX + (gx - gx0)) * NC + comp];
    if (mode == kModeCDM)
      out[dof] = fma(2.0, uval, -out[dof]) + delta;
    else
      out[dof] = uval - pb.dt * out[dof] + 0.5 * delta;
  }
  if (bad) atomicOr(pb.flags, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
  }
  if (mode == kModeCDM && tid == 0) {
    __threadfence();
    unsigned prev = atomicAdd(pb.done, 1u);
    if (prev == gridDim.x - 1) {
      *pb.step = k + 1;
      *pb.done = 0u;
      __threadfence();
    }
  }
}

// ------------------------------------------------------------------ host side
#define IBFEM_TC_SHAPES(X) X(2, 2, 1) X(2, 3, 1) X(2, 4, 1) X(2, 2, 2) X(2, 3, 2) X(2, 4, 2) X(3, 2, 1) X(3, 3, 1)

bool op_tc_supported(int dim, int p, int ncomp) {
#define X(D, P, N) if (dim == D && p == P && ncomp == N) return true;
  IBFEM_TC_SHAPES(X)
#undef X
  return false;
}

void op_tc_tiles(int dim, int p, int ncomp, int* t) {
  int nl = ncomp;
  for (int k = 0; k < dim; ++k) nl *= p + 1;
  t[0] = tc_tile_x(dim, nl);
  t[1] = tc_tile_y(dim, nl);
  t[2] = tc_tile_z(dim);
}

void op_tc_dims(int dim, int p, int ncomp, int* kp, int* np) {
  int nl = ncomp;
  for (int k = 0; k < dim; ++k) nl *= p + 1;
  *kp = (nl + 7) / 8 * 8;
  *np = (nl + 15) / 16 * 16;
}

int op_tc_core_offset(int kp, int row, int k) {
  return (row >> 3) * (kp / 4) * 32 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

template <int D, int P, int N>
static cudaError_t launch_tc_t(const DevProblem& pb, const double* u, double* out, int mode, int passes,
                               cudaStream_t st) {
  using C = TcCfg<D, P, N>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(op_tc_kernel<D, P, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int blocks = pb.tc_tiles[0] * pb.tc_tiles[1] * pb.tc_tiles[2];
  op_tc_kernel<D, P, N><<<blocks, 256, C::SMEM, st>>>(pb, u, out, mode, passes);
  return cudaGetLastError();
}

cudaError_t launch_op_tc(const DevProblem& pb, const double* u, double* out, int mode, int passes,
                         cudaStream_t st) {
#define X(D, P, N) \
  if (pb.dim == D && pb.p == P && pb.ncomp == N) return launch_tc_t<D, P, N>(pb, u, out, mode, passes, st);
  IBFEM_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace ibfem
