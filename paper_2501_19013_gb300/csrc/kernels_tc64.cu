// FP64-grade element operator on the tensor cores, fused with the FP64 central-difference
// update (Eq. cdm of Buerchner et al., arXiv 2501.19013), for sm_103a (tcgen05 + TMEM).
//
// The exact-slice product of the mixed path (kernels_tc.cu) carried to FP64 precision:
//   x_j  = 2^(E - 1077) sum_{s<7} d_s 2^(48 - 8 s)      (E: the largest biased exponent of
//   K_ij = 2^(G - 54)   sum_{t<7} c_t 2^(48 - 8 t)       the tile's node patch; G: of K_ref)
// with balanced 8-bit digits (|digit| <= 128: 55 significant bits of each operand, exact
// in BF16).  The 28 digit pairs of the levels l = s + t <= 6 run as tcgen05 kind::f16 MMA
// chains into seven FP32 TMEM accumulators; every level is an integer sum below 2^24, so
// the accumulation is exact.  The dropped levels (l >= 7) are below 2^-54 of the largest
// product.  One exponent for all of K_ref (instead of one per row) puts every element
// product of a tile on one fixed-point scale, so the node sums over the cells of a node are
// integer sums, exact: levels 0-3 as integers (packed in pairs), levels 4-6 folded into one
// FP32 tail (2^-56 relative).  K u is rounded once, in FP64, after the cancellation of the
// element contributions:
//   K u = 2^(E + G - 1059) (H + T 2^-8),  H = sum over cells of (V0 2^24 + V1 2^16 + V2 2^8 + V3)
// and u^{k+1} = fma(c, H, fma(c, T 2^-8, fma(2, u^k, -u^{k-1}))) with c = -(dt^2/m) 2^(E+G-1059):
// four FP64 operations per DOF.  Cut cells take K^e x_e from the FP64 cut-cell kernel that
// runs before this one (written to global memory) and enter the node sums in FP64: a cut
// cell's rows can be many orders of magnitude below the tile's scale (the fictitious part,
// alpha = 1e-12), while the lumped mass of a DOF it alone carries is as small, so such a
// row needs FP64's relative precision, not the tile's absolute one.
// The persistent tile loop, the halo recompute and the node ownership follow kernels_tc.cu.
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tc_common.cuh"

namespace ibfem {

using namespace tc;

namespace {

constexpr int kThreads64 = 512;

// Balanced 8-bit digits of round(|x| 2^(1077 - em)) (< 2^55) of an FP64 x whose biased
// exponent is at most em, the sign applied to every digit, packed as seven BF16 values
// (slices 0..6 in the halves of .x .y .z and the low half of .w).  Integer operations only.
__device__ __forceinline__ uint4 fp64_digits7(double x, int em) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((bits >> 52) & 0x7ffull);
  unsigned long long V = 0;
  if (eb > 0) {
    const unsigned long long m53 = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = em - eb - 2;   // V = m53 2^(-sh)
    if (sh < 0) {
      V = m53 << (-sh);
    } else if (sh == 0) {
      V = m53;
    } else if (sh < 55) {
      V = (m53 >> sh) + ((m53 >> (sh - 1)) & 1ull);
    }
  }
  const uint32_t lo = (uint32_t)V, hi = (uint32_t)(V >> 32);
  int d[7];
  int c = 0;
#pragma unroll
  for (int i = 0; i < 7; ++i) {   // byte i of V is digit 6 - i
    const uint32_t w = i < 4 ? lo : hi;
    int t = (int)((w >> (8 * (i & 3))) & 0xffu) + c;
    if (i < 6) {
      c = t >= 128 ? 1 : 0;
      t -= c << 8;
    }
    d[6 - i] = t;
  }
  if (bits >> 63) {
#pragma unroll
    for (int s = 0; s < 7; ++s) d[s] = -d[s];
  }
  return make_uint4(bf16x2_of_small_ints(d[0], d[1]), bf16x2_of_small_ints(d[2], d[3]),
                    bf16x2_of_small_ints(d[4], d[5]), bf16x2_of_small_ints(d[6], 0));
}

// an integer-valued FP32 accumulator (|v| < 2^22) as an int (exact; see f32_bits_of_small_int)
__device__ __forceinline__ int small_int_of_f32(float v) {
  return (int)__float_as_uint(v + 12582912.0f) - 0x4B400000;
}

// FP64 value of an int64 |h| < 2^51 (exact): the pattern of 1.5 * 2^52 plus h, minus 1.5 * 2^52
__device__ __forceinline__ double f64_of_i64(long long h) {
  return __longlong_as_double(0x4338000000000000ll + h) - 6755399441055744.0;
}

// x 2^z for a normal FP64 x (exponent arithmetic on the bits; 0 when the result would
// leave the normal range downwards)
__device__ __forceinline__ double f64_scale2(double x, int z) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return 0.0;
  const int e2 = e + z;
  if (e2 <= 0) return 0.0;
  if (e2 >= 2047) return x * 1e308 * 1e308;   // overflow: infinity with x's sign
  return __longlong_as_double(b + ((long long)z << 52));
}

}  // namespace

template <int DIM, int P, int NC>
struct Tc64Cfg {
  static constexpr int NN1 = P + 1;
  static constexpr int NNL = DIM == 2 ? NN1 * NN1 : NN1 * NN1 * NN1;
  static constexpr int NL = NNL * NC;
  static constexpr int KP = (NL + 15) / 16 * 16;
  static constexpr int NP = (NL + 15) / 16 * 16;
  static constexpr int NLEV = 7;
  static constexpr int TMEM_COLS = NLEV * NP <= 128 ? 128 : (NLEV * NP <= 256 ? 256 : 512);
  static constexpr int VARIANT = DIM == 3 ? 1 : 0;   // tile shape (the 3D full tile needs too much shared memory)
  static constexpr int TX = tc_tile_x(DIM, NL, VARIANT), TY = tc_tile_y(DIM, NL, VARIANT), TZ = tc_tile_z(DIM, VARIANT);
  static constexpr int EX = TX + 1, EY = TY + 1, EZ = DIM == 3 ? TZ + 1 : 1;
  static constexpr int NE = EX * EY * EZ;
  static constexpr int PX = EX * P + 1, PY = EY * P + 1, PZ = DIM == 3 ? EZ * P + 1 : 1;
  static constexpr int PATCH = PX * PY * PZ * NC;
  static constexpr int LBO = 128;
  static constexpr int SBO = (KP / 8) * 128;
  static constexpr int A_SLICE = 128 * KP;
  static constexpr int B_SLICE = NP * KP;
  static constexpr int A_SLOTS = 4;
  static constexpr size_t A_BYTES = 2 * (size_t)A_SLOTS * A_SLICE;
  static constexpr size_t B_BYTES = 2 * (size_t)NLEV * B_SLICE;
  static constexpr size_t Y_BYTES = 16 * (size_t)NE * NL;   // int4 {V0 2^8 + V1, V2 2^8 + V3, tail, 0}
  static constexpr bool Y_ALIAS = Y_BYTES <= A_BYTES;
  static constexpr size_t OFF_A = 0;
  static constexpr size_t OFF_B = OFF_A + A_BYTES;
  static constexpr size_t OFF_Y = Y_ALIAS ? 0 : OFF_B + B_BYTES;
  static constexpr size_t OFF_P = ((Y_ALIAS ? OFF_B + B_BYTES : OFF_Y + Y_BYTES) + 15) / 16 * 16;
  static constexpr size_t PATCH_BYTES = (8 * (size_t)PATCH + 15) / 16 * 16;
  static constexpr size_t OFF_D = OFF_P + 2 * PATCH_BYTES;   // digits: uint4 per value
  static constexpr size_t OFF_I = OFF_D + 16 * (size_t)PATCH;  // ints: lists, exponents
  static constexpr size_t OFF_CI = OFF_I + 4 * (8 + 16 + 128);   // int cut index per halo cell (-1: not cut)
  static constexpr size_t OFF_OFF = OFF_CI + 4 * 128;
  static constexpr size_t OFF_BAR = (OFF_OFF + 4 * (size_t)KP + 15) / 16 * 16;
  static constexpr size_t SMEM = OFF_BAR + 64;
  static_assert(NE <= 128, "halo'd tile must fit one M = 128 MMA");
  static_assert(NLEV * NP <= 512, "accumulators must fit the TMEM columns");
  static_assert(SMEM <= 232448 - 1024, "shared memory");
  static_assert(NL <= 85, "levels 0-2 of the digit sums must stay below 2^22");
};

// One CTA per SM takes tiles from the global counter (CTA b starts with tile b); mode is
// kModeCDM, kModeStartup, kModeApply or kModeImex (Algorithm 2's explicit part: the CDM
// update on the d-DOFs, which only uncut cells carry, and the Newmark predictor on the
// c-DOFs, marked by dt^2/m = -(c + 1)).  Except in kModeImex the cut-cell products pb.Ycut
// of this input must be in global memory before the launch.
template <int DIM, int P, int NC>
__global__ void __launch_bounds__(kThreads64, 1) op_tc64_kernel(const __grid_constant__ DevProblem pb,
                                                             const double* __restrict__ u,
                                                             double* __restrict__ out, int mode) {
  using C = Tc64Cfg<DIM, P, NC>;
  constexpr int NL = C::NL, NN1 = C::NN1, KP = C::KP, NP = C::NP;
  constexpr int EX = C::EX, EY = C::EY, PX = C::PX, PY = C::PY;
  constexpr int NV = C::PATCH;
  constexpr int NT = kThreads64, NW = NT / 32;
  // levels 3 and up may exceed 2^22: exact conversion by the conversion pipe unless the
  // bound (l + 1) NL 2^14 < 2^22 holds
  constexpr bool MAGIC3 = 4 * NL < 256;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint16_t* A = reinterpret_cast<uint16_t*>(smem + C::OFF_A);
  uint16_t* B = reinterpret_cast<uint16_t*>(smem + C::OFF_B);
  int4* yb = reinterpret_cast<int4*>(smem + C::OFF_Y);
  auto pbuf = [&](int which) { return reinterpret_cast<double*>(smem + C::OFF_P + which * C::PATCH_BYTES); };
  uint4* dig = reinterpret_cast<uint4*>(smem + C::OFF_D);
  int* ib = reinterpret_cast<int*>(smem + C::OFF_I);
  int* wmax = ib;             // [NW] per-warp exponent maxima
  int* next_tile = ib + 16;   // next global tile, its tile in processing order
  int* next_local = ib + 17;
  int* n_special = ib + 18;
  int* special = ib + 24;     // cut / outside cells of the halo'd tile
  int* off = reinterpret_cast<int*>(smem + C::OFF_OFF);
  int* cidx = reinterpret_cast<int*>(smem + C::OFF_CI);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);   // 0: B copy, 1/2: MMA phases
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 32);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_tiles = pb.tc_tiles[0] * pb.tc_tiles[1] * pb.tc_tiles[2];
  int* const tcount = pb.tile_counter;

  auto issue_patch = [&](int t, double* patch) {
    const int ibx = t % pb.tc_tiles[0];
    const int iby = (t / pb.tc_tiles[0]) % pb.tc_tiles[1];
    const int ibz = DIM == 3 ? t / (pb.tc_tiles[0] * pb.tc_tiles[1]) : 0;
    const int hx0 = (ibx * C::TX - 1) * P, hy0 = (iby * C::TY - 1) * P;
    const int hz0 = DIM == 3 ? (ibz * C::TZ - 1) * P : 0;
    for (int node = tid; node < NV / NC; node += NT) {
      int px = node % PX, py = (node / PX) % PY, pz = node / (PX * PY);
      int gx = hx0 + px, gy = hy0 + py, gz = hz0 + pz;
      bool in = gx >= 0 && gx < pb.lat[0] && gy >= 0 && gy < pb.lat[1] && gz >= 0 && gz < pb.lat[2];
      int64_t g = in ? (((int64_t)gz * pb.lat[1] + gy) * pb.lat[0] + gx) * NC : 0;
      cp_async_zfill<8 * NC>(patch + node * NC, u + g, in ? 8 * NC : 0);
    }
  };
  // global index of halo cell m of tile t (-1 outside the domain)
  auto halo_cell = [&](int t, int m) -> int64_t {
    const int tbx = t % pb.tc_tiles[0];
    const int tby = (t / pb.tc_tiles[0]) % pb.tc_tiles[1];
    const int tbz = DIM == 3 ? t / (pb.tc_tiles[0] * pb.tc_tiles[1]) : 0;
    const int elx = m % EX, ely = (m / EX) % EY, elz = m / (EX * EY);
    const int ex = tbx * C::TX - 1 + elx, ey = tby * C::TY - 1 + ely, ez = DIM == 3 ? tbz * C::TZ - 1 + elz : 0;
    const bool in_dom =
        ex >= 0 && ex < pb.n[0] && ey >= 0 && ey < pb.n[1] && (DIM == 2 || (ez >= 0 && ez < pb.n[2]));
    return in_dom ? ((int64_t)ez * pb.n[1] + ey) * pb.n[0] + ex : -1;
  };
  auto halo_class = [&](int t, int m) -> int {
    const int tbx = t % pb.tc_tiles[0];
    const int tby = (t / pb.tc_tiles[0]) % pb.tc_tiles[1];
    const int tbz = DIM == 3 ? t / (pb.tc_tiles[0] * pb.tc_tiles[1]) : 0;
    const int elx = m % EX, ely = (m / EX) % EY, elz = m / (EX * EY);
    const int ex = tbx * C::TX - 1 + elx, ey = tby * C::TY - 1 + ely, ez = DIM == 3 ? tbz * C::TZ - 1 + elz : 0;
    const bool in_dom =
        ex >= 0 && ex < pb.n[0] && ey >= 0 && ey < pb.n[1] && (DIM == 2 || (ez >= 0 && ez < pb.n[2]));
    return in_dom ? (int)pb.cls[((int64_t)ez * pb.n[1] + ey) * pb.n[0] + ex] : 0;
  };
  auto order = [&](int g) { return pb.tc_order ? pb.tc_order[g] : g; };

  // ---- once per CTA: TMEM, barriers, the K_ref digits (bulk copy), gather offsets
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(C::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int b = 0; b < 3; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[b])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
    const uint32_t bytes = (uint32_t)C::B_BYTES;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bars[0])), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(B)),
                 "l"(pb.tc_bimg), "r"(bytes), "r"(smem_u32(&bars[0]))
                 : "memory");
  }
  int pcur = 0;
  {
    const int t0 = order((int)blockIdx.x);
    issue_patch(t0, pbuf(0));
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (tid == 0) {
      *next_tile = (int)blockIdx.x;
      *next_local = t0;
    }
  }
  for (int j = tid; j < KP; j += NT) {
    int node = j / NC, comp = j % NC;
    int a = node % NN1, b = (node / NN1) % NN1, c = DIM == 3 ? node / (NN1 * NN1) : 0;
    off[j] = j < NL ? ((c * PY + b) * PX + a) * NC + comp : -1;
  }
  unsigned long long k = 0;
  if (mode == kModeCDM) k = *((volatile unsigned long long*)pb.step);
  double fk = 0.0;
  if (mode == kModeImex) k = *((volatile unsigned long long*)pb.step);
  if ((mode == kModeCDM || mode == kModeStartup || mode == kModeImex) && pb.tsrc_ptr && pb.f_e > 0.0)
    fk = ricker_tc((double)k * pb.dt, pb.f_e);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  uint32_t aS[C::A_SLOTS];
#pragma unroll
  for (int q = 0; q < C::A_SLOTS; ++q) aS[q] = smem_u32(A + q * C::A_SLICE);
  const uint32_t bS0 = smem_u32(B);
  bool ok = true, bimg_ready = false, bad = false;
  uint32_t mma_phase = 0;
  constexpr int KG = KP / 8;
  constexpr int ROWS = (C::NE + 7) / 8 * 8;
  constexpr int ITEMS = ROWS * KG;

  // A operand of digit slices [s0, s0 + ns) into slots 0.. (one 16-byte core-matrix row per item)
  auto gather = [&](int s0, int ns) {
    for (int item = tid; item < ITEMS; item += NT) {
      const int r8 = item & 7, rest = item >> 3;
      const int kg = rest % KG, rg = rest / KG;
      const int m = rg * 8 + r8;
      uint32_t w[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) w[a][b] = 0u;
      if (m < C::NE) {
        const int elx = m % EX, ely = (m / EX) % EY, elz = m / (EX * EY);
        const uint2* xe = reinterpret_cast<const uint2*>(dig + ((elz * P * PY + ely * P) * PX + elx * P) * NC);
        const int half = s0 >> 2;   // slices 0-3 in the first 8 bytes of a record, 4-6 in the second
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          const int j = kg * 8 + q;
          const uint2 a = j < NL ? xe[2 * off[j] + half] : make_uint2(0u, 0u);
          const uint2 b = j + 1 < NL ? xe[2 * off[j + 1] + half] : make_uint2(0u, 0u);
          w[0][q >> 1] = __byte_perm(a.x, b.x, 0x5410);
          w[1][q >> 1] = __byte_perm(a.x, b.x, 0x7632);
          w[2][q >> 1] = __byte_perm(a.y, b.y, 0x5410);
          w[3][q >> 1] = __byte_perm(a.y, b.y, 0x7632);
        }
      }
      const int o = item * 8;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < ns) *reinterpret_cast<uint4*>(A + q * C::A_SLICE + o) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
  };
  // MMA chains of the digit pairs (s, t), s in [s0, s0 + ns), s + t <= 6, into level s + t
  auto issue = [&](int s0, int ns) {
    for (int s = s0; s < s0 + ns; ++s)
      for (int t = 0; s + t < C::NLEV; ++t) {
        const uint32_t acc_addr = tmem + (uint32_t)((s + t) * NP);
        for (int kk = 0; kk < KP / 16; ++kk) {
          const uint64_t da = umma_desc(aS[s - s0] + kk * 2 * C::LBO, C::LBO, C::SBO);
          const uint64_t db = umma_desc(bS0 + (uint32_t)(t * C::B_SLICE * 2) + kk * 2 * C::LBO, C::LBO, C::SBO);
          mma_bf16(acc_addr, da, db, idesc, (s == 0 && kk == 0) ? 0u : 1u);
        }
      }
  };

  for (;;) {
    const int gt = *next_tile;
    if (gt >= n_tiles) break;
    const int tile = *next_local;
    const uint32_t par = mma_phase & 1u;
    const int bx = tile % pb.tc_tiles[0];
    const int by = (tile / pb.tc_tiles[0]) % pb.tc_tiles[1];
    const int bz = DIM == 3 ? tile / (pb.tc_tiles[0] * pb.tc_tiles[1]) : 0;
    const int X0 = bx * C::TX, Y0 = by * C::TY, Z0 = bz * C::TZ;
    const int X1 = min(X0 + C::TX, pb.n[0]), Y1 = min(Y0 + C::TY, pb.n[1]);
    const int Z1 = DIM == 3 ? min(Z0 + C::TZ, pb.n[2]) : 1;
    double* const pf = pbuf(pcur);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (tid == 0) *n_special = 0;
    __syncthreads();   // the patch has landed for every thread; the list is empty
    int g_next = 0;
    if (tid == 0) g_next = atomicAdd(tcount, 1) + (int)gridDim.x;
    if (tid < C::NE) {
      const int64_t cell = halo_cell(tile, tid);
      const int cl = cell < 0 ? 0 : (int)pb.cls[cell];
      cidx[tid] = cl == 1 && mode != kModeImex ? pb.cut_index[cell] : -1;
      if (cl != 2) special[atomicAdd(n_special, 1)] = tid | (cl << 8);
    }
    // ---- tile exponent, then the seven digits of every patch value
    int e = 0;
    for (int i = tid; i < NV; i += NT) e = max(e, (int)((__double_as_longlong(pf[i]) >> 52) & 0x7ff));
    e = __reduce_max_sync(0xffffffffu, e);
    if (lane == 0) wmax[warp] = e;
    __syncthreads();
    int em = wmax[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) em = max(em, wmax[w]);
    for (int i = tid; i < NV; i += NT) dig[i] = fp64_digits7(pf[i], em);
    if (tid == 0) {
      *next_tile = g_next;
      *next_local = g_next < n_tiles ? order(g_next) : 0;
    }
    __syncthreads();
    // ---- phase 1: digit slices 0-3 of x against all slices of K_ref (22 chains)
    gather(0, 4);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the next tile's FP64 patch goes to the other buffer (free since the previous tile ended)
    const int nt = *next_tile, nl_ = *next_local;
    if (nt < n_tiles) issue_patch(nl_, pbuf(pcur ^ 1));
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (tid == 0) {
      if (!bimg_ready) {
        ok = mbar_wait(smem_u32(&bars[0]), 0u);
        bimg_ready = true;
      }
      if (ok) issue(0, 4);
      mma_commit(smem_u32(&bars[1]));
    }
    const bool r1 = mbar_wait(smem_u32(&bars[1]), par);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- phase 2: slices 4-6 (6 chains)
    gather(4, 3);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      if (ok && r1) issue(4, 3);
      mma_commit(smem_u32(&bars[2]));
    }
    const bool ready = mbar_wait(smem_u32(&bars[2]), par) && r1 && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ready) {
      if (tid == 0) atomicOr(pb.flags, 2);
    } else {
      // ---- drain: per (cell, row) the exact integers V0..V3 packed in pairs and the tail
      // V4 + 2^-8 V5 + 2^-16 V6 (in units of level 4), into yb (over the A slots)
      const int m = (warp & 3) * 32 + lane;
      const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
      constexpr int CGR = NW / 4;
#pragma unroll 1
      for (int c0 = (warp >> 2) * 8; c0 < NP; c0 += CGR * 8) {
        uint32_t r[C::NLEV][8];
#pragma unroll
        for (int l = 0; l < C::NLEV; ++l) {
          const uint32_t addr = lane_base + (uint32_t)(l * NP + c0);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(r[l][0]), "=r"(r[l][1]), "=r"(r[l][2]), "=r"(r[l][3]), "=r"(r[l][4]), "=r"(r[l][5]),
                         "=r"(r[l][6]), "=r"(r[l][7])
                       : "r"(addr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (m < C::NE) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int i = c0 + q;
            if (i < NL) {
              const int v0 = small_int_of_f32(__uint_as_float(r[0][q]));
              const int v1 = small_int_of_f32(__uint_as_float(r[1][q]));
              const int v2 = small_int_of_f32(__uint_as_float(r[2][q]));
              const int v3 = MAGIC3 ? small_int_of_f32(__uint_as_float(r[3][q])) : __float2int_rn(__uint_as_float(r[3][q]));
              const float tl = fmaf(__uint_as_float(r[5][q]), 0.00390625f,
                                    fmaf(__uint_as_float(r[6][q]), 1.52587890625e-05f, __uint_as_float(r[4][q])));
              yb[m * NL + i] = make_int4(v0 * 256 + v1, v2 * 256 + v3, __float_as_int(tl), 0);
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // ---- cut and outside cells: their rows leave the integer sums (zero); the assembly adds
    // the cut cells' K^e x_e in FP64 from the cut-cell kernel's output
    const int zsc = em + pb.tc_gexp - 1035;   // level-0 unit 2^(E + G - 1035)
    const int nsp = *n_special;
    for (int q = warp; q < nsp; q += NW) {
      const int mm = special[q] & 0xff;
      for (int i = lane; i < NL; i += 32) yb[mm * NL + i] = make_int4(0, 0, 0, 0);
    }
    __syncthreads();
    // ---- assembly (integer node sums, owned nodes as in kernels_tc.cu) and the FP64 update
    const int ox0 = X0 * P, oy0 = Y0 * P, oz0 = DIM == 3 ? Z0 * P : 0;
    int src_lo = 0, src_hi = 0;
    if ((mode == kModeCDM || mode == kModeStartup || mode == kModeImex) && pb.tsrc_ptr && pb.f_e > 0.0) {
      src_lo = pb.tsrc_ptr[tile];
      src_hi = pb.tsrc_ptr[tile + 1];
    }
    const int zku = zsc - 24;   // K u = 2^zku (H + tail 2^-8)
    // yc: the FP64 sum of the node's cut-cell contributions
    auto update = [&](int64_t dof, long long h01, long long h23, float tl, double yc, double uval, double upv,
                      double mi) {
      const long long H = h01 * 65536 + h23;
      const double hd = f64_of_i64(H);
      const double td = f32_to_f64_scaled(tl, -8);
      if (mode == kModeApply) {
        out[dof] = f64_scale2(hd + td, zku) + yc;
        return;
      }
      if (mode == kModeImex && mi < 0.0) {
        // c-DOF: Newmark predictor of Algorithm 2 (its K u is taken by the c-set solve)
        const int64_t ci = (int64_t)(-mi) - 1;
        const double a = pb.imex_ac[ci], v = pb.imex_vc[ci];
        out[dof] = uval + pb.dt * v + pb.imex_c1 * a;
        pb.imex_vc[ci] = v + pb.imex_c2 * a;
        return;
      }
      if (!(mi > 0.0)) return;
      const double c = -f64_scale2(mi, zku);   // -(dt^2 / m) 2^zku
      double r;
      if (mode == kModeCDM || mode == kModeImex)
        r = fma(c, hd, fma(c, td, fma(-mi, yc, fma(2.0, uval, -upv))));
      else
        r = fma(0.5 * c, hd, fma(0.5 * c, td, fma(-0.5 * mi, yc, fma(-pb.dt, upv, uval))));
      if (!isfinite(r)) bad = true;
      out[dof] = r;
    };
    {
      constexpr int PD = DIM == 3 ? P * P * P : P * P;
      constexpr int OWNC = PD * NC;
      constexpr int NCELL = C::TX * C::TY * C::TZ;
      constexpr int TOT = OWNC * NCELL;
      const int tx = X1 - X0, ty = Y1 - Y0, tz = DIM == 3 ? Z1 - Z0 : 1;
      for (int i = tid; i < TOT; i += NT) {
        const int q = i % OWNC, cell = i / OWNC;
        const int comp = q % NC, nd = q / NC;
        const int a = nd % P, bb = (nd / P) % P, cc = DIM == 3 ? nd / (P * P) : 0;
        const int ox = cell % C::TX, oy = (cell / C::TX) % C::TY, oz = DIM == 3 ? cell / (C::TX * C::TY) : 0;
        if (!(ox < tx && oy < ty && oz < tz)) continue;
        const int lx = ox * P + a, ly = oy * P + bb, lz = oz * P + cc;
        const int64_t dof = (((int64_t)(oz0 + lz) * pb.lat[1] + (oy0 + ly)) * pb.lat[0] + (ox0 + lx)) * NC + comp;
        double mi = 0.0, upv = 0.0, uval = 0.0;
        if (mode != kModeApply) {
          mi = __ldg(pb.minv + dof);
          upv = out[dof];
          uval = pf[(((DIM == 3 ? lz + P : 0) * PY + (ly + P)) * PX + (lx + P)) * NC + comp];
        }
        const int m = ((DIM == 3 ? oz + 1 : 0) * EY + (oy + 1)) * EX + (ox + 1);
        const int row = (((DIM == 3 ? cc * NN1 : 0) + bb) * NN1 + a) * NC + comp;
        long long h01 = 0, h23 = 0;
        float tl = 0.f;
        double yc = 0.0;
#pragma unroll
        for (int jz = 0; jz < (DIM == 3 ? 2 : 1); ++jz)
#pragma unroll
          for (int jy = 0; jy < 2; ++jy)
#pragma unroll
            for (int jx = 0; jx < 2; ++jx) {
              const bool val = (jx || a == 0) && (jy || bb == 0) && (DIM == 2 || jz || cc == 0);
              if (val) {
                const int mn = m - ((jx ? 0 : 1) + (jy ? 0 : EX) + (DIM == 3 && !jz ? EX * EY : 0));
                const int rn = row + (jx ? 0 : P * NC) + (jy ? 0 : P * NN1 * NC) + (DIM == 3 && !jz ? P * NN1 * NN1 * NC : 0);
                const int4 y = yb[mn * NL + rn];
                h01 += y.x;
                h23 += y.y;
                tl += __int_as_float(y.z);
                const int ci = cidx[mn];
                if (ci >= 0) yc += pb.Ycut[(size_t)ci * NL + rn];
              }
            }
        update(dof, h01, h23, tl, yc, uval, upv, mi);
      }
    }
    if (X1 == pb.n[0] || Y1 == pb.n[1] || (DIM == 3 && Z1 == pb.n[2])) {
      const int ex_ = (X1 - X0) * P, ey_ = (Y1 - Y0) * P, ez_ = DIM == 3 ? (Z1 - Z0) * P : 0;
      const int nox = ex_ + (X1 == pb.n[0] ? 1 : 0);
      const int noy = ey_ + (Y1 == pb.n[1] ? 1 : 0);
      const int noz = DIM == 3 ? ez_ + (Z1 == pb.n[2] ? 1 : 0) : 1;
      const int total = nox * noy * noz * NC;
      for (int i = tid; i < total; i += NT) {
        const int comp = i % NC, node = i / NC;
        const int lx = node % nox, ly = (node / nox) % noy, lz = node / (nox * noy);
        if (!(lx == ex_ || ly == ey_ || (DIM == 3 && lz == ez_))) continue;
        const int64_t dof = (((int64_t)(oz0 + lz) * pb.lat[1] + (oy0 + ly)) * pb.lat[0] + (ox0 + lx)) * NC + comp;
        const int px = lx + P, py = ly + P, pz = DIM == 3 ? lz + P : 0;
        const int cx = px / P, cy = py / P, cz = DIM == 3 ? pz / P : 0;
        const bool bxv = px - cx * P == 0, byv = py - cy * P == 0, bzv = DIM == 3 && pz - cz * P == 0;
        long long h01 = 0, h23 = 0;
        float tl = 0.f;
        double yc = 0.0;
        for (int jz = 0; jz < (DIM == 3 ? 2 : 1); ++jz)
          for (int jy = 0; jy < 2; ++jy)
            for (int jx = 0; jx < 2; ++jx) {
              const int ecx = cx - 1 + jx, ecy = cy - 1 + jy, ecz = DIM == 3 ? cz - 1 + jz : 0;
              const bool val = (jx ? cx < EX : bxv) && (jy ? cy < EY : byv) && (DIM == 2 || (jz ? cz < C::EZ : bzv));
              if (val) {
                const int m = (ecz * EY + ecy) * EX + ecx;
                const int row = (((DIM == 3 ? (pz - ecz * P) * NN1 : 0) + (py - ecy * P)) * NN1 + (px - ecx * P)) * NC + comp;
                const int4 y = yb[m * NL + row];
                h01 += y.x;
                h23 += y.y;
                tl += __int_as_float(y.z);
                const int ci = cidx[m];
                if (ci >= 0) yc += pb.Ycut[(size_t)ci * NL + row];
              }
            }
        double mi = 0.0, upv = 0.0, uval = 0.0;
        if (mode != kModeApply) {
          mi = __ldg(pb.minv + dof);
          upv = out[dof];
          uval = pf[(((DIM == 3 ? lz + P : 0) * PY + (ly + P)) * PX + (lx + P)) * NC + comp];
        }
        update(dof, h01, h23, tl, yc, uval, upv, mi);
      }
    }
    // the load F_k of this tile's DOFs, added after the update in FP64
    if (src_lo < src_hi && mode != kModeApply) {
      __syncthreads();
      const double w = mode == kModeStartup ? 0.5 : 1.0;
      for (int s2 = src_lo + tid; s2 < src_hi; s2 += NT) {
        const int64_t dof = pb.tsrc_dof[s2];
        const double mi = pb.minv[dof];
        if (mi > 0.0) out[dof] = fma(w * mi, pb.tsrc_val[s2] * fk, out[dof]);
      }
    }
    ++mma_phase;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();   // patches, lists, A / yb and next_tile are reused by the next tile
    pcur ^= 1;
  }
  if (bad) atomicOr(pb.flags, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
  }
  if (tid == 0) {
    __threadfence();
    unsigned prev = atomicAdd(pb.done, 1u);
    if (prev == gridDim.x - 1) {
      if (mode == kModeCDM) *pb.step = k + 1;
      *tcount = 0;
      *pb.done = 0u;
      __threadfence();
    }
  }
}

// ------------------------------------------------------------------ host side
#define IBFEM_TC64_SHAPES(X) X(2, 2, 1) X(2, 3, 1) X(2, 4, 1) X(2, 2, 2) X(2, 3, 2) X(2, 4, 2) X(3, 2, 1) X(3, 3, 1)

int op_tc64_variant(int dim) { return dim == 3 ? 1 : 0; }

template <int D, int P, int N>
static cudaError_t launch_tc64_t(const DevProblem& pb, const double* u, double* out, int mode, cudaStream_t st) {
  using C = Tc64Cfg<D, P, N>;
  static const cudaError_t cfg = [] {
    cudaError_t e = cudaFuncSetAttribute(op_tc64_kernel<D, P, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(op_tc64_kernel<D, P, N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    return e;
  }();
  if (cfg != cudaSuccess) return cfg;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = pb.tc_tiles[0] * pb.tc_tiles[1] * pb.tc_tiles[2];
  const int blocks = std::min(tiles, sms);
  op_tc64_kernel<D, P, N><<<blocks, kThreads64, C::SMEM, st>>>(pb, u, out, mode);
  return cudaGetLastError();
}

cudaError_t launch_op_tc64(const DevProblem& pb, const double* u, double* out, int mode, cudaStream_t st) {
#define X(D, P, N) \
  if (pb.dim == D && pb.p == P && pb.ncomp == N) return launch_tc64_t<D, P, N>(pb, u, out, mode, st);
  IBFEM_TC64_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace ibfem
