// Tensor-core element operator fused with the FP64 central-difference update
// (Eq. cdm of Buerchner et al., arXiv 2501.19013), for sm_103a (tcgen05 + TMEM).
//
// A persistent kernel: each CTA takes tiles of cells from a global counter (the host gives
// the processing order, costliest first); it owns the lattice nodes of its tile and
// recomputes the one-cell halo, so each node's sum over its cells is formed once, in a
// fixed order, without atomics.  The cells of the halo'd tile (one row of the MMA per
// cell, M = 128) are contracted with the shared reference matrix K_ref on the tensor
// cores:
//
//   exact scheme (IBFEM_EXACT_TC) -- an exact-slice (Ozaki-type) product:
//     x_j = 2^(E - 1054) sum_s d_s 2^(24 - 8 s),  K_ij = 2^(F_i - 31) sum_t c_t 2^(24 - 8 t)
//     with balanced 8-bit digits d_s, c_t (|digit| <= 256, exact in BF16), E the largest
//     biased FP64 exponent of the tile's node patch and F_i the K row's.  Products of
//     digits accumulate EXACTLY in the FP32 accumulators of tcgen05.mma kind::f16 (integers
//     below 2^24), one TMEM accumulator per level l = s + t <= 3 (10 MMA chains).  The drain
//     scales level 0 and the combined levels 1-3 by a power of two (exact); the node sums of
//     level 0 are error-free FP32 sums, so the cancellation in K u (element products
//     ~ lambda_max |u|, the sum much smaller) costs no precision before the one rounding of
//     the residual to FP32; the result carries about 32 significant bits.
//   bf16x3 / bf16 -- hi/lo BF16 splits with three MMA passes (hi.hi + hi.lo + lo.hi), or one
//     pass, accumulated in FP32 (the plain mixed-precision contraction).
//
// Cut cells replace their rows with K^e x_e computed on the CUDA cores in double-FP32
// arithmetic (FP32 (hi, lo) matrix pairs, error-free products and sums).  Per owned DOF:
// r = -(K u)_i rounded once to FP32, delta = (dt^2/m_i) r with a two-slice FP32 dt^2/m,
// widened to FP64 by bit manipulation, and u^{k+1} = (2 u^k - u^{k-1}) + delta in FP64: two
// FP64 operations per DOF, the only FP64 arithmetic of the step besides the loads, which
// are added per tile in FP64 (u^{k+1} += dt^2/m F_k).
// The FP64 node patch of the next tile is loaded with cp.async while the current one is
// finished; the K_ref digit image is copied into shared memory with the bulk-async (TMA)
// engine once per CTA (per member image in the batched form).
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tc_common.cuh"

namespace ibfem {

using namespace tc;

namespace {

// Balanced 8-bit digits of round(|x| 2^(31 - E)) for an FP64 x whose biased exponent is at
// most em (the tile's largest), sign applied to every digit, as four BF16 values (digits 0, 1
// in .x, digits 2, 3 in .y, low half first); 32-bit integer operations only.  d0 in [0, 256],
// d1..d3 in [-128, 128) before the sign.
__device__ __forceinline__ uint2 fp64_digits_bf16(double x, int em) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const uint32_t hw = (uint32_t)(bits >> 32), lw = (uint32_t)bits;
  const int eb = (int)((hw >> 20) & 0x7ffu);
  uint32_t V = 0;
  if (eb > 0) {
    const int sh = 21 + (em - eb);                 // >= 21
    const uint32_t mh = (hw & 0xFFFFFu) | 0x100000u;  // top 21 bits of the 53-bit significand
    if (sh < 32) {
      uint32_t t = __funnelshift_r(lw, mh, sh);     // (mh:lw) >> sh, fits 32 bits for sh >= 21
      uint32_t rb = (lw >> (sh - 1)) & 1u;          // rounding bit (sh - 1 < 32)
      V = t + rb;
      if (V < t) V = 0xFFFFFFFFu;                   // saturate the single all-ones carry case
    } else if (sh < 53) {
      uint32_t t = mh >> (sh - 32);
      uint32_t rb = sh == 32 ? (lw >> 31) : ((mh >> (sh - 33)) & 1u);
      V = t + rb;
    }
  }
  // balanced digits: the lower three are the bytes of (V mod 2^24) + 0x808080 minus 128
  // (each in [-128, 127]); the carry out of them goes to the top digit (in [0, 256])
  const uint32_t wl = (V & 0xFFFFFFu) + 0x808080u;
  const int d0 = (int)(V >> 24) + (int)(wl >> 24);
  // exact FP32 of byte b minus 128: the pattern 0x4B4000bb is the float 1.5 * 2^23 + b
  const uint32_t f0 = f32_bits_of_small_int(d0);
  const uint32_t f1 = __float_as_uint(__uint_as_float(__byte_perm(wl, 0x4B400000u, 0x7652)) - 12583040.0f);
  const uint32_t f2 = __float_as_uint(__uint_as_float(__byte_perm(wl, 0x4B400000u, 0x7651)) - 12583040.0f);
  const uint32_t f3 = __float_as_uint(__uint_as_float(__byte_perm(wl, 0x4B400000u, 0x7650)) - 12583040.0f);
  // BF16 = upper half of the FP32 pattern (at most 8 significant bits: exact); the sign of
  // x goes to every digit
  const uint32_t sgn = (hw >> 31) ? 0x80008000u : 0u;
  return make_uint2(__byte_perm(f0, f1, 0x7632) ^ sgn, __byte_perm(f2, f3, 0x7632) ^ sgn);
}

// Diagnostic of the bounded waits: one thread waits, with the poll limit given by the host,
// on an mbarrier that nothing arrives on (no MMA or copy is in flight), exactly as the
// operator kernel waits for its MMA completions; when the limit runs out it records the
// timeout in the problem's flag word (bit 1), the same record the operator kernel leaves,
// and returns.
__global__ void bounded_wait_probe_kernel(int* flags, int polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (!mbar_wait(smem_u32(&bar), 0u, polls)) atomicOr(flags, 2);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)));
  }
}

}  // namespace

cudaError_t launch_bounded_wait_probe(int* flags, int polls, cudaStream_t st) {
  bounded_wait_probe_kernel<<<1, 32, 0, st>>>(flags, polls);
  return cudaGetLastError();
}

template <int DIM, int P, int NC, int TILE>
struct TcCfg {
  static constexpr int NN1 = P + 1;
  static constexpr int NNL = DIM == 2 ? NN1 * NN1 : NN1 * NN1 * NN1;
  static constexpr int NL = NNL * NC;
  static constexpr int KP = (NL + 15) / 16 * 16;   // K padded to the BF16 MMA step (16)
  static constexpr int NP = (NL + 15) / 16 * 16;   // N padded (M = 128 needs N % 16 == 0)
  static constexpr int NACC = 4;                    // accumulators (levels 0..3)
  static constexpr int TMEM_COLS = NACC * NP <= 32 ? 32 : (NACC * NP <= 64 ? 64 : (NACC * NP <= 128 ? 128 : (NACC * NP <= 256 ? 256 : 512)));
  static constexpr int TX = tc_tile_x(DIM, NL, TILE), TY = tc_tile_y(DIM, NL, TILE), TZ = tc_tile_z(DIM, TILE);
  static constexpr int EX = TX + 1, EY = TY + 1, EZ = DIM == 3 ? TZ + 1 : 1;
  static constexpr int NE = EX * EY * EZ;
  static constexpr int PX = EX * P + 1, PY = EY * P + 1, PZ = DIM == 3 ? EZ * P + 1 : 1;
  static constexpr int PATCH = PX * PY * PZ * NC;
  static constexpr int LBO = 128;                   // bytes between K-adjacent core matrices
  static constexpr int SBO = (KP / 8) * 128;        // bytes between M/N-adjacent core matrices
  static constexpr int A_SLICE = 128 * KP;          // BF16 elements of one A slice
  static constexpr int B_SLICE = NP * KP;           // BF16 elements of one B slice
  static constexpr size_t A_BYTES = 2 * 2 * (size_t)A_SLICE;  // two slots
  static constexpr size_t B_BYTES = 4 * 2 * (size_t)B_SLICE;  // four digit slices
  static constexpr size_t Y_BYTES = 8 * (size_t)NE * NL;      // (D0, L) per (cell, row)
  static constexpr bool Y_ALIAS = Y_BYTES <= A_BYTES;   // B persists across tiles
  static constexpr size_t OFF_A = 0;
  static constexpr size_t OFF_B = OFF_A + A_BYTES;
  static constexpr size_t OFF_Y = Y_ALIAS ? 0 : OFF_B + B_BYTES;
  static constexpr size_t OFF_PATCH = ((Y_ALIAS ? OFF_B + B_BYTES : OFF_Y + Y_BYTES) + 15) / 16 * 16;
  static constexpr size_t PATCH_BYTES = (8 * (size_t)PATCH + 15) / 16 * 16;  // one patch buffer
  static constexpr size_t OFF_E = OFF_PATCH + 2 * PATCH_BYTES;              // int E[128]
  static constexpr size_t OFF_F = OFF_E + 4 * (4 + 128 + 8);                 // int F[NP]
  static constexpr size_t OFF_SC = OFF_F + 4 * (size_t)NP;                   // float scale[NP]
  static constexpr size_t OFF_OFF = OFF_SC + 4 * (size_t)NP;                 // int off[KP]
  static constexpr size_t OFF_XS = (OFF_OFF + 4 * (size_t)KP + 15) / 16 * 16;  // 8 warps x 2 x NL floats
  static constexpr size_t OFF_BAR = (OFF_XS + 4 * 2 * 8 * (size_t)NL + 15) / 16 * 16;
  static constexpr size_t SMEM = OFF_BAR + 64;
  // never co-schedule more CTAs on an SM than its 512 TMEM columns can hold
  static constexpr int CTA_TMEM_MAX = 512 / TMEM_COLS;
  static constexpr size_t SMEM_FLOOR = 233472 / (CTA_TMEM_MAX + 1) - 1024 + 16;
  static constexpr size_t SMEM_LAUNCH = SMEM > SMEM_FLOOR ? SMEM : SMEM_FLOOR;
  static_assert(NE <= 128, "halo'd tile must fit one M = 128 MMA");
  static_assert(KP % 8 == 0 && (KP / 8) <= 32, "K layout");
};

// scheme: 0 exact, 1 bf16x3, 2 bf16.  Persistent: each CTA loads the K_ref digits once and
// takes tiles from a global counter until none are left.
// BATCH: the tiles of several problems (members) of one shape in one launch, CDM mode.  A
// CTA keeps the descriptor of its current member in shared memory and reloads the K_ref
// image only when a member with another image comes up (the host orders members by image).
template <int DIM, int P, int NC, int SCHEME, bool BATCH, int TILE>
__global__ void __launch_bounds__(256, 2) op_tc_kernel(const __grid_constant__ DevProblem pb_arg, const double* u_arg,
                                                    double* out_arg, int mode,
                                                    const BatchMember* __restrict__ members,
                                                    const int* __restrict__ tile_start, int n_members,
                                                    int total_tiles, BatchCtl* ctl) {
  using C = TcCfg<DIM, P, NC, TILE>;
  constexpr int NL = C::NL, NN1 = C::NN1, KP = C::KP, NP = C::NP;
  constexpr int EX = C::EX, EY = C::EY, PX = C::PX, PY = C::PY;
  constexpr int NV = C::PATCH;                                // patch values
  extern __shared__ __align__(1024) unsigned char smem[];
  uint16_t* A = reinterpret_cast<uint16_t*>(smem + C::OFF_A);
  uint16_t* B = reinterpret_cast<uint16_t*>(smem + C::OFF_B);
  // per (cell, row): level 0 and the combined levels 1-3, both scaled to their value
  float2* yb = reinterpret_cast<float2*>(smem + C::OFF_Y);
  // two patch buffers, swapped every tile: the FP64 node patch of u^k (read by the digit
  // conversion, the cut cells and the update) and the BF16 digits of it (read by the A
  // gather), which then receives the next tile's FP64 patch
  auto pbuf = [&](int which) { return reinterpret_cast<double*>(smem + C::OFF_PATCH + which * C::PATCH_BYTES); };
  int pcur = 0;
  int* Eb = reinterpret_cast<int*>(smem + C::OFF_E);          // Eb[0]: tile exponent; Eb[1..]: lists
  int* Fr = reinterpret_cast<int*>(smem + C::OFF_F);
  float* scl = reinterpret_cast<float*>(smem + C::OFF_SC);   // per tile: 2^(E + F_i - 1037)
  int* off = reinterpret_cast<int*>(smem + C::OFF_OFF);
  float* xs = reinterpret_cast<float*>(smem + C::OFF_XS);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);  // 0: B copy, 1: MMA phase 1, 2: phase 2
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 32);
  int* next_tile = reinterpret_cast<int*>(smem + C::OFF_BAR + 40);
  int* n_special = reinterpret_cast<int*>(smem + C::OFF_BAR + 44);
  int* special = Eb + 4;                                      // cut / outside cells of the tile
  int* wmax = Eb + 4 + 128;                                   // per-warp exponent maxima
  int* next_member = n_special + 1;                           // batched: member of next_tile
  int* next_local = n_special + 2;                            // next_tile within its problem, ordered
  BatchMember* sbm = reinterpret_cast<BatchMember*>(smem + C::SMEM);  // batched: current member
  const DevProblem& pb = BATCH ? sbm->pb : pb_arg;
  const double* __restrict__ u = u_arg;
  double* __restrict__ out = out_arg;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_tiles = BATCH ? total_tiles : pb_arg.tc_tiles[0] * pb_arg.tc_tiles[1] * pb_arg.tc_tiles[2];
  int* const tcount = BATCH ? &ctl->tile_counter : pb_arg.tile_counter;
  // batched: the member of global tile g (binary search of the tile ranges)
  auto member_of = [&](int g) {
    int lo = 0, hi = n_members;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tile_start[mid] <= g) lo = mid;
      else hi = mid;
    }
    return lo;
  };

  // asynchronous load of the node patch of `tile` (zero outside the lattice)
  auto issue_patch = [&](int t, double* patch) {
    const int ibx = t % pb.tc_tiles[0];
    const int iby = (t / pb.tc_tiles[0]) % pb.tc_tiles[1];
    const int ibz = DIM == 3 ? t / (pb.tc_tiles[0] * pb.tc_tiles[1]) : 0;
    const int hx0 = (ibx * C::TX - 1) * P, hy0 = (iby * C::TY - 1) * P;
    const int hz0 = DIM == 3 ? (ibz * C::TZ - 1) * P : 0;
    for (int node = tid; node < NV / NC; node += blockDim.x) {
      int px = node % PX, py = (node / PX) % PY, pz = node / (PX * PY);
      int gx = hx0 + px, gy = hy0 + py, gz = hz0 + pz;
      bool in = gx >= 0 && gx < pb.lat[0] && gy >= 0 && gy < pb.lat[1] && gz >= 0 && gz < pb.lat[2];
      int64_t g = in ? (((int64_t)gz * pb.lat[1] + gy) * pb.lat[0] + gx) * NC : 0;
      cp_async_zfill<8 * NC>(patch + node * NC, u + g, in ? 8 * NC : 0);
    }
  };

  // class of halo cell m of local tile t (0 outside the domain)
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
  int my_cl = 0;   // class of halo cell `tid` of the prefetched tile (valid with have_patch)
  bool have_patch = false;   // the current tile's patch was loaded ahead

  // ---- once per CTA: TMEM, barriers, K_ref digits (bulk copy), tables, observers
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(C::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int b = 0; b < 3; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[b])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
  }
  if (!BATCH && tid == 32) {
    const uint32_t bytes = (uint32_t)C::B_BYTES;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bars[0])), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(B)),
                 "l"(pb.tc_bimg), "r"(bytes), "r"(smem_u32(&bars[0]))
                 : "memory");
  }
  // global tile g -> (member, tile of that member in processing order); thread 0 only
  auto resolve = [&](int g, int& m, int& t) {
    m = 0;
    t = 0;
    if (g >= n_tiles) return;
    if (BATCH) m = member_of(g);
    const int local = BATCH ? g - tile_start[m] : g;
    const int32_t* ord = BATCH ? members[m].pb.tc_order : pb_arg.tc_order;
    t = ord ? ord[local] : local;
  };
  // single problem: CTA b starts with global tile b (the counter hands out the rest), whose
  // patch load is issued right away and overlaps the set-up below
  if (!BATCH) {
    const int t0 = pb_arg.tc_order ? pb_arg.tc_order[blockIdx.x] : (int)blockIdx.x;
    issue_patch(t0, pbuf(0));
    asm volatile("cp.async.commit_group;" ::: "memory");
    have_patch = true;
    if (tid < C::NE) my_cl = halo_class(t0, tid);
  }
  if (tid == 0) {
    const int g = BATCH ? atomicAdd(tcount, 1) : (int)blockIdx.x;
    int m, t;
    resolve(g, m, t);
    *next_tile = g;
    *next_member = m;
    *next_local = t;
  }
  if (!BATCH)
    for (int i = tid; i < NP; i += blockDim.x) Fr[i] = pb.tc_frow ? pb.tc_frow[i] : 0;
  for (int j = tid; j < KP; j += blockDim.x) {
    int node = j / NC, comp = j % NC;
    int a = node % NN1, b = (node / NN1) % NN1, c = DIM == 3 ? node / (NN1 * NN1) : 0;
    off[j] = j < NL ? ((c * PY + b) * PX + a) * NC + comp : -1;
  }
  unsigned long long k = 0;
  if (!BATCH && (mode == kModeCDM || mode == kModeImex)) k = *((volatile unsigned long long*)pb.step);
  if (!BATCH && blockIdx.x == 0 && mode == kModeCDM && pb.n_obs_rows > 0 && pb.ring_cap > 0) {
    for (int r = tid; r < pb.n_obs_rows; r += blockDim.x) {
      double acc = 0.0;
      for (int j = 0; j < pb.obs_nodes; ++j)
        acc += pb.obs_w[(size_t)r * pb.obs_nodes + j] * u[pb.obs_dof[(size_t)r * pb.obs_nodes + j]];
      pb.ring[(size_t)(k % (unsigned long long)pb.ring_cap) * pb.n_obs_rows + r] = acc;
    }
  }
  double fk = 0.0;
  if (!BATCH && (mode == kModeCDM || mode == kModeStartup || mode == kModeImex) && pb.tsrc_ptr && pb.f_e > 0.0)
    fk = ricker_tc((double)k * pb.dt, pb.f_e);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NP >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  const uint32_t aS[2] = {smem_u32(A), smem_u32(A + C::A_SLICE)};
  const uint32_t bS0 = smem_u32(B);
  bool ok = true, bimg_ready = false, bad = false;
  int cur_m = -1;                       // batched: member whose descriptor is in shared memory
  const uint16_t* cur_bimg = nullptr;   // batched: K_ref image in shared memory
  uint32_t b_loads = BATCH ? 0u : 1u;   // K_ref image loads issued (phase of bars[0])
  uint32_t mma_phase = 0;               // tiles whose MMAs were committed (phase of bars[1], bars[2])
  constexpr int KG = KP / 8;
  constexpr int ROWS = (C::NE + 7) / 8 * 8;   // MMA rows that carry cells (the rest are ignored)
  constexpr int ITEMS = ROWS * KG;
  constexpr int IPT = (ITEMS + 255) / 256;


  for (;;) {
    const int gt = *next_tile;
    if (gt >= n_tiles) break;
    const int tile = *next_local;   // this problem's tile, in processing order
    bool skip = false;
    if constexpr (BATCH) {
      const int m = *next_member;
      if (m != cur_m) {
        // switch members (nothing reads the old descriptor after the loop-end barrier)
        if (tid == 0) *sbm = members[m];
        __syncthreads();
        k = *((volatile unsigned long long*)sbm->pb.step);
        if (k < sbm->step_end && sbm->pb.tc_bimg != cur_bimg) {
          // new K_ref image (only for a member that still steps, so that a load is always
          // waited on before the next one): every MMA of the previous tile has completed
          cur_bimg = sbm->pb.tc_bimg;
          ++b_loads;
          bimg_ready = false;
          if (tid == 0) {
            const uint32_t bytes = (uint32_t)C::B_BYTES;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bars[0])), "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(B)),
                "l"(cur_bimg), "r"(bytes), "r"(smem_u32(&bars[0]))
                : "memory");
          }
          for (int i = tid; i < NP; i += blockDim.x) Fr[i] = sbm->pb.tc_frow[i];
        }
        fk = (sbm->pb.tsrc_ptr && sbm->pb.f_e > 0.0) ? ricker_tc((double)k * sbm->pb.dt, sbm->pb.f_e) : 0.0;
        u = (k & 1ull) ? sbm->Ub : sbm->Ua;
        out = (k & 1ull) ? sbm->Ua : sbm->Ub;
        cur_m = m;
        have_patch = false;
      }
      skip = k >= sbm->step_end;
    }
    const uint32_t par = mma_phase & 1u;
    const int bx = tile % pb.tc_tiles[0];
    const int by = (tile / pb.tc_tiles[0]) % pb.tc_tiles[1];
    const int bz = DIM == 3 ? tile / (pb.tc_tiles[0] * pb.tc_tiles[1]) : 0;
    const int X0 = bx * C::TX, Y0 = by * C::TY, Z0 = bz * C::TZ;
    const int X1 = min(X0 + C::TX, pb.n[0]), Y1 = min(Y0 + C::TY, pb.n[1]);
    const int Z1 = DIM == 3 ? min(Z0 + C::TZ, pb.n[2]) : 1;

    // ---- node patch of u^k: prefetched during the previous tile's update, else loaded now
    double* const pf = pbuf(pcur);                                  // FP64 patch of u^k
    uint2* const dpd = reinterpret_cast<uint2*>(pbuf(pcur ^ 1));    // its digits
    if (!have_patch && !skip) {
      issue_patch(tile, pf);
      cp_async_commit_wait_all();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // a patch loaded ahead has landed
    // cut / outside cells of the halo'd tile (class byte per cell, compact list)
    if (tid == 0) *n_special = 0;
    __syncthreads();
    // the next tile: the atomic's latency is hidden behind this tile's work; thread 0
    // publishes the result before the drain barrier (it is read after that barrier)
    // (its lookups are resolved after the digit conversion, published before the drain
    // barrier and read after it)
    int g_next = 0, m_next = 0, t_next = 0;
    if (tid == 0) g_next = atomicAdd(tcount, 1) + (BATCH ? 0 : (int)gridDim.x);
    auto publish_next = [&]() {
      if (tid == 0) {
        *next_tile = g_next;
        *next_member = m_next;
        *next_local = t_next;
      }
    };
    if (skip) {   // batched: this member has taken all its steps
      have_patch = false;
      if (tid == 0) resolve(g_next, m_next, t_next);
      publish_next();
      __syncthreads();
      continue;
    }
    if (BATCH && tile == 0 && pb.n_obs_rows > 0 && pb.ring_cap > 0) {
      for (int r = tid; r < pb.n_obs_rows; r += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < pb.obs_nodes; ++j)
          acc += pb.obs_w[(size_t)r * pb.obs_nodes + j] * u[pb.obs_dof[(size_t)r * pb.obs_nodes + j]];
        pb.ring[(size_t)(k % (unsigned long long)pb.ring_cap) * pb.n_obs_rows + r] = acc;
      }
    }
    if (tid < C::NE) {
      const int cl = have_patch ? my_cl : halo_class(tile, tid);
      if (cl != 2) special[atomicAdd(n_special, 1)] = tid | (cl << 8);
    }

    // ---- tile exponent (largest biased FP64 exponent of the patch), then the patch is
    // rewritten in place as four BF16 digits per value (8 bytes, like the FP64 value)
    int em = 0;
    if (SCHEME == 0) {
      int e = 0;
      for (int i = tid; i < NV; i += blockDim.x) e = max(e, (int)((__double_as_longlong(pf[i]) >> 52) & 0x7ff));
      e = __reduce_max_sync(0xffffffffu, e);
      if (lane == 0) wmax[warp] = e;
      __syncthreads();
      em = wmax[0];
#pragma unroll
      for (int w = 1; w < 8; ++w) em = max(em, wmax[w]);
      // the drain's scale of output row i: 2^(E + F_i - 1037), zero below the FP32 normals
      // (read after the barrier that ends the digit conversion)
      for (int i = tid; i < NP; i += blockDim.x) {
        const int sh = em - 1023 - 14 + Fr[i];
        scl[i] = sh < -126 ? 0.f : __int_as_float((min(sh, 127) + 127) << 23);
      }
    }
    for (int i = tid; i < NV; i += blockDim.x) {
      double x = pf[i];
      uint32_t lo16, hi16;
      if (SCHEME == 0) {
        const uint2 dg = fp64_digits_bf16(x, em);
        lo16 = dg.x;
        hi16 = dg.y;
      } else {
        float xf = f64_to_f32_rn(x);
        uint16_t h = bf16_rn(xf);
        lo16 = h | ((uint32_t)bf16_rn(xf - __uint_as_float((uint32_t)h << 16)) << 16);
        hi16 = 0;
      }
      dpd[i] = make_uint2(lo16, hi16);
    }
    __syncthreads();

    if (tid == 0) resolve(g_next, m_next, t_next);   // the atomic has long returned
    // ---- A operand: each item writes one 8-element row of a core matrix (16 bytes) of slots
    // 0 and 1 by copying digits; slices 2 and 3 stay in registers until phase 2
    uint32_t keep[IPT][8];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      int item = tid + it * 256;
      if (item >= ITEMS) break;
      int r8 = item & 7, rest = item >> 3;
      int kg = rest % KG, rg = rest / KG;
      int m = rg * 8 + r8;
      uint32_t w[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
      if (m < C::NE && kg * 8 < NL) {
        int elx = m % EX, ely = (m / EX) % EY, elz = m / (EX * EY);
        const uint2* xe = dpd + ((elz * P * PY + ely * P) * PX + elx * P) * NC;
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          const int j = kg * 8 + q;
          uint2 a = j < NL ? xe[off[j]] : make_uint2(0u, 0u);
          uint2 b = j + 1 < NL ? xe[off[j + 1]] : make_uint2(0u, 0u);
          w[0][q >> 1] = __byte_perm(a.x, b.x, 0x5410);   // slice 0 of j and j+1
          w[1][q >> 1] = __byte_perm(a.x, b.x, 0x7632);   // slice 1
          w[2][q >> 1] = __byte_perm(a.y, b.y, 0x5410);   // slice 2
          w[3][q >> 1] = __byte_perm(a.y, b.y, 0x7632);   // slice 3
        }
      }
      const int o = item * 8;   // == bf16_core_offset<KP>(m, kg * 8)
      *reinterpret_cast<uint4*>(A + o) = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
      *reinterpret_cast<uint4*>(A + C::A_SLICE + o) = make_uint4(w[1][0], w[1][1], w[1][2], w[1][3]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        keep[it][q] = w[2][q];
        keep[it][4 + q] = w[3][q];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- phase 1 MMAs (A slots hold x-digit slices 0 and 1)
    if (tid == 0) {
      if (!bimg_ready) {
        ok = mbar_wait(smem_u32(&bars[0]), (b_loads - 1u) & 1u);  // K_ref digits have landed
        bimg_ready = true;
      }
      if (ok) {
        const int S1 = SCHEME == 0 ? 7 : (SCHEME == 1 ? 3 : 1);
        const int ps[7] = {0, 0, 1, 0, 1, 0, 1};
        const int pt[7] = {0, 1, 0, 2, 1, 3, 2};
        const int pl[7] = {0, 1, 1, 2, 2, 3, 3};
        const int pf[7] = {1, 1, 0, 1, 0, 1, 0};
        const int qs[3] = {0, 0, 1};
        const int qt[3] = {0, 1, 0};
        for (int w = 0; w < S1; ++w) {
          int s = SCHEME == 0 ? ps[w] : qs[w], t = SCHEME == 0 ? pt[w] : qt[w];
          int l = SCHEME == 0 ? pl[w] : 0;
          int first = SCHEME == 0 ? pf[w] : (w == 0);
          uint32_t acc_addr = tmem + (uint32_t)(l * NP);
          for (int kk = 0; kk < KP / 16; ++kk) {
            uint64_t da = umma_desc(aS[s] + kk * 2 * C::LBO, C::LBO, C::SBO);
            uint64_t db = umma_desc(bS0 + (uint32_t)(t * C::B_SLICE * 2) + kk * 2 * C::LBO, C::LBO, C::SBO);
            mma_bf16(acc_addr, da, db, idesc, (first && kk == 0) ? 0u : 1u);
          }
        }
      }
      mma_commit(smem_u32(&bars[1]));
    }
    bool r_all = true;
    if (SCHEME == 0) {
      bool r1 = mbar_wait(smem_u32(&bars[1]), par);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int it = 0; it < IPT; ++it) {
        int item = tid + it * 256;
        if (item >= ITEMS) break;
        const int o = item * 8;
        *reinterpret_cast<uint4*>(A + o) = make_uint4(keep[it][0], keep[it][1], keep[it][2], keep[it][3]);
        *reinterpret_cast<uint4*>(A + C::A_SLICE + o) = make_uint4(keep[it][4], keep[it][5], keep[it][6], keep[it][7]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        if (ok && r1) {
          const int qs2[3] = {0, 0, 1};
          const int qt2[3] = {0, 1, 0};
          const int ql2[3] = {2, 3, 3};
          for (int w = 0; w < 3; ++w) {
            uint32_t acc_addr = tmem + (uint32_t)(ql2[w] * NP);
            for (int kk = 0; kk < KP / 16; ++kk) {
              uint64_t da = umma_desc(aS[qs2[w]] + kk * 2 * C::LBO, C::LBO, C::SBO);
              uint64_t db = umma_desc(bS0 + (uint32_t)(qt2[w] * C::B_SLICE * 2) + kk * 2 * C::LBO, C::LBO, C::SBO);
              mma_bf16(acc_addr, da, db, idesc, 1u);
            }
          }
        }
        mma_commit(smem_u32(&bars[2]));
      }
      r_all = r1;
    }
    const bool ready = mbar_wait(smem_u32(&bars[SCHEME == 0 ? 2 : 1]), par) && r_all;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ready) {
      if (tid == 0) atomicOr(pb.flags, 2);
    } else {
      // ---- drain TMEM: level 0 and the combined levels 1-3, both scaled to their value by
      // a multiplication with 2^(E + F_i - 14) (exact: D0 is an integer below 2^24; values
      // below the FP32 normal range are negligible).  Warps w and w + 4 share the lane
      // quarter w % 4 and split the column blocks.
      const int m = (warp & 3) * 32 + lane;
      const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
      for (int c0 = (warp >> 2) * 16; c0 < NP; c0 += 32) {
        uint32_t r[4][16];
#pragma unroll
        for (int l = 0; l < (SCHEME == 0 ? 4 : 1); ++l) {
          uint32_t addr = lane_base + (uint32_t)(l * NP + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(r[l][0]), "=r"(r[l][1]), "=r"(r[l][2]), "=r"(r[l][3]), "=r"(r[l][4]), "=r"(r[l][5]),
                "=r"(r[l][6]), "=r"(r[l][7]), "=r"(r[l][8]), "=r"(r[l][9]), "=r"(r[l][10]), "=r"(r[l][11]),
                "=r"(r[l][12]), "=r"(r[l][13]), "=r"(r[l][14]), "=r"(r[l][15])
              : "r"(addr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float scq[16];
        if (SCHEME == 0) {
#pragma unroll
          for (int q = 0; q < 16; q += 4) {
            const float4 v = *reinterpret_cast<const float4*>(scl + c0 + q);
            scq[q] = v.x;
            scq[q + 1] = v.y;
            scq[q + 2] = v.z;
            scq[q + 3] = v.w;
          }
        }
        if (m < C::NE) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            int i = c0 + q;
            if (i < NL) {
              if (SCHEME == 0) {
                const float sc = scq[q];
                float lo = fmaf(__uint_as_float(r[1][q]), 0.00390625f,
                                fmaf(__uint_as_float(r[2][q]), 1.52587890625e-05f,
                                     __uint_as_float(r[3][q]) * 5.9604644775390625e-08f));
                yb[m * NL + i] = make_float2(__uint_as_float(r[0][q]) * sc, lo * sc);
              } else {
                yb[m * NL + i] = make_float2(__uint_as_float(r[0][q]), 0.f);
              }
            }
          }
        }
      }
    }
    publish_next();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();

    // ---- the digit buffer is free: the next tile's FP64 patch goes there (asynchronously,
    // landing during the cut cells and the update)
    {
      const int nt = *next_tile;
      have_patch = nt < n_tiles && (!BATCH || *next_member == cur_m);
      if (have_patch) {
        const int lt = *next_local;
        issue_patch(lt, pbuf(pcur ^ 1));
        if (tid < C::NE) my_cl = halo_class(lt, tid);   // consumed at the next tile's top
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }

    // ---- cut and outside cells replace their rows (double-FP32 on the CUDA cores; u^k from
    // global memory, the patch now holds digits)
    const int nsp = *n_special;
    for (int q = warp; q < nsp; q += 8) {
      const int m = special[q] & 0xff, cl = special[q] >> 8;
      int elx = m % EX, ely = (m / EX) % EY, elz = m / (EX * EY);
      int ex = X0 - 1 + elx, ey = Y0 - 1 + ely, ez = DIM == 3 ? Z0 - 1 + elz : 0;
      if (cl == 0) {
        for (int i = lane; i < NL; i += 32) yb[m * NL + i] = make_float2(0.f, 0.f);
        continue;
      }
      float* xh = xs + warp * 2 * NL;
      float* xl = xh + NL;
      const double* xe = pf + ((elz * P * PY + ely * P) * PX + elx * P) * NC;
      for (int j = lane; j < NL; j += 32) {
        const double x = xe[off[j]];
        float h = f64_to_f32_rn(x);
        xh[j] = h;
        xl[j] = f64_to_f32_rn(x - f32_to_f64_scaled(h, 0));
      }
      __syncwarp();
      const int64_t cell = ((int64_t)ez * pb.n[1] + ey) * pb.n[0] + ex;
      // K^e as (hi, lo) FP32 pairs, column j contiguous over the rows i; the lane's rows
      // run as independent chains and the loads of several columns are in flight together
      const int32_t ci = pb.cut_index[cell];
      const float2* K2 =
          reinterpret_cast<const float2*>(pb.Kcut32) + (size_t)(pb.cut_mat ? pb.cut_mat[ci] : ci) * NL * NL;
      constexpr int R = (NL + 31) / 32;
      float sacc[R], cacc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) sacc[r] = cacc[r] = 0.f;
#pragma unroll 10
      for (int j = 0; j < NL; ++j) {
        const float xhj = xh[j], xlj = xl[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          // rows past NL (last chain of some lanes) compute on row NL - 1 and are dropped
          const float2 kk = __ldg(K2 + (size_t)j * NL + min(lane + 32 * r, NL - 1));
          const float p = kk.x * xhj;
          float pe = fmaf(kk.x, xhj, -p);          // exact error of the product
          pe = fmaf(kk.x, xlj, fmaf(kk.y, xhj, pe));
          float t, e;
          two_sum(sacc[r], p, t, e);
          sacc[r] = t;
          cacc[r] += e + pe;
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        if (i < NL) {
          float hs, he;
          two_sum(sacc[r], cacc[r], hs, he);
          yb[m * NL + i] = make_float2(hs, he);
        }
      }
      __syncwarp();
    }
    __syncthreads();
    // ---- node-centric assembly and the FP64 update.  Each owned cell owns the nodes whose
    // local indices all lie below P (its low corner block), so the cells around an owned
    // node sit at fixed offsets of the halo'd tile and of their output rows; the nodes on
    // the domain's high faces (local index P in the last cell) follow in a second pass.
    // The cells of a node are summed in the order (z, y, x) of their offsets, lower first.
    const int ox0 = X0 * P, oy0 = Y0 * P, oz0 = DIM == 3 ? Z0 * P : 0;
    int src_lo = 0, src_hi = 0;
    if ((mode == kModeCDM || mode == kModeStartup || mode == kModeImex) && pb.tsrc_ptr && pb.f_e > 0.0) {
      src_lo = pb.tsrc_ptr[tile];
      src_hi = pb.tsrc_ptr[tile + 1];
    }
    // the update of one owned DOF from its sum -K u = -(sh + (se + lo))
    auto update = [&](int64_t dof, float sh, float se, float lo, double uval, double upv, float mh, float ml) {
      if (mode == kModeApply) {
        out[dof] = f32_to_f64_scaled(sh, 0) + f32_to_f64_scaled(se + lo, 0);
        return;
      }
      if (!(mh > 0.f)) {
        // IMEX mode, a c-DOF (dt^2/m = -(c + 1) in FP64, no FP32 slices): the Newmark
        // predictor of Algorithm 2 (its K u is taken by the c-set solve)
        if (mode == kModeImex) {
          const double mi = pb.minv[dof];
          if (mi < 0.0) {
            const int64_t ci = (int64_t)(-mi) - 1;
            const double a = pb.imex_ac[ci], v = pb.imex_vc[ci];
            out[dof] = uval + pb.dt * v + pb.imex_c1 * a;
            pb.imex_vc[ci] = v + pb.imex_c2 * a;
          }
        }
        return;
      }
      const float r = -(sh + (se + lo));   // -K u rounded once to FP32 (the load follows below)
      const float d32 = fmaf(mh, r, ml * r);
      if (!isfinite(d32)) bad = true;
      const double delta = f32_to_f64_scaled(d32, 0);
      if (mode == kModeCDM || mode == kModeImex)
        out[dof] = fma(2.0, uval, -upv) + delta;
      else
        out[dof] = uval - pb.dt * upv + 0.5 * delta;
    };
    {
      constexpr int PD = DIM == 3 ? P * P * P : P * P;
      constexpr int OWNC = PD * NC;                                 // DOFs a cell owns
      constexpr int NCELL = C::TX * C::TY * C::TZ;
      constexpr int TOT = OWNC * NCELL;
      constexpr int NB = (TOT + 255) / 256 < 4 ? (TOT + 255) / 256 : 4;
      // offsets (in float2 entries of yb) of the lower neighbours' rows of the same node
      constexpr int DX = NL - P * NC, DY = EX * NL - P * NN1 * NC, DZ = EX * EY * NL - P * NN1 * NN1 * NC;
      const int tx = X1 - X0, ty = Y1 - Y0, tz = DIM == 3 ? Z1 - Z0 : 1;
      for (int base = tid; base < TOT; base += NB * 256) {
        double upv[NB], ukv[NB];
        float mhv[NB], mlv[NB];
        int64_t dofv[NB];
        int yix[NB], key[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int i = base + b * 256;
          const int q = i % OWNC, cell = i / OWNC;
          const int comp = q % NC, nd = q / NC;
          const int a = nd % P, bb = (nd / P) % P, cc = DIM == 3 ? nd / (P * P) : 0;
          const int ox = cell % C::TX, oy = (cell / C::TX) % C::TY, oz = DIM == 3 ? cell / (C::TX * C::TY) : 0;
          const bool act = i < TOT && ox < tx && oy < ty && oz < tz;
          const int lx = ox * P + a, ly = oy * P + bb, lz = oz * P + cc;
          const int64_t dof = (((int64_t)(oz0 + lz) * pb.lat[1] + (oy0 + ly)) * pb.lat[0] + (ox0 + lx)) * NC + comp;
          // own cell (ox + 1, oy + 1[, oz + 1]) of the halo'd tile and the node's row in it
          const int m = ((DIM == 3 ? oz + 1 : 0) * EY + (oy + 1)) * EX + (ox + 1);
          const int row = (((DIM == 3 ? cc * NN1 : 0) + bb) * NN1 + a) * NC + comp;
          dofv[b] = act ? dof : -1;
          yix[b] = m * NL + row;
          key[b] = (a == 0 ? 1 : 0) | (bb == 0 ? 2 : 0) | (DIM == 3 && cc == 0 ? 4 : 0);
          upv[b] = 0.0;
          ukv[b] = 0.0;
          mhv[b] = 0.f;
          mlv[b] = 0.f;
          if (act && mode != kModeApply) {
            mhv[b] = __ldg(pb.minv32 + dof);
            mlv[b] = __ldg(pb.minv32 + pb.n_lat_dof + dof);
            upv[b] = out[dof];
            ukv[b] = pf[(((DIM == 3 ? lz + P : 0) * PY + (ly + P)) * PX + (lx + P)) * NC + comp];
          }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (dofv[b] < 0) continue;
          // level-0 parts summed error-free in FP32 (sh + se is their exact sum)
          float sh = 0.f, se = 0.f, lo = 0.f;
#pragma unroll
          for (int jz = 0; jz < (DIM == 3 ? 2 : 1); ++jz)
#pragma unroll
            for (int jy = 0; jy < 2; ++jy)
#pragma unroll
              for (int jx = 0; jx < 2; ++jx) {
                const bool val = (jx || (key[b] & 1)) && (jy || (key[b] & 2)) && (DIM == 2 || jz || (key[b] & 4));
                if (val) {
                  const int off_n = (jx ? 0 : DX) + (jy ? 0 : DY) + (DIM == 3 && !jz ? DZ : 0);
                  const float2 y = yb[yix[b] - off_n];
                  float t1, t2;
                  two_sum(sh, y.x, t1, t2);
                  sh = t1;
                  se += t2;
                  lo += y.y;
                }
              }
          update(dofv[b], sh, se, lo, ukv[b], upv[b], mhv[b], mlv[b]);
        }
      }
    }
    // nodes on the domain's high faces (their cell's local index P): generic search of the
    // (up to 2^DIM) cells that hold them, in the same order
    if (X1 == pb.n[0] || Y1 == pb.n[1] || (DIM == 3 && Z1 == pb.n[2])) {
      const int ex_ = (X1 - X0) * P, ey_ = (Y1 - Y0) * P, ez_ = DIM == 3 ? (Z1 - Z0) * P : 0;
      const int nox = ex_ + (X1 == pb.n[0] ? 1 : 0);
      const int noy = ey_ + (Y1 == pb.n[1] ? 1 : 0);
      const int noz = DIM == 3 ? ez_ + (Z1 == pb.n[2] ? 1 : 0) : 1;
      const int total = nox * noy * noz * NC;
      for (int i = tid; i < total; i += blockDim.x) {
        const int comp = i % NC, node = i / NC;
        const int lx = node % nox, ly = (node / nox) % noy, lz = node / (nox * noy);
        if (!(lx == ex_ || ly == ey_ || (DIM == 3 && lz == ez_))) continue;   // first pass
        const int64_t dof = (((int64_t)(oz0 + lz) * pb.lat[1] + (oy0 + ly)) * pb.lat[0] + (ox0 + lx)) * NC + comp;
        const int px = lx + P, py = ly + P, pz = DIM == 3 ? lz + P : 0;
        const int cx = px / P, cy = py / P, cz = DIM == 3 ? pz / P : 0;
        const bool bx = px - cx * P == 0, by = py - cy * P == 0, bz = DIM == 3 && pz - cz * P == 0;
        float sh = 0.f, se = 0.f, lo = 0.f;
        for (int jz = 0; jz < (DIM == 3 ? 2 : 1); ++jz)
          for (int jy = 0; jy < 2; ++jy)
            for (int jx = 0; jx < 2; ++jx) {
              const int ecx = cx - 1 + jx, ecy = cy - 1 + jy, ecz = DIM == 3 ? cz - 1 + jz : 0;
              const bool val = (jx ? cx < EX : bx) && (jy ? cy < EY : by) && (DIM == 2 || (jz ? cz < C::EZ : bz));
              if (val) {
                const int m = (ecz * EY + ecy) * EX + ecx;
                const int row = (((DIM == 3 ? (pz - ecz * P) * NN1 : 0) + (py - ecy * P)) * NN1 + (px - ecx * P)) * NC + comp;
                const float2 y = yb[m * NL + row];
                float t1, t2;
                two_sum(sh, y.x, t1, t2);
                sh = t1;
                se += t2;
                lo += y.y;
              }
            }
        float mh = 0.f, ml = 0.f;
        double upv = 0.0, uval = 0.0;
        if (mode != kModeApply) {
          mh = __ldg(pb.minv32 + dof);
          ml = __ldg(pb.minv32 + pb.n_lat_dof + dof);
          upv = out[dof];
          uval = pf[(((DIM == 3 ? lz + P : 0) * PY + (ly + P)) * PX + (lx + P)) * NC + comp];
        }
        update(dof, sh, se, lo, uval, upv, mh, ml);
      }
    }
    // the load F_k of this tile's DOFs (each DOF once per tile), added after the update in
    // FP64: u^{k+1} += (dt^2 / m) F_k (start-up step: half of it)
    if (src_lo < src_hi && mode != kModeApply) {
      __syncthreads();   // this tile's updates of `out` are visible to every thread
      const double w = mode == kModeStartup ? 0.5 : 1.0;
      for (int s2 = src_lo + tid; s2 < src_hi; s2 += blockDim.x) {
        const int64_t dof = pb.tsrc_dof[s2];
        const double mi = pb.minv[dof];
        if (mi > 0.0) out[dof] = fma(w * mi, pb.tsrc_val[s2] * fk, out[dof]);
      }
    }
    if (BATCH && bad) {
      atomicOr(pb.flags, 1);
      bad = false;
    }
    ++mma_phase;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();   // patch (prefetched), lists, A/ybuf and next_tile are reused by the next tile
    if (have_patch) pcur ^= 1;
  }
  if (!BATCH && bad) atomicOr(pb.flags, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
  }
  if (tid == 0) {
    __threadfence();
    unsigned int* const donep = BATCH ? &ctl->done : pb_arg.done;
    unsigned prev = atomicAdd(donep, 1u);
    if (prev == gridDim.x - 1) {
      if constexpr (BATCH) {
        for (int m = 0; m < n_members; ++m) {
          unsigned long long* sp = members[m].pb.step;
          const unsigned long long km = *((volatile unsigned long long*)sp);
          if (km < members[m].step_end) *sp = km + 1;
        }
      } else {
        if (mode == kModeCDM) *pb_arg.step = k + 1;
      }
      *tcount = 0;
      *donep = 0u;
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

void op_tc_tiles(int dim, int p, int ncomp, int variant, int* t) {
  int nl = ncomp;
  for (int k = 0; k < dim; ++k) nl *= p + 1;
  t[0] = tc_tile_x(dim, nl, variant);
  t[1] = tc_tile_y(dim, nl, variant);
  t[2] = tc_tile_z(dim, variant);
}

void op_tc_dims(int dim, int p, int ncomp, int* kp, int* np) {
  int nl = ncomp;
  for (int k = 0; k < dim; ++k) nl *= p + 1;
  *kp = (nl + 15) / 16 * 16;
  *np = (nl + 15) / 16 * 16;
}

int op_tc_core_offset(int kp, int row, int k) {
  return (row >> 3) * (kp / 8) * 64 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

// Resident CTAs per SM of one instantiation, from the kernel's own limits: registers,
// shared memory (plus the 1 KB the runtime reserves per CTA), threads and the 512 TMEM
// columns.  Also raises the dynamic shared memory limit and the carveout (all of the unified
// L1/shared storage as shared memory).  Returns 0 on failure.
template <typename KernelT>
static int tc_configure(KernelT kernel, size_t smem_launch, int tmem_max) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_launch) != cudaSuccess)
    return 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return 0;
  int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 0;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
  const int by_regs = regs_sm / (regs_warp * (256 / 32));
  const int by_smem = smem_sm / ((int)smem_launch + 1024 + (int)fa.sharedSizeBytes);
  int per_sm = std::min(std::min(by_regs, by_smem), std::min(tmem_max, 2048 / 256));
  if (per_sm < 1) per_sm = 1;
  return per_sm * sms;
}

template <int D, int P, int N, int S, int T>
static cudaError_t launch_tc_t(const DevProblem& pb, const double* u, double* out, int mode, int ctas_per_sm,
                               cudaStream_t st) {
  using C = TcCfg<D, P, N, T>;
  // thread-safe one-time configuration (function-local static initialisation)
  static const int resident = tc_configure(op_tc_kernel<D, P, N, S, false, T>, C::SMEM_LAUNCH, C::CTA_TMEM_MAX);
  if (resident == 0) return cudaErrorInvalidConfiguration;
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
  }();
  int tiles = pb.tc_tiles[0] * pb.tc_tiles[1] * pb.tc_tiles[2];
  int blocks = std::min(tiles, ctas_per_sm > 0 ? std::min(resident, ctas_per_sm * sms) : resident);
  op_tc_kernel<D, P, N, S, false, T><<<blocks, 256, C::SMEM_LAUNCH, st>>>(pb, u, out, mode, nullptr, nullptr, 0, 0,
                                                                         nullptr);
  return cudaGetLastError();
}

template <int D, int P, int N, int T>
static cudaError_t launch_tc_batch_t(const BatchMember* members, const int* tile_start, int n_members,
                                     int total_tiles, BatchCtl* ctl, cudaStream_t st) {
  using C = TcCfg<D, P, N, T>;
  constexpr size_t smem = std::max(C::SMEM + (sizeof(BatchMember) + 15) / 16 * 16, C::SMEM_FLOOR);
  static const int resident = tc_configure(op_tc_kernel<D, P, N, 0, true, T>, smem, C::CTA_TMEM_MAX);
  if (resident == 0) return cudaErrorInvalidConfiguration;
  if (total_tiles <= 0) return cudaSuccess;
  int blocks = std::min(total_tiles, resident);
  DevProblem none{};
  op_tc_kernel<D, P, N, 0, true, T><<<blocks, 256, smem, st>>>(none, nullptr, nullptr, kModeCDM, members, tile_start,
                                                               n_members, total_tiles, ctl);
  return cudaGetLastError();
}

cudaError_t launch_op_tc_batch(int dim, int p, int ncomp, int variant, const BatchMember* members,
                               const int* tile_start, int n_members, int total_tiles, BatchCtl* ctl,
                               cudaStream_t st) {
#define X(D, P, N)                                                                                       \
  if (dim == D && p == P && ncomp == N) {                                                                \
    if (variant == 1) return launch_tc_batch_t<D, P, N, 1>(members, tile_start, n_members, total_tiles, ctl, st); \
    return launch_tc_batch_t<D, P, N, 0>(members, tile_start, n_members, total_tiles, ctl, st);          \
  }
  IBFEM_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

// the small tile (variant 1) exists for the exact scheme, which is the one the batch and
// the serving loop run
cudaError_t launch_op_tc(const DevProblem& pb, const double* u, double* out, int mode, int scheme, int variant,
                         cudaStream_t st, int ctas_per_sm) {
#define X(D, P, N)                                                                 \
  if (pb.dim == D && pb.p == P && pb.ncomp == N) {                                 \
    if (scheme == 0 && variant == 1) return launch_tc_t<D, P, N, 0, 1>(pb, u, out, mode, ctas_per_sm, st); \
    if (variant != 0) return cudaErrorInvalidValue;                                \
    if (scheme == 0) return launch_tc_t<D, P, N, 0, 0>(pb, u, out, mode, ctas_per_sm, st);      \
    if (scheme == 1) return launch_tc_t<D, P, N, 1, 0>(pb, u, out, mode, ctas_per_sm, st);      \
    return launch_tc_t<D, P, N, 2, 0>(pb, u, out, mode, ctas_per_sm, st);                       \
  }
  IBFEM_TC_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace ibfem
