// Device helpers shared by the tensor-core operator kernels (kernels_tc.cu, kernels_tc64.cu):
// shared-memory addresses, exact FP32 <-> FP64 bit conversions, UMMA descriptors and MMA
// issue, bounded mbarrier waits, error-free FP32 sums, asynchronous copies, BF16 digits of
// small integers, and the tile shapes of the persistent kernels.
#pragma once

#include <cstdint>

#include "internal.h"

namespace ibfem {
namespace tc {


__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// FP32 -> FP64 exactly by bit manipulation with an extra power-of-two scale 2^sh
// (integer pipe only; zero and subnormal inputs give zero).
__device__ __forceinline__ double f32_to_f64_scaled(float f, int sh) {
  uint32_t b = __float_as_uint(f);
  int e = (int)((b >> 23) & 0xffu);
  if (e == 0) return 0.0;
  uint32_t sign = b & 0x80000000u, m = b & 0x7fffffu;
  int e64 = e + 896 + sh;
  if (e64 <= 0) return 0.0;                                   // below FP64 normals: negligible
  if (e64 >= 2047) return __hiloint2double((int)(sign | 0x7ff00000u), 0);
  uint32_t hi = sign | ((uint32_t)e64 << 20) | (m >> 3);
  uint32_t lo = m << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// f * 2^sh in FP32 by exponent arithmetic (flush to zero on underflow)
__device__ __forceinline__ float f32_scale(float f, int sh) {
  uint32_t b = __float_as_uint(f);
  int e = (int)((b >> 23) & 0xffu);
  if (e == 0) return 0.f;
  int e2 = e + sh;
  if (e2 <= 0) return 0.f;
  if (e2 >= 255) return __uint_as_float((b & 0x80000000u) | 0x7f800000u);
  return __uint_as_float((b & 0x807fffffu) | ((uint32_t)e2 << 23));
}

// FP64 -> FP32 rounding to nearest by bit manipulation (ties away from zero).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  uint32_t sign = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7ffu) - 896;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  uint32_t r = ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  r += (lo >> 28) & 1u;  // carry may bump the exponent: still correct
  return __uint_as_float(sign | r);
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

// FP32 value of a small integer v (|v| < 2^22) without the conversion pipe: the pattern
// of 1.5 * 2^23 plus v is the float 1.5 * 2^23 + v (unit spacing in [2^23, 2^24)), and
// subtracting 1.5 * 2^23 leaves v exactly.
__device__ __forceinline__ uint32_t f32_bits_of_small_int(int v) {
  return __float_as_uint(__int_as_float(0x4B400000 + v) - 12582912.0f);
}

// Two BF16 values of small integers (|v| <= 256: at most 8 significant bits, so the upper
// half of the FP32 pattern is exact) packed as (a | b << 16).
__device__ __forceinline__ uint32_t bf16x2_of_small_ints(int a, int b) {
  return __byte_perm(f32_bits_of_small_int(a), f32_bits_of_small_int(b), 0x7632);
}

__device__ __forceinline__ uint16_t bf16_rn(float f) {
  uint32_t b = __float_as_uint(f);
  b += 0x7fffu + ((b >> 16) & 1u);  // round to nearest even (finite inputs)
  return (uint16_t)(b >> 16);
}

// Bounded wait for the phase `parity` of an mbarrier: at most `polls` try_wait calls (each
// may suspend the thread for a hardware-defined while); false when the phase never came.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int polls = 1 << 24) {
  uint32_t ok = 0;
  for (int it = 0; it < polls && !ok; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
  return ok != 0;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// error-free transformations of double-FP32 arithmetic
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}


// Asynchronous copy global -> shared of 8 or 16 bytes; src_bytes = 0 writes zeros.
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

}  // namespace tc

// Tile shapes (owned cells per axis; the halo adds one cell on the low side of each axis,
// and the halo'd tile must fit the M = 128 rows of one MMA).  Variant 0 fills the MMA;
// variant 1 is a smaller tile (more tiles for small problems, less shared memory in 3D);
// the autotuner picks between them per problem.
__host__ __device__ constexpr int tc_tile_x(int dim, int nl, int v) {
  return dim == 3 ? (v ? 3 : 4) : (nl >= 32 ? (v ? 5 : 8) : (v ? 7 : 15));
}
__host__ __device__ constexpr int tc_tile_y(int dim, int nl, int v) {
  return dim == 3 ? (v ? 3 : 4) : (nl >= 32 ? (v ? 5 : 8) : 7);
}
__host__ __device__ constexpr int tc_tile_z(int dim, int v) { return dim == 3 ? (v ? 3 : 4) : 1; }

template <int KP>
__host__ __device__ __forceinline__ int bf16_core_offset(int row, int k) {
  return (row >> 3) * (KP / 8) * 64 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

}  // namespace ibfem
