// C ABI runtime: handle, device buffers, CUDA-graph replay of the per-step kernels.
//
// The public functions are declared and documented in include/ibfem.h.  The time step
// is Eq. cdm of Buerchner et al. (arXiv 2501.19013); the critical step follows Sec. 2.3.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ibfem.h"
#include "host_setup.h"
#include "internal.h"
#include "runtime_internal.h"

using namespace ibfem;

namespace {
thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

struct CudaFail : std::runtime_error {
  explicit CudaFail(const std::string& m) : std::runtime_error(m) {}
};

void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw CudaFail(std::string(what) + ": " + cudaGetErrorString(e));
}
}  // namespace

namespace ibfem {

void* Handle::dalloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (opt.dev_alloc) {
    p = opt.dev_alloc(bytes, opt.alloc_ctx);
    if (!p) throw std::bad_alloc();
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
  }
  if (to_shared) {
    shared->ptrs.push_back(p);
    shared->bytes += bytes;
  } else {
    allocs.push_back(p);
    device_bytes += bytes;
  }
  return p;
}

void Handle::dfree_all() {
  for (void* p : allocs) {
    if (opt.dev_free) opt.dev_free(p, opt.alloc_ctx);
    else cudaFree(p);
  }
  allocs.clear();
  device_bytes = 0;
  shared.reset();   // the last handle of a discretisation frees its shared arrays
  to_shared = false;
}

DeviceShared::~DeviceShared() {
  cudaSetDevice(device);
  for (void* p : ptrs) {
    if (dev_free) dev_free(p, alloc_ctx);
    else cudaFree(p);
  }
}

template <typename T>
T* Handle::upload(const std::vector<T>& v) {
  T* d = static_cast<T*>(dalloc(std::max<size_t>(v.size(), 1) * sizeof(T)));
  if (!v.empty()) check(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, stream), "upload");
  return d;
}

void Handle::to_lattice(const double* kept, std::vector<double>& lat) const {
  lat.assign(setup.n_lat_dof, 0.0);
  if (!kept) return;
  const int nc = setup.ncomp;
  for (int64_t i = 0; i < setup.n_kept_nodes; ++i)
    for (int c = 0; c < nc; ++c) lat[setup.lat_of_kept[i] * nc + c] = kept[i * nc + c];
}

void Handle::from_lattice(const std::vector<double>& lat, double* kept) const {
  const int nc = setup.ncomp;
  for (int64_t i = 0; i < setup.n_kept_nodes; ++i)
    for (int c = 0; c < nc; ++c) kept[i * nc + c] = lat[setup.lat_of_kept[i] * nc + c];
}

void Handle::build_device() {
  const Setup& s = setup;
  DevProblem& pb = dev;
  std::memset(&pb, 0, sizeof(pb));
  pb.dim = s.dim;
  pb.p = s.p;
  pb.ncomp = s.ncomp;
  pb.n_loc = s.n_loc;
  pb.nn_loc = s.nn_loc;
  for (int k = 0; k < 3; ++k) {
    pb.n[k] = s.n[k];
    pb.lat[k] = (int)s.lat[k];
  }
  pb.n_lat_dof = s.n_lat_dof;
  shared = std::make_shared<DeviceShared>();
  shared->device = opt.device;
  shared->dev_free = opt.dev_free;
  shared->alloc_ctx = opt.alloc_ctx;
  to_shared = true;   // geometry and matrices: shared with clones
  pb.cls = upload(s.cls);
  pb.cut_index = upload(s.cut_index);
  pb.cut_mat = upload(s.cut_mat);
  pb.cut_cell = upload(s.cut_cells);
  pb.n_cut = (int)s.n_cut;
  pb.Kref = upload(s.Kref);
  pb.Kcut = upload(s.Kcut);
  to_shared = false;
  pb.Ycut = static_cast<double*>(dalloc(std::max<int64_t>(s.n_cut, 1) * s.n_loc * sizeof(double)));
  // 1/M_L (dt = 1 until set_dt) and 1/sqrt(M_L)
  std::vector<double> minv(s.n_lat_dof, 0.0), sinv(s.n_lat_dof, 0.0);
  for (int64_t i = 0; i < s.n_lat_dof; ++i)
    if (s.ML[i] > 0) {
      minv[i] = 1.0 / s.ML[i];
      sinv[i] = 1.0 / std::sqrt(s.ML[i]);
    }
  if (imex)
    for (int64_t ci = 0; ci < imex_host.n_c; ++ci) sinv[imex_host.c_dof[ci]] = 0.0;  // d-block only
  d_minv = upload(minv);
  pb.minv = d_minv;
  to_shared = !imex;   // IMEX zeroes its c-DOFs in 1/sqrt(M_L): then it is the handle's own
  pb.sinv = upload(sinv);
  to_shared = false;
  if (imex) {
    const ImexData& I = imex_host;
    ImexDev& D = imex_dev;
    std::memset(&D, 0, sizeof(D));
    D.n_cells = (int)I.ccells.size();
    D.cells = upload(I.ccells);
    D.Y = static_cast<double*>(dalloc(std::max<size_t>(I.ccells.size(), 1) * s.n_loc * sizeof(double)));
    D.n_rows = I.n_c;
    D.g_ptr = upload(I.g_ptr);
    D.g_idx = upload(I.g_idx);
    D.work = static_cast<double*>(dalloc(I.n_c * sizeof(double)));
    D.perm = upload(I.perm);
    D.c_dof = upload(I.c_dof);
    D.vc = static_cast<double*>(dalloc(I.n_c * sizeof(double)));
    D.ac = static_cast<double*>(dalloc(I.n_c * sizeof(double)));
    check(cudaMemsetAsync(D.vc, 0, I.n_c * sizeof(double), stream), "memset");
    check(cudaMemsetAsync(D.ac, 0, I.n_c * sizeof(double), stream), "memset");
    pb.imex_vc = D.vc;
    pb.imex_ac = D.ac;
  }
  for (int b = 0; b < 2; ++b) {
    U[b] = static_cast<double*>(dalloc(s.n_lat_dof * sizeof(double)));
    check(cudaMemsetAsync(U[b], 0, s.n_lat_dof * sizeof(double), stream), "memset");
  }
  W = static_cast<double*>(dalloc(s.n_lat_dof * sizeof(double)));
  check(cudaMemsetAsync(W, 0, s.n_lat_dof * sizeof(double), stream), "memset");
  counters = static_cast<unsigned long long*>(dalloc(4 * sizeof(unsigned long long)));
  check(cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), stream), "memset");
  pb.step = counters;
  pb.done = reinterpret_cast<unsigned int*>(counters + 1);
  pb.flags = reinterpret_cast<int*>(counters + 2);
  pb.tile_counter = reinterpret_cast<int*>(counters + 3);
  if (imex) imex_dev.flags = pb.flags;
  op_fp64_tiles(s.dim, s.p, s.ncomp, tile);
  for (int k = 0; k < 3; ++k) pb.tiles[k] = k < s.dim ? (s.n[k] + tile[k] - 1) / tile[k] : 1;
  n_blocks = op_fp64_blocks(pb);
  partials = static_cast<double*>(dalloc(2 * (size_t)n_blocks * sizeof(double)));
  if (opt.precision != IBFEM_FP64) {
    // K_ref as the UMMA B operand (row i = K_ref[i, :], K-major BF16 core matrices), four
    // slices: balanced 8-bit digits (exact scheme) or BF16 hi / lo splits
    int kp = 0, np = 0;
    op_tc_dims(s.dim, s.p, s.ncomp, &kp, &np);
    const size_t slice = (size_t)np * kp;
    const bool fp64grade = tc_scheme() == 3;
    std::vector<uint16_t> img((fp64grade ? 7 : 4) * slice, 0);
    std::vector<int> frow(np, 0);
    auto bf16 = [](float f) {
      uint32_t b;
      std::memcpy(&b, &f, 4);
      b += 0x7fffu + ((b >> 16) & 1u);
      return (uint16_t)(b >> 16);
    };
    auto bf16_to_f = [](uint16_t h) {
      uint32_t b = (uint32_t)h << 16;
      float f;
      std::memcpy(&f, &b, 4);
      return f;
    };
    // FP64-grade scheme: one exponent G for the whole matrix (max |K| < 2^(G + 1)) and seven
    // balanced 8-bit digits of round(|K_ij| 2^(54 - G)) < 2^55 (|digit| <= 128)
    int G = 0;
    if (fp64grade) {
      double amax = 0.0;
      for (double v : s.Kref) amax = std::max(amax, std::fabs(v));
      if (amax > 0.0) {
        G = (int)std::floor(std::log2(amax));
        if (std::ldexp(1.0, G + 1) <= amax) ++G;
        if (std::ldexp(1.0, G) > amax) --G;
      }
      for (int i = 0; i < s.n_loc; ++i)
        for (int j = 0; j < s.n_loc; ++j) {
          const double v = s.Kref[(size_t)i * s.n_loc + j];
          unsigned long long W = (unsigned long long)std::llround(std::ldexp(std::fabs(v), 54 - G));
          long long c[7];
          int carry = 0;
          for (int b = 0; b < 7; ++b) {   // byte b of W is digit 6 - b
            int t = (int)((W >> (8 * b)) & 0xffu) + carry;
            if (b < 6) {
              carry = t >= 128 ? 1 : 0;
              t -= carry << 8;
            }
            c[6 - b] = v < 0 ? -t : t;
          }
          const int o = op_tc_core_offset(kp, i, j);
          for (int t = 0; t < 7; ++t) img[t * slice + o] = bf16((float)c[t]);
        }
    }
    for (int i = 0; i < s.n_loc && !fp64grade; ++i) {
      double amax = 0.0;
      for (int j = 0; j < s.n_loc; ++j) amax = std::max(amax, std::fabs(s.Kref[(size_t)i * s.n_loc + j]));
      int F = 0;
      if (amax > 0.0) F = (int)std::floor(std::log2(amax));
      if (amax > 0.0 && std::ldexp(1.0, F + 1) <= amax) ++F;   // guard log2 rounding
      if (amax > 0.0 && std::ldexp(1.0, F) > amax) --F;
      frow[i] = F;
      for (int j = 0; j < s.n_loc; ++j) {
        double v = s.Kref[(size_t)i * s.n_loc + j];
        int o = op_tc_core_offset(kp, i, j);
        if (tc_scheme() == 0) {
          long long W = std::llround(std::ldexp(v, 31 - F));
          long long c0 = (W + (1ll << 23)) >> 24;
          long long r = W - (c0 << 24);
          long long c1 = (r + (1ll << 15)) >> 16;
          r -= c1 << 16;
          long long c2 = (r + (1ll << 7)) >> 8;
          long long c3 = r - (c2 << 8);
          long long c[4] = {c0, c1, c2, c3};
          for (int t = 0; t < 4; ++t) img[t * slice + o] = bf16((float)c[t]);
        } else {
          uint16_t h = bf16((float)v);
          img[o] = h;
          if (tc_scheme() == 1) img[slice + o] = bf16((float)(v - (double)bf16_to_f(h)));
        }
      }
    }
    to_shared = true;
    pb.tc_bimg = upload(img);
    pb.tc_frow = upload(frow);
    pb.tc_gexp = G;
    tc_img_host = img;
    tc_frow_host = frow;
    if (fp64grade) {
      // the FP64 cut-cell kernel supplies the cut products; dt^2 / M_L is read in FP64
      to_shared = false;
      tc_variant = op_tc64_variant(s.dim);
    } else {
      // cut matrices as interleaved (hi, lo) FP32 pairs: one 8-byte load per entry
      std::vector<float> k32(2 * (size_t)s.n_cut_mat * s.n_loc * s.n_loc);
      const size_t nl2 = (size_t)s.n_loc * s.n_loc;
      for (int64_t c = 0; c < s.n_cut_mat; ++c)
        for (size_t q = 0; q < nl2; ++q) {
          double v = s.Kcut[c * nl2 + q];
          float h = (float)v;
          k32[2 * (c * nl2 + q)] = h;
          k32[2 * (c * nl2 + q) + 1] = (float)(v - (double)h);
        }
      pb.Kcut32 = upload(k32);
      to_shared = false;
      std::vector<float> m32(2 * (size_t)s.n_lat_dof, 0.f);
      for (int64_t i = 0; i < s.n_lat_dof; ++i)
        if (s.ML[i] > 0) {
          double v = 1.0 / s.ML[i];
          float h = (float)v;
          m32[i] = h;
          m32[s.n_lat_dof + i] = (float)(v - (double)h);
        }
      d_minv32 = upload(m32);
      pb.minv32 = d_minv32;
    }
    build_tc_tiles();
  }
  scalars = static_cast<double*>(dalloc(8 * sizeof(double)));
  lam_hist = static_cast<double*>(dalloc(kPowerChunk * sizeof(double)));
  scratch = static_cast<double*>(dalloc(s.n_lat_dof * sizeof(double)));
  check(cudaStreamSynchronize(stream), "setup sync");
}

// a clone: the source's shared arrays, its own state, work arrays, counters and
// dt^2 / M_L (copied from the source, so the source's dt carries over); no load and no
// observers until they are set
void Handle::build_clone(const Handle& src) {
  const Setup& s = setup;
  DevProblem& pb = dev;
  pb = src.dev;
  pb.src_ptr = nullptr;
  pb.src_dof = nullptr;
  pb.src_val = nullptr;
  pb.f_e = 0.0;
  pb.tsrc_ptr = nullptr;
  pb.tsrc_dof = nullptr;
  pb.tsrc_val = nullptr;
  pb.n_obs_rows = 0;
  pb.obs_dof = nullptr;
  pb.obs_w = nullptr;
  pb.ring = nullptr;
  pb.ring_cap = 0;
  pb.imex_vc = nullptr;
  pb.imex_ac = nullptr;
  pb.Ycut = static_cast<double*>(dalloc(std::max<int64_t>(s.n_cut, 1) * s.n_loc * sizeof(double)));
  d_minv = static_cast<double*>(dalloc(s.n_lat_dof * sizeof(double)));
  check(cudaMemcpyAsync(d_minv, src.d_minv, s.n_lat_dof * sizeof(double), cudaMemcpyDeviceToDevice, stream), "minv");
  pb.minv = d_minv;
  for (int b = 0; b < 2; ++b) {
    U[b] = static_cast<double*>(dalloc(s.n_lat_dof * sizeof(double)));
    check(cudaMemsetAsync(U[b], 0, s.n_lat_dof * sizeof(double), stream), "memset");
  }
  W = static_cast<double*>(dalloc(s.n_lat_dof * sizeof(double)));
  check(cudaMemsetAsync(W, 0, s.n_lat_dof * sizeof(double), stream), "memset");
  counters = static_cast<unsigned long long*>(dalloc(4 * sizeof(unsigned long long)));
  check(cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), stream), "memset");
  pb.step = counters;
  pb.done = reinterpret_cast<unsigned int*>(counters + 1);
  pb.flags = reinterpret_cast<int*>(counters + 2);
  pb.tile_counter = reinterpret_cast<int*>(counters + 3);
  partials = static_cast<double*>(dalloc(2 * (size_t)n_blocks * sizeof(double)));
  if (src.d_minv32) {
    d_minv32 = static_cast<float*>(dalloc(2 * s.n_lat_dof * sizeof(float)));
    check(cudaMemcpyAsync(d_minv32, src.d_minv32, 2 * s.n_lat_dof * sizeof(float), cudaMemcpyDeviceToDevice,
                          stream), "minv32");
    pb.minv32 = d_minv32;
  }
  if (opt.precision != IBFEM_FP64)
    build_tc_tiles();   // the source's tile order may be its own array (a later tile variant)
  scalars = static_cast<double*>(dalloc(8 * sizeof(double)));
  lam_hist = static_cast<double*>(dalloc(kPowerChunk * sizeof(double)));
  scratch = static_cast<double*>(dalloc(s.n_lat_dof * sizeof(double)));
  check(cudaStreamSynchronize(stream), "clone sync");
}

// tile grid of the tensor-core kernel for the current tile variant and the processing
// order of its tiles: the persistent kernel hands tiles out in this order, so the slow ones
// (cut cells of the halo'd tile run on the CUDA cores, one warp per cell, eight at a time)
// start first and short tiles fill the end of the step
void Handle::build_tc_tiles() {
  const Setup& s = setup;
  DevProblem& pb = dev;
  op_tc_tiles(s.dim, s.p, s.ncomp, tc_variant, tc_tile);
  for (int k = 0; k < 3; ++k) pb.tc_tiles[k] = k < s.dim ? (s.n[k] + tc_tile[k] - 1) / tc_tile[k] : 1;
  const int ntx = pb.tc_tiles[0], nty = pb.tc_tiles[1], ntz = pb.tc_tiles[2];
  std::vector<int> ncut_tile((size_t)ntx * nty * ntz, 0);
  for (int t = 0; t < ntx * nty * ntz; ++t) {
    const int bx = t % ntx, by = (t / ntx) % nty, bz = t / (ntx * nty);
    int c = 0;
    for (int ez = (s.dim == 3 ? bz * tc_tile[2] - 1 : 0); ez < (s.dim == 3 ? (bz + 1) * tc_tile[2] : 1); ++ez)
      for (int ey = by * tc_tile[1] - 1; ey < (by + 1) * tc_tile[1]; ++ey)
        for (int ex = bx * tc_tile[0] - 1; ex < (bx + 1) * tc_tile[0]; ++ex) {
          if (ex < 0 || ey < 0 || ez < 0 || ex >= s.n[0] || ey >= s.n[1] || (s.dim == 3 && ez >= s.n[2])) continue;
          if (s.cls[((int64_t)ez * s.n[1] + ey) * s.n[0] + ex] == kCut) ++c;
        }
    ncut_tile[t] = (c + 7) / 8;   // rounds of eight warps
  }
  std::vector<int32_t> order(ncut_tile.size());
  for (size_t t = 0; t < order.size(); ++t) order[t] = (int32_t)t;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return ncut_tile[a] > ncut_tile[b]; });
  pb.tc_order = upload(order);
}

// the load CSR over the tensor-core tiles (rebuilt when the tile variant changes)
void Handle::upload_tc_sources() {
  const Setup& s = setup;
  const int nt = dev.tc_tiles[0] * dev.tc_tiles[1] * dev.tc_tiles[2];
  std::vector<std::vector<std::pair<int64_t, double>>> per2(nt);
  for (auto& e : src_host) {
    int64_t rem = e.first / s.ncomp;
    int t = 0, stride = 1;
    for (int k = 0; k < s.dim; ++k) {
      int64_t g = rem % s.lat[k];
      rem /= s.lat[k];
      int b = (int)std::min<int64_t>(g / ((int64_t)tc_tile[k] * s.p), dev.tc_tiles[k] - 1);
      t += b * stride;
      stride *= dev.tc_tiles[k];
    }
    per2[t].push_back(e);
  }
  std::vector<int32_t> p2(nt + 1, 0);
  std::vector<int64_t> d2;
  std::vector<double> v2;
  for (int t = 0; t < nt; ++t) {
    for (auto& e : per2[t]) {
      d2.push_back(e.first);
      v2.push_back(e.second);
    }
    p2[t + 1] = (int32_t)d2.size();
  }
  dev.tsrc_ptr = upload(p2);
  dev.tsrc_dof = upload(d2);
  dev.tsrc_val = upload(v2);
}

void Handle::set_tc_variant(int v) {
  if (v == tc_variant) return;
  tc_variant = v;
  build_tc_tiles();
  if (dev.tsrc_ptr) upload_tc_sources();
  invalidate_graphs();
  check(cudaStreamSynchronize(stream), "tile variant");
}

size_t Handle::planned_device_bytes() const {
  const Setup& s = setup;
  auto arr = [](int64_t count, size_t elem) { return (size_t)std::max<int64_t>(count, 1) * elem; };
  const int64_t nl = s.n_loc, nlat = s.n_lat_dof, ncut = s.n_cut, nel = s.n_elem, nmat = s.n_cut_mat;
  size_t b = 0;
  b += arr(nel, 1) + arr(nel, 4) + arr(ncut, 8) + arr(ncut, 4);   // cls, cut_index, cut_cells, cut_mat
  b += arr(nl * nl, 8) + arr(nmat * nl * nl, 8);          // Kref, Kcut
  b += arr(ncut, 8) * nl;                                 // Ycut
  b += 2 * arr(nlat, 8);                                  // minv, sinv
  if (imex) {
    const ImexData& I = imex_host;
    const int64_t ncell = (int64_t)I.ccells.size();
    b += arr(ncell, 8) + arr(ncell, 8) * nl + arr((int64_t)I.g_ptr.size(), 8) +
         arr((int64_t)I.g_idx.size(), 4) + 3 * arr(I.n_c, 8) + arr((int64_t)I.perm.size(), 8) +
         arr((int64_t)I.c_dof.size(), 8);
  }
  b += 3 * arr(nlat, 8) + 32;                             // U[2], W, counters
  int t[3] = {1, 1, 1};
  op_fp64_tiles(s.dim, s.p, s.ncomp, t);
  int64_t nb = 1;
  for (int k = 0; k < s.dim; ++k) nb *= (s.n[k] + t[k] - 1) / t[k];
  b += 2 * (size_t)nb * 8;                                // partials
  if (opt.precision != IBFEM_FP64) {
    int kp = 0, np = 0;
    op_tc_dims(s.dim, s.p, s.ncomp, &kp, &np);
    b += (tc_scheme() == 3 ? 7 : 4) * (size_t)kp * np * 2 + arr(np, 4);   // K_ref image, row exponents
    int tt[3] = {1, 1, 1};
    op_tc_tiles(s.dim, s.p, s.ncomp, tc_scheme() == 3 ? op_tc64_variant(s.dim) : tc_variant, tt);
    int64_t ntc = 1;
    for (int k = 0; k < s.dim; ++k) ntc *= (s.n[k] + tt[k] - 1) / tt[k];
    b += arr(ntc, 4);                                     // tile order
    if (tc_scheme() != 3) b += arr(2 * nmat * nl * nl, 4) + arr(2 * nlat, 4);   // Kcut32, minv32
  }
  b += 64 + kPowerChunk * 8 + arr(nlat, 8);               // scalars, lam_hist, scratch
  return b;
}

// consistent-mass CDM: S = M^cc does not depend on dt, so it is factored once
void Handle::prepare_consistent() {
  std::string err;
  if (!imex_factor(setup, 0.0, imex_host, err)) throw std::runtime_error("consistent mass factorisation: " + err);
  imex_upload_factor();
  imex_dev.beta_dt2 = 0.0;
}

void Handle::imex_upload_factor() {
  const ImexData& I = imex_host;
  const SparseChol& L = I.chol;
  ImexDev& D = imex_dev;
  size_t nnz = L.Lx.size();
  const int64_t n_parts = std::max<int64_t>({I.fsplit.n_parts, I.bsplit.n_parts, 32});
  if (imex_nnz_alloc != nnz) {
    // the pattern, the order, the supernodes and the work split do not depend on dt:
    // uploaded once (32-bit column indices and entry offsets)
    if (nnz > (size_t)INT32_MAX || I.n_c > (int64_t)INT32_MAX)
      throw std::runtime_error("IMEX factor too large for 32-bit indices");
    const size_t nd = I.sn_D.size();
    std::vector<int32_t> li(std::max<size_t>(nnz, 1), 0), ui(li.size(), 0);
    for (size_t k = 0; k < nnz; ++k) {
      li[k] = (int32_t)L.Li[k];
      ui[k] = (int32_t)L.Ui[k];
    }
    D.Li = upload(li);
    D.Ui = upload(ui);
    D.Lx = static_cast<double*>(dalloc(std::max<size_t>(nnz, 1) * sizeof(double)));
    D.Ux = static_cast<double*>(dalloc(std::max<size_t>(nnz, 1) * sizeof(double)));
    D.D = static_cast<double*>(dalloc(std::max<size_t>(nd, 1) * sizeof(double)));
    D.DT = static_cast<double*>(dalloc(std::max<size_t>(nd, 1) * sizeof(double)));
    // one task per CTA of each sweep, in ticket order
    const size_t nsn = I.sn_start.size();
    for (int dir = 0; dir < 2; ++dir) {
      const ImexSplit& sp = dir == 0 ? I.fsplit : I.bsplit;
      std::vector<LevelTask> t;
      for (const int32_t q : sp.order)
        for (int32_t c = 0; c < sp.g[q]; ++c) {
          LevelTask e{};
          e.st = (int32_t)I.sn_start[q];
          e.wd_tpr = I.sn_size[q] | (sp.tpr[q] << 16);
          e.c = c;
          e.g = sp.g[q];
          e.doff = I.sn_doff[q];
          e.pbase = sp.pbase[q];
          e.sn = q;
          e.dep_beg = sp.dep_ptr[q];
          e.dep_n = sp.dep_ptr[q + 1] - sp.dep_ptr[q];
          t.push_back(e);
        }
      ImexSplitDev& sd = dir == 0 ? D.fs : D.bs;
      sd.n_tasks = (int)t.size();
      sd.task = upload(t);
      sd.dep = upload(sp.dep);
      sd.done = static_cast<unsigned int*>(dalloc(std::max<size_t>(nsn, 1) * sizeof(unsigned int)));
      check(cudaMemsetAsync(sd.done, 0, std::max<size_t>(nsn, 1) * sizeof(unsigned int), stream), "memset");
    }
    D.ctl = static_cast<SweepCtl*>(dalloc(sizeof(SweepCtl)));
    check(cudaMemsetAsync(D.ctl, 0, sizeof(SweepCtl), stream), "memset");
    D.part = static_cast<double*>(dalloc(n_parts * sizeof(double)));
    D.cnt = static_cast<unsigned int*>(dalloc((n_parts / 32) * sizeof(unsigned int)));
    // one 8-byte descriptor per row (its off-block entry range), so that a row costs one
    // load before its entries
    std::vector<int32_t> fd(2 * std::max<int64_t>(I.n_c, 1), 0), bd(fd.size(), 0);
    for (int64_t r = 0; r < I.n_c; ++r) {
      fd[2 * r] = (int32_t)L.Lp[r];
      fd[2 * r + 1] = (int32_t)I.f_off_end[r];
      bd[2 * r] = (int32_t)I.b_off_beg[r];
      bd[2 * r + 1] = (int32_t)L.Up[r + 1];
    }
    D.row_fdesc = reinterpret_cast<const int2*>(upload(fd));
    D.row_bdesc = reinterpret_cast<const int2*>(upload(bd));
    imex_nnz_alloc = nnz;
  }
  auto cp = [&](const void* dst, const void* src, size_t bytes) {
    if (bytes) check(cudaMemcpyAsync(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice, stream), "factor upload");
  };
  cp(D.Lx, L.Lx.data(), nnz * sizeof(double));
  cp(D.Ux, L.Ux.data(), nnz * sizeof(double));
  cp(D.D, I.sn_D.data(), I.sn_D.size() * sizeof(double));
  cp(D.DT, I.sn_DT.data(), I.sn_DT.size() * sizeof(double));
  check(cudaMemsetAsync(D.cnt, 0, (n_parts / 32) * sizeof(unsigned int), stream), "memset");
  check(cudaStreamSynchronize(stream), "factor upload");
}

void Handle::invalidate_graphs() {
  for (auto& g : graphs) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

void Handle::timed_begin(int slot) {
  if (!timing) return;
  while (ev_pool.size() < ev_used + 2) {
    cudaEvent_t e;
    check(cudaEventCreate(&e), "event");
    ev_pool.push_back(e);
  }
  check(cudaEventRecord(ev_pool[ev_used], stream), "event record");
  ev_slot.push_back(slot);
  n_slots = std::max(n_slots, slot + 1);
}

void Handle::timed_end() {
  if (!timing) return;
  check(cudaEventRecord(ev_pool[ev_used + 1], stream), "event record");
  ev_used += 2;
}

void Handle::timed_collect() {
  check(cudaStreamSynchronize(stream), "timed sync");
  for (size_t i = 0; i < ev_slot.size(); ++i) {
    float ms = 0.f;
    check(cudaEventElapsedTime(&ms, ev_pool[2 * i], ev_pool[2 * i + 1]), "elapsed");
    slot_ms[ev_slot[i]] += ms;
  }
  for (size_t s = 0; s < step_first_ev.size(); ++s) {
    float ms = 0.f;
    check(cudaEventElapsedTime(&ms, ev_pool[step_first_ev[s]], ev_pool[step_last_ev[s]]), "elapsed");
    slot_ms[0] += ms;
  }
  step_first_ev.clear();
  step_last_ev.clear();
  ev_slot.clear();
  ev_used = 0;
}

// One CDM step with u = U[cur], out = U[1 - cur] (in place over u^{k-1}).
void Handle::enqueue_step(int cur) {
  if (opt.precision == IBFEM_EXACT64_TC && !imex) {
    // FP64-grade tensor-core step: the FP64 cut-cell products (and the observers), then the
    // fused tensor-core operator and update
    OpInput x{U[cur], nullptr, nullptr};
    slot_name[1] = "cut_apply_fp64";
    slot_name[2] = "op_tc_exact64_fused_cdm";
    if (timing) step_first_ev.push_back(ev_used);
    timed_begin(1);
    check(launch_cut_apply_fp64(dev, x, true, stream), "cut_apply");
    timed_end();
    timed_begin(2);
    check(launch_op_tc64(dev, U[cur], U[1 - cur], kModeCDM, stream), "op_tc64");
    timed_end();
    if (timing) step_last_ev.push_back(ev_used - 1);
    return;
  }
  if (opt.precision != IBFEM_FP64 && opt.precision != IBFEM_EXACT64_TC && !imex) {
    slot_name[1] = tc_scheme() == 0 ? "op_tc_exact_fused_cdm" : (tc_scheme() == 1 ? "op_tc_bf16x3_fused_cdm" : "op_tc_bf16_fused_cdm");
    if (timing) step_first_ev.push_back(ev_used);
    timed_begin(1);
    check(launch_op_tc(dev, U[cur], U[1 - cur], kModeCDM, tc_scheme(), tc_variant, stream, tc_ctas), "op_tc");
    timed_end();
    if (timing) step_last_ev.push_back(ev_used - 1);
    return;
  }
  if (imex) {
    // Algorithm 2: the explicit part (d-DOF update and c-DOF predictor) by the FP64 kernel,
    // the FP64-grade or the exact tensor-core kernel, then the c-cells' products and the
    // c-set solve
    const bool tc64 = opt.precision == IBFEM_EXACT64_TC, tc = opt.precision == IBFEM_EXACT_TC;
    OpInput x{U[cur], nullptr, nullptr};
    slot_name[1] = "observers";
    slot_name[2] = tc64 ? "op_tc_exact64_fused_imex_explicit"
                        : (tc ? "op_tc_exact_fused_imex_explicit" : "op_fp64_fused_imex_explicit");
    slot_name[3] = "imex_cell_apply";
    slot_name[4] = "imex_solve";
    if (timing) step_first_ev.push_back(ev_used);
    timed_begin(1);
    check(launch_cut_apply_fp64(dev, x, true, stream, false), "observers");
    timed_end();
    timed_begin(2);
    if (tc64)
      check(launch_op_tc64(dev, U[cur], U[1 - cur], kModeImex, stream), "op_tc64_imex");
    else if (tc)
      check(launch_op_tc(dev, U[cur], U[1 - cur], kModeImex, tc_scheme(), tc_variant, stream, tc_ctas), "op_tc_imex");
    else
      check(launch_op_fp64(dev, x, U[1 - cur], kModeImex, nullptr, stream), "op_imex");
    timed_end();
    timed_begin(3);
    check(launch_imex_cell_apply(dev, imex_dev, U[1 - cur], stream), "imex_cells");
    timed_end();
    timed_begin(4);
    check(launch_imex_solve(dev, imex_dev, U[1 - cur], stream), "imex_solve");
    timed_end();
    if (timing) step_last_ev.push_back(ev_used - 1);
    return;
  }
  OpInput x{U[cur], nullptr, nullptr};
  slot_name[1] = "cut_apply_fp64";
  slot_name[2] = "op_fp64_fused_cdm";
  if (timing) step_first_ev.push_back(ev_used);
  timed_begin(1);
  check(launch_cut_apply_fp64(dev, x, true, stream), "cut_apply");
  timed_end();
  timed_begin(2);
  check(launch_op_fp64(dev, x, U[1 - cur], kModeCDM, nullptr, stream), "op_fused");
  timed_end();
  if (timing) step_last_ev.push_back(ev_used - 1);
}

void Handle::run_steps(int64_t n) {
  if (n <= 0) return;
  int64_t done_n = 0;
  // align to even parity so that the captured chunk starts with U[0] as u^k
  while (done_n < n && (cur != 0 || n - done_n < kGraphSteps)) {
    enqueue_step(cur);
    cur ^= 1;
    ++done_n;
  }
  while (n - done_n >= kGraphSteps) {
    if (!graphs[0]) {
      cudaGraph_t g;
      check(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      int c = 0;
      for (int i = 0; i < kGraphSteps; ++i) {
        enqueue_step(c);
        c ^= 1;
      }
      check(cudaStreamEndCapture(stream, &g), "end capture");
      cudaError_t e = cudaGraphInstantiate(&graphs[0], g, 0);
      cudaGraphDestroy(g);
      check(e, "graph instantiate");
    }
    check(cudaGraphLaunch(graphs[0], stream), "graph launch");
    done_n += kGraphSteps;  // kGraphSteps is even: parity unchanged
  }
  while (done_n < n) {
    enqueue_step(cur);
    cur ^= 1;
    ++done_n;
  }
}

}  // namespace ibfem

// ====================================================================== C ABI
#define IBFEM_TRY try {
#define IBFEM_CATCH                                                          \
  }                                                                          \
  catch (const CudaFail& e) { return fail(IBFEM_ERR_CUDA, e.what()); }      \
  catch (const std::bad_alloc&) { return fail(IBFEM_ERR_OOM, "allocation failed"); } \
  catch (const std::invalid_argument& e) { return fail(IBFEM_ERR_ARG, e.what()); } \
  catch (const std::domain_error& e) { return fail(IBFEM_ERR_GEOMETRY, e.what()); } \
  catch (const std::exception& e) { return fail(IBFEM_ERR_EIG, e.what()); }

namespace ibfem {
// lets other translation units report through ibfem_last_error()
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace ibfem

namespace {
void check_shape_supported(int dim, int p, int physics, int precision) {
  const int nc = physics == IBFEM_ELASTIC_PLANE_STRAIN ? 2 : 1;
  if (!op_fp64_supported(dim, p, nc)) throw std::invalid_argument("no kernel instantiation for this (dim, p, ncomp)");
  if (precision != IBFEM_FP64 && !op_tc_supported(dim, p, nc))
    throw std::invalid_argument("no tensor-core kernel instantiation for this (dim, p, ncomp)");
}

// device half of ibfem_create (and of ibfem_upload for a host-only handle)
void attach_device(ibfem_t* h) {
  check(cudaSetDevice(h->opt.device), "cudaSetDevice");
  h->stream = static_cast<cudaStream_t>(h->opt.stream);
  if (!h->stream) {
    // graphs cannot be captured on the legacy stream: use a private one
    check(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "stream");
    h->own_stream = true;
  }
  h->build_device();
  if (h->consistent && h->imex) h->prepare_consistent();
}

// undo a failed attach_device or build_clone: free what was allocated and the private stream
void detach_device(ibfem_t* h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  h->dfree_all();
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  h->stream = nullptr;
  h->own_stream = false;
}
}  // namespace

extern "C" {

const char* ibfem_last_error(void) { return g_last_error.c_str(); }

int ibfem_create(const ibfem_grid* grid, int p, const ibfem_geometry* geometry, double alpha,
                 const ibfem_stab* stab, const ibfem_options* opt, ibfem_t** out) {
  if (!grid || !out) return fail(IBFEM_ERR_ARG, "grid and out are required");
  *out = nullptr;
  std::unique_ptr<ibfem_t> h(new ibfem_t());
  IBFEM_TRY
  ibfem_options o{};
  o.physics = IBFEM_SCALAR;
  o.rho = 1.0;
  o.c = 1.0;
  o.E = 1.0;
  o.nu = 0.3;
  if (opt) o = *opt;
  h->opt = o;
  SetupInput& in = h->input;
  in.dim = grid->dim;
  for (int k = 0; k < 3; ++k) {
    in.n[k] = grid->n[k];
    in.lo[k] = grid->lo[k];
    in.hi[k] = grid->hi[k];
  }
  in.p = p;
  in.physics = o.physics;
  in.rho = o.rho;
  in.c = o.c;
  in.E = o.E;
  in.nu = o.nu;
  in.alpha = alpha;
  if (!(alpha >= 0.0)) throw std::invalid_argument("alpha must be >= 0");
  if (o.physics != IBFEM_SCALAR && o.physics != IBFEM_ELASTIC_PLANE_STRAIN)
    throw std::invalid_argument("unknown physics");
  if (o.scheme != IBFEM_CDM && o.scheme != IBFEM_IMEX && o.scheme != IBFEM_CDM_CONSISTENT)
    throw std::invalid_argument("unknown scheme");
  if (o.scheme != IBFEM_CDM && o.precision != IBFEM_FP64 && o.precision != IBFEM_EXACT64_TC &&
      o.precision != IBFEM_EXACT_TC)
    throw std::invalid_argument(
        "IMEX and the consistent-mass CDM take precision IBFEM_FP64, IBFEM_EXACT64_TC or IBFEM_EXACT_TC");
  in.need_consistent_mass = o.scheme != IBFEM_CDM;
  if (o.precision != IBFEM_FP64 && o.precision != IBFEM_EXACT_TC && o.precision != IBFEM_BF16X3_TC &&
      o.precision != IBFEM_BF16_TC && o.precision != IBFEM_EXACT64_TC)
    throw std::invalid_argument("unknown precision");
  if (!(o.rho > 0)) throw std::invalid_argument("rho must be > 0");
  if (stab) {
    in.stab = stab->kind;
    in.eps = stab->eps;
    in.f_lambda = stab->f_lambda;
    if (in.stab < 0 || in.stab > 2) throw std::invalid_argument("unknown stabilisation");
  }
  if (geometry) {
    GeometryDesc& g = in.geom;
    g.kind = geometry->kind;
    g.quad_depth = geometry->quad_depth;
    if (g.quad_depth < 0 || g.quad_depth > 12) throw std::invalid_argument("quad_depth out of range");
    if (g.kind == IBFEM_GEOM_HOLES) {
      if (geometry->count < 0 || (geometry->count > 0 && !geometry->shapes))
        throw std::invalid_argument("holes need shapes");
      g.shapes.assign(geometry->shapes, geometry->shapes + (size_t)geometry->count * (grid->dim + 1));
    } else if (g.kind == IBFEM_GEOM_VOXELS) {
      size_t nv = 1;
      for (int k = 0; k < grid->dim; ++k) {
        if (geometry->vn[k] < 1) throw std::invalid_argument("voxel counts must be >= 1");
        g.vn[k] = geometry->vn[k];
        nv *= (size_t)geometry->vn[k];
      }
      if (!geometry->voxels) throw std::invalid_argument("voxel image missing");
      g.voxels.assign(geometry->voxels, geometry->voxels + nv);
    } else if (g.kind == IBFEM_GEOM_ROTATED_BOX) {
      if (grid->dim != 3 || !geometry->shapes) throw std::invalid_argument("rotated box needs dim 3 and shapes");
      g.shapes.assign(geometry->shapes, geometry->shapes + 13);
    } else if (g.kind != IBFEM_GEOM_NONE) {
      throw std::invalid_argument("unknown geometry kind");
    }
  }
  if (!o.host_only) check_shape_supported(in.dim, in.p, in.physics, o.precision);
  h->setup = build_setup(in);
  if (o.scheme != IBFEM_CDM) {
    imex_partition(h->setup, h->imex_host);
    h->imex = h->imex_host.n_c > 0;   // without cut cells both are the CDM
    h->consistent = o.scheme == IBFEM_CDM_CONSISTENT;
    h->beta = h->consistent ? 0.0 : 0.25;
  }
  if (!o.host_only) {
    try {
      attach_device(h.get());
    } catch (...) {
      detach_device(h.get());
      throw;
    }
  }
  *out = h.release();
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_upload(ibfem_t* h) {
  if (!h) return fail(IBFEM_ERR_ARG, "null handle");
  if (!h->opt.host_only) return fail(IBFEM_ERR_STATE, "handle is already on the device");
  IBFEM_TRY
  check_shape_supported(h->input.dim, h->input.p, h->input.physics, h->opt.precision);
  h->opt.host_only = 0;
  try {
    attach_device(h);
  } catch (...) {
    detach_device(h);   // back to a host-only handle
    h->opt.host_only = 1;
    throw;
  }
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_clone(ibfem_t* src, ibfem_t** out) {
  if (!src || !out) return fail(IBFEM_ERR_ARG, "null argument");
  *out = nullptr;
  if (src->opt.host_only) return fail(IBFEM_ERR_STATE, "handle was created host_only");
  if (src->imex) return fail(IBFEM_ERR_ARG, "clones are for the lumped-mass CDM (this handle solves a c-set)");
  IBFEM_TRY
  check(cudaSetDevice(src->opt.device), "cudaSetDevice");
  std::unique_ptr<ibfem_t> h(new ibfem_t(src->setup_p));
  h->opt = src->opt;
  h->input = src->input;
  h->consistent = src->consistent;
  h->beta = src->beta;
  h->tc_variant = src->tc_variant;
  for (int k = 0; k < 3; ++k) h->tile[k] = src->tile[k];
  h->n_blocks = src->n_blocks;
  h->tc_img_host = src->tc_img_host;
  h->tc_frow_host = src->tc_frow_host;
  h->shared = src->shared;
  h->dt = src->dt;
  h->have_dt = src->have_dt;
  h->stream = static_cast<cudaStream_t>(h->opt.stream);
  if (!h->stream) {
    check(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "stream");
    h->own_stream = true;
  }
  try {
    h->build_clone(*src);
  } catch (...) {
    detach_device(h.get());
    throw;
  }
  *out = h.release();
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_destroy(ibfem_t* h) {
  if (!h) return IBFEM_OK;
  if (h->batch) batch_forget(h);   // drains the batch stream, then drops the member
  if (!h->opt.host_only) {
    cudaSetDevice(h->opt.device);
    cudaStreamSynchronize(h->stream);
    h->invalidate_graphs();
    h->dfree_all();
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->own_stream) cudaStreamDestroy(h->stream);
  }
  delete h;
  return IBFEM_OK;
}

int ibfem_info(const ibfem_t* h, ibfem_info_t* out) {
  if (!h || !out) return fail(IBFEM_ERR_ARG, "null argument");
  std::memset(out, 0, sizeof(*out));
  const Setup& s = h->setup;
  out->n_dof = s.n_dof;
  out->n_lattice_dof = s.n_lat_dof;
  out->n_elem = s.n_elem;
  out->n_uncut = s.n_uncut;
  out->n_cut = s.n_cut;
  out->n_outside = s.n_outside;
  out->n_loc = s.n_loc;
  out->ncomp = s.ncomp;
  out->precision = h->opt.precision;
  out->step = h->step;
  out->dt = h->dt;
  out->t = h->step * h->dt;
  out->lambda_ref = s.lambda_ref;
  if (h->imex) {
    out->n_c = h->imex_host.n_c;
    out->nnz_L = (int64_t)h->imex_host.chol.Lx.size();
    // heights of the dissection tree: the launches of one triangular solve
    out->n_levels = (int32_t)h->imex_host.gh_sn_ptr.size() - 1;
  }
  out->shared_device_bytes = h->shared ? h->shared->bytes : 0;
  out->device_bytes = h->opt.host_only ? h->planned_device_bytes() : h->device_bytes + out->shared_device_bytes;
  out->n_cut_matrices = s.n_cut_mat;
  out->tile_variant = h->tc_variant;
  out->tc_ctas_per_sm = h->tc_ctas;
  out->autotune_cached = h->tune_cached ? 1 : 0;
  for (int k = 0; k < 3; ++k) out->tile[k] = h->tc_tile[k];
  return IBFEM_OK;
}

static int require_device(ibfem_t* h) {
  if (!h) return fail(IBFEM_ERR_ARG, "null handle");
  if (h->opt.host_only) return fail(IBFEM_ERR_STATE, "handle was created host_only");
  if (h->batch) return fail(IBFEM_ERR_STATE, "handle is a member of a batch (poll it out first)");
  cudaError_t e = cudaSetDevice(h->opt.device);
  if (e != cudaSuccess) return fail(IBFEM_ERR_CUDA, cudaGetErrorString(e));
  return IBFEM_OK;
}

int ibfem_set_source(ibfem_t* h, int kind, const double* params, int nparams, double f_e) {
  int rc = require_device(h);
  if (rc) return rc;
  IBFEM_TRY
  const Setup& s = h->setup;
  std::vector<int64_t> dofs;
  std::vector<double> vals;
  if (kind == IBFEM_SRC_NONE) {
    // nothing
  } else if (kind == IBFEM_SRC_POINT) {
    if (!params || nparams < s.dim) throw std::invalid_argument("point source needs coordinates");
    double x[3] = {0, 0, 0};
    for (int k = 0; k < s.dim; ++k) x[k] = params[k];
    int64_t cell = locate_cell(s, x);
    if (cell < 0) throw std::domain_error("point source outside the kept cells");
    double dir[2] = {1.0, 0.0};
    if (s.ncomp == 2 && nparams >= s.dim + 2) {
      dir[0] = params[s.dim];
      dir[1] = params[s.dim + 1];
    }
    std::vector<double> N(s.nn_loc);
    shape_values(s, cell, x, N.data());
    double a = indicator(h->input, x) * h->input.rho;
    for (int l = 0; l < s.nn_loc; ++l)
      for (int c = 0; c < s.ncomp; ++c) {
        double v = a * N[l] * (s.ncomp == 2 ? dir[c] : 1.0);
        if (v == 0.0) continue;
        dofs.push_back(lattice_node(s, cell, l) * s.ncomp + c);
        vals.push_back(v);
      }
  } else if (kind == IBFEM_SRC_GAUSS) {
    if (!params || nparams < s.dim + 1 || !(params[s.dim] > 0))
      throw std::invalid_argument("Gaussian load needs (x_l[dim], sigma > 0)");
    double xl[3] = {0, 0, 0};
    for (int k = 0; k < s.dim; ++k) xl[k] = params[k];
    gauss_load(s, h->input, xl, params[s.dim], dofs, vals);
  } else if (kind == IBFEM_SRC_EDGE_TRACTION) {
    if (s.dim != 2 || !params || nparams < 3) throw std::invalid_argument("edge traction needs (y0, y1, t_x[, t_y]) in 2D");
    double t[2] = {params[2], nparams >= 4 ? params[3] : 0.0};
    edge_traction(s, h->input, params[0], params[1], t, dofs, vals);
  } else {
    throw std::invalid_argument("unknown source kind");
  }
  if (kind != IBFEM_SRC_NONE && !(f_e > 0)) throw std::invalid_argument("f_e must be > 0");
  // merge duplicates and bucket by owning tile
  std::vector<std::pair<int64_t, double>> ent;
  for (size_t i = 0; i < dofs.size(); ++i) ent.push_back({dofs[i], vals[i]});
  std::sort(ent.begin(), ent.end());
  std::vector<std::pair<int64_t, double>> merged;
  for (auto& e : ent) {
    if (!merged.empty() && merged.back().first == e.first) merged.back().second += e.second;
    else merged.push_back(e);
  }
  h->src_host = merged;
  h->src_fe = kind == IBFEM_SRC_NONE ? 0.0 : f_e;
  if (h->imex) {
    std::vector<double> fc(h->imex_host.n_c, 0.0);
    bool any = false;
    for (auto& e : merged) {
      int64_t ci = h->imex_host.c_of_dof[e.first];
      if (ci >= 0) {
        fc[h->imex_host.iperm[ci]] += e.second;
        any = true;
      }
    }
    h->imex_dev.Fc = any ? h->upload(fc) : nullptr;
  }
  int ntiles = h->n_blocks;
  std::vector<std::vector<std::pair<int64_t, double>>> per(ntiles);
  for (auto& e : merged) {
    int64_t node = e.first / s.ncomp;
    int64_t rem = node;
    int t = 0, stride = 1;
    for (int k = 0; k < s.dim; ++k) {
      int64_t g = rem % s.lat[k];
      rem /= s.lat[k];
      int b = (int)std::min<int64_t>(g / ((int64_t)h->tile[k] * s.p), h->dev.tiles[k] - 1);
      t += b * stride;
      stride *= h->dev.tiles[k];
    }
    per[t].push_back(e);
  }
  std::vector<int32_t> ptr(ntiles + 1, 0);
  std::vector<int64_t> sd;
  std::vector<double> sv;
  for (int t = 0; t < ntiles; ++t) {
    for (auto& e : per[t]) {
      sd.push_back(e.first);
      sv.push_back(e.second);
    }
    ptr[t + 1] = (int32_t)sd.size();
  }
  h->dev.src_ptr = h->upload(ptr);
  h->dev.src_dof = h->upload(sd);
  h->dev.src_val = h->upload(sv);
  if (h->opt.precision != IBFEM_FP64) h->upload_tc_sources();
  h->dev.f_e = kind == IBFEM_SRC_NONE ? 0.0 : f_e;
  h->invalidate_graphs();
  check(cudaStreamSynchronize(h->stream), "source upload");
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_set_observers(ibfem_t* h, int npts, const double* xyz, int64_t capacity) {
  int rc = require_device(h);
  if (rc) return rc;
  IBFEM_TRY
  const Setup& s = h->setup;
  if (npts < 0 || (npts > 0 && !xyz) || capacity < 0) throw std::invalid_argument("bad observers");
  std::vector<int64_t> od;
  std::vector<double> ow;
  std::vector<double> N(s.nn_loc);
  for (int o = 0; o < npts; ++o) {
    double x[3] = {0, 0, 0};
    for (int k = 0; k < s.dim; ++k) x[k] = xyz[o * s.dim + k];
    int64_t cell = locate_cell(s, x);
    if (cell < 0) throw std::domain_error("observer outside the kept cells");
    shape_values(s, cell, x, N.data());
    for (int c = 0; c < s.ncomp; ++c)
      for (int l = 0; l < s.nn_loc; ++l) {
        od.push_back(lattice_node(s, cell, l) * s.ncomp + c);
        ow.push_back(N[l]);
      }
  }
  h->dev.n_obs_rows = npts * s.ncomp;
  h->dev.obs_nodes = s.nn_loc;
  h->dev.obs_dof = h->upload(od);
  h->dev.obs_w = h->upload(ow);
  h->dev.ring_cap = capacity;
  h->dev.ring = static_cast<double*>(h->dalloc(std::max<int64_t>(capacity, 1) * std::max(h->dev.n_obs_rows, 1) * sizeof(double)));
  h->obs_out = static_cast<double*>(h->dalloc(std::max(h->dev.n_obs_rows, 1) * sizeof(double)));
  h->ring_start = h->step;
  h->invalidate_graphs();
  check(cudaStreamSynchronize(h->stream), "observer upload");
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_set_dt(ibfem_t* h, double dt) {
  int rc = require_device(h);
  if (rc) return rc;
  if (!(dt > 0) || !std::isfinite(dt)) return fail(IBFEM_ERR_ARG, "dt must be positive");
  IBFEM_TRY
  const Setup& s = h->setup;
  std::vector<double> minv(s.n_lat_dof, 0.0);
  for (int64_t i = 0; i < s.n_lat_dof; ++i)
    if (s.ML[i] > 0) minv[i] = dt * dt / s.ML[i];
  if (h->imex) {
    // c-DOFs carry -(c + 1): the fused kernel then forms the Newmark predictor there
    for (int64_t ci = 0; ci < h->imex_host.n_c; ++ci) minv[h->imex_host.c_dof[ci]] = -(double)(ci + 1);
    std::string err;
    const double beta = h->beta, gamma = 0.5;
    if (!h->consistent) {   // S = M^cc + beta dt^2 K^cc (the consistent-mass S was factored at setup)
      if (!imex_factor(s, beta * dt * dt, h->imex_host, err)) throw std::runtime_error("IMEX factorisation: " + err);
      h->imex_upload_factor();
    }
    h->imex_dev.beta_dt2 = beta * dt * dt;
    h->imex_dev.gamma_dt = gamma * dt;
    h->dev.imex_c1 = (0.5 - beta) * dt * dt;
    h->dev.imex_c2 = (1.0 - gamma) * dt;
  }
  check(cudaMemcpyAsync(h->d_minv, minv.data(), minv.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "minv");
  std::vector<float> m32;
  if (h->d_minv32) {
    // two FP32 slices: hi then lo (the pair carries dt^2/m to about 48 bits)
    m32.assign(2 * minv.size(), 0.f);
    for (size_t i = 0; i < minv.size(); ++i) {
      if (!(minv[i] > 0)) continue;
      float hh = (float)minv[i];
      m32[i] = hh;
      m32[minv.size() + i] = (float)(minv[i] - (double)hh);
    }
    check(cudaMemcpyAsync(h->d_minv32, m32.data(), m32.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream), "minv32");
  }
  check(cudaStreamSynchronize(h->stream), "set_dt");
  h->dt = dt;
  h->dev.dt = dt;
  h->have_dt = true;
  h->invalidate_graphs();
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_set_initial(ibfem_t* h, const double* u0, const double* v0) {
  int rc = require_device(h);
  if (rc) return rc;
  if (!h->have_dt) return fail(IBFEM_ERR_STATE, "set_dt before set_initial");
  IBFEM_TRY
  std::vector<double> lu, lv;
  h->to_lattice(u0, lu);
  h->to_lattice(v0, lv);
  h->cur = 0;
  check(cudaMemcpyAsync(h->U[0], lu.data(), lu.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "u0");
  check(cudaMemcpyAsync(h->U[1], lv.data(), lv.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "v0");
  check(cudaMemsetAsync(h->counters, 0, 4 * sizeof(unsigned long long), h->stream), "counters");
  OpInput x{h->U[0], nullptr, nullptr};
  check(launch_cut_apply_fp64(h->dev, x, false, h->stream), "cut_apply");
  check(launch_op_fp64(h->dev, x, h->U[1], kModeStartup, nullptr, h->stream), "startup");
  if (h->imex) {
    // Psi'_0 on c and Psi''_0 = (M^cc)^{-1} (F_0^c - K^c Psi_0) (Algorithm 2, initialisation)
    const Setup& s = h->setup;
    const ImexData& I = h->imex_host;
    const int nl = s.n_loc, nc = s.ncomp;
    std::vector<double> rhs(I.n_c, 0.0), vc(I.n_c, 0.0), ac;
    for (auto& e : h->src_host) {
      int64_t ci = I.c_of_dof[e.first];
      if (ci >= 0 && h->src_fe > 0) {
        const double pi = 3.141592653589793238462643383279502884;
        double ts = 2.0 * std::sqrt(6.0) / (pi * h->src_fe), q = pi * h->src_fe * (0.0 - ts);
        rhs[ci] += e.second * (1.0 - 2.0 * q * q) * std::exp(-q * q);
      }
    }
    std::vector<double> xe(nl);
    std::vector<int64_t> dofs(nl);
    for (int64_t e : I.ccells) {
      for (int l = 0; l < s.nn_loc; ++l)
        for (int c = 0; c < nc; ++c) {
          dofs[l * nc + c] = lattice_node(s, e, l) * nc + c;
          xe[l * nc + c] = lu[dofs[l * nc + c]];
        }
      const double* K = s.cls[e] == kCut ? &s.Kcut[(size_t)s.cut_mat[s.cut_index[e]] * nl * nl] : s.Kref.data();
      for (int a = 0; a < nl; ++a) {
        int64_t ci = I.c_of_dof[dofs[a]];
        if (ci < 0) continue;
        double acc = 0.0;
        for (int b = 0; b < nl; ++b) acc += K[(size_t)a * nl + b] * xe[b];
        rhs[ci] -= acc;
      }
    }
    for (int64_t ci = 0; ci < I.n_c; ++ci) vc[ci] = lv[I.c_dof[ci]];
    std::string err;
    if (!imex_mass_solve(I, rhs, ac, err)) throw std::runtime_error("IMEX mass solve: " + err);
    check(cudaMemcpyAsync(h->imex_dev.vc, vc.data(), vc.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "vc");
    check(cudaMemcpyAsync(h->imex_dev.ac, ac.data(), ac.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "ac");
  }
  check(cudaStreamSynchronize(h->stream), "set_initial");
  h->step = 0;
  h->ring_start = 0;
  h->have_init = true;
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_step(ibfem_t* h, int64_t n) {
  int rc = require_device(h);
  if (rc) return rc;
  if (n < 0) return fail(IBFEM_ERR_ARG, "n must be >= 0");
  if (!h->have_init) return fail(IBFEM_ERR_STATE, "set_initial (or set_state) before step");
  IBFEM_TRY
  h->run_steps(n);
  h->step += n;
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_step_timed(ibfem_t* h, int64_t n, void* flush_buf, size_t flush_bytes, double* ms,
                     int max_slots, int* n_slots) {
  int rc = require_device(h);
  if (rc) return rc;
  if (n < 0 || (max_slots > 0 && !ms) || (flush_bytes > 0 && !flush_buf))
    return fail(IBFEM_ERR_ARG, "bad arguments");
  if (!h->have_init) return fail(IBFEM_ERR_STATE, "set_initial (or set_state) before step");
  IBFEM_TRY
  for (double& v : h->slot_ms) v = 0.0;
  h->timing = true;
  for (int64_t i = 0; i < n; ++i) {
    if (flush_bytes > 0) check(launch_l2_evict(flush_buf, flush_bytes, h->stream), "flush");
    h->enqueue_step(h->cur);
    h->cur ^= 1;
    if (h->ev_used > 512) h->timed_collect();
  }
  h->timed_collect();
  h->timing = false;
  h->step += n;
  for (int i = 0; i < std::min(max_slots, h->n_slots); ++i) ms[i] = h->slot_ms[i];
  if (n_slots) *n_slots = h->n_slots;
  return IBFEM_OK;
  IBFEM_CATCH
}

const char* ibfem_kernel_name(const ibfem_t* h, int slot) {
  if (!h || slot < 0 || slot >= 8) return "";
  return h->slot_name[slot];
}

int ibfem_sync(ibfem_t* h) {
  int rc = require_device(h);
  if (rc) return rc;
  IBFEM_TRY
  check(cudaStreamSynchronize(h->stream), "sync");
  int flags = 0;
  check(cudaMemcpy(&flags, h->dev.flags, sizeof(int), cudaMemcpyDeviceToHost), "flags");
  if (flags & 2) return fail(IBFEM_ERR_TIMEOUT, "a bounded device wait gave up (results of that step are invalid)");
  if (flags & 1) return fail(IBFEM_ERR_DIVERGED, "non-finite value in the state");
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_sample(ibfem_t* h, int64_t max_rows, double* out, int64_t* rows) {
  int rc = require_device(h);
  if (rc) return rc;
  if (!out || !rows || max_rows < 0) return fail(IBFEM_ERR_ARG, "bad output");
  IBFEM_TRY
  const int nr = h->dev.n_obs_rows;
  check(cudaStreamSynchronize(h->stream), "sync");
  int64_t cap = h->dev.ring_cap;
  int64_t first = std::max<int64_t>(h->ring_start, h->step - cap);
  int64_t nrec = h->step - first;  // rows in the ring
  int64_t total = nrec + 1;        // plus the current state
  int64_t take = std::min(total, max_rows);
  std::vector<double> ring((size_t)std::max<int64_t>(cap, 1) * std::max(nr, 1));
  if (nr > 0 && cap > 0)
    check(cudaMemcpy(ring.data(), h->dev.ring, (size_t)cap * nr * sizeof(double), cudaMemcpyDeviceToHost), "ring");
  int64_t r = 0;
  for (int64_t k = first; k < h->step && r < take; ++k, ++r)
    std::memcpy(out + r * nr, ring.data() + (size_t)(k % cap) * nr, nr * sizeof(double));
  if (r < take && nr > 0) {
    check(launch_sample_now(h->dev, h->U[h->cur], h->obs_out, h->stream), "sample_now");
    check(cudaMemcpyAsync(out + r * nr, h->obs_out, nr * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "sample");
    check(cudaStreamSynchronize(h->stream), "sample sync");
    ++r;
  }
  *rows = r;
  int flags = 0;
  check(cudaMemcpy(&flags, h->dev.flags, sizeof(int), cudaMemcpyDeviceToHost), "flags");
  if (flags & 2) return fail(IBFEM_ERR_TIMEOUT, "a bounded device wait gave up (results of that step are invalid)");
  if (flags & 1) return fail(IBFEM_ERR_DIVERGED, "non-finite value in the state");
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_get_state(ibfem_t* h, double* u, double* u_prev) {
  int rc = require_device(h);
  if (rc) return rc;
  IBFEM_TRY
  const Setup& s = h->setup;
  std::vector<double> lat(s.n_lat_dof);
  check(cudaStreamSynchronize(h->stream), "sync");
  if (u) {
    check(cudaMemcpy(lat.data(), h->U[h->cur], lat.size() * sizeof(double), cudaMemcpyDeviceToHost), "u");
    h->from_lattice(lat, u);
  }
  if (u_prev) {
    check(cudaMemcpy(lat.data(), h->U[1 - h->cur], lat.size() * sizeof(double), cudaMemcpyDeviceToHost), "u_prev");
    h->from_lattice(lat, u_prev);
  }
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_check_bounded_wait(ibfem_t* h, int polls) {
  int rc = require_device(h);
  if (rc) return rc;
  if (polls < 1 || polls > (1 << 24)) return fail(IBFEM_ERR_ARG, "polls must be in [1, 2^24]");
  IBFEM_TRY
  check(launch_bounded_wait_probe(h->dev.flags, polls, h->stream), "bounded_wait_probe");
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_check_solve_schedule(ibfem_t* h, double beta_dt2, uint64_t seed, int64_t* violations,
                               double* rel_err) {
  if (!h) return fail(IBFEM_ERR_ARG, "null handle");
  if (!violations || !rel_err || !(beta_dt2 >= 0.0)) return fail(IBFEM_ERR_ARG, "bad arguments");
  if (!h->imex) return fail(IBFEM_ERR_STATE, "the handle solves no c-set (scheme IBFEM_CDM or no cut cells)");
  IBFEM_TRY
  std::string err;
  if (!imex_check_schedule(h->setup, h->imex_host, beta_dt2, seed, *violations, *rel_err, err))
    return fail(IBFEM_ERR_ARG, "S = M^cc + beta_dt2 K^cc is not positive definite: " + err);
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_set_state(ibfem_t* h, const double* u, const double* u_prev, int64_t step) {
  int rc = require_device(h);
  if (rc) return rc;
  if (!u || !u_prev || step < 0) return fail(IBFEM_ERR_ARG, "u, u_prev and step >= 0 required");
  if (!h->have_dt) return fail(IBFEM_ERR_STATE, "set_dt before set_state");
  IBFEM_TRY
  std::vector<double> a, b;
  h->to_lattice(u, a);
  h->to_lattice(u_prev, b);
  h->cur = 0;
  check(cudaMemcpyAsync(h->U[0], a.data(), a.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "u");
  check(cudaMemcpyAsync(h->U[1], b.data(), b.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "u_prev");
  unsigned long long cnt[4] = {(unsigned long long)step, 0, 0, 0};
  check(cudaMemcpyAsync(h->counters, cnt, sizeof(cnt), cudaMemcpyHostToDevice, h->stream), "counters");
  check(cudaStreamSynchronize(h->stream), "set_state");
  h->step = step;
  h->ring_start = step;
  h->have_init = true;
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_apply_operator(ibfem_t* h, const double* x, double* y) {
  int rc = require_device(h);
  if (rc) return rc;
  if (!x || !y) return fail(IBFEM_ERR_ARG, "null vector");
  IBFEM_TRY
  std::vector<double> lx;
  h->to_lattice(x, lx);
  check(cudaMemcpyAsync(h->W, lx.data(), lx.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "x");
  OpInput in{h->W, nullptr, nullptr};
  if (h->opt.precision == IBFEM_EXACT64_TC) {
    check(launch_cut_apply_fp64(h->dev, in, false, h->stream), "cut_apply");
    check(launch_op_tc64(h->dev, h->W, h->scratch, kModeApply, h->stream), "apply_tc64");
  } else if (h->opt.precision != IBFEM_FP64) {
    check(launch_op_tc(h->dev, h->W, h->scratch, kModeApply, h->tc_scheme(), h->tc_variant, h->stream, h->tc_ctas),
          "apply_tc");
  } else {
    check(launch_cut_apply_fp64(h->dev, in, false, h->stream), "cut_apply");
    check(launch_op_fp64(h->dev, in, h->scratch, kModeApply, nullptr, h->stream), "apply");
  }
  check(cudaMemcpyAsync(lx.data(), h->scratch, lx.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "y");
  check(cudaStreamSynchronize(h->stream), "apply sync");
  h->from_lattice(lx, y);
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_set_tile_variant(ibfem_t* h, int variant) {
  int rc = require_device(h);
  if (rc) return rc;
  if (variant != 0 && variant != 1) return fail(IBFEM_ERR_ARG, "tile variant must be 0 or 1");
  if (h->opt.precision == IBFEM_EXACT64_TC)
    return variant == h->tc_variant ? IBFEM_OK : fail(IBFEM_ERR_ARG, "the FP64-grade tensor-core path has one tile shape");
  if (variant == 1 && h->tc_scheme() != 0)
    return fail(IBFEM_ERR_ARG, "the small tile exists for the exact tensor-core path (IBFEM_EXACT_TC)");
  if (h->opt.precision == IBFEM_FP64) return variant == 0 ? IBFEM_OK : fail(IBFEM_ERR_ARG, "FP64 path has one tile shape");
  IBFEM_TRY
  h->set_tc_variant(variant);
  return IBFEM_OK;
  IBFEM_CATCH
}

}  // extern "C"

namespace {
// Choices of the exact kernel's autotuner, per (device, dim, p, ncomp, log2 of the cell
// count): later handles of the same class of problem reuse them without timing.
struct TuneChoice {
  int variant, ctas;
  double ms[2];
};
std::mutex g_tune_mutex;
std::map<std::array<int, 5>, TuneChoice> g_tune_cache;
}  // namespace

extern "C" {

int ibfem_autotune(ibfem_t* h, int reps, int* variant, double* ms) {
  int rc = require_device(h);
  if (rc) return rc;
  if (reps < 1) return fail(IBFEM_ERR_ARG, "reps must be >= 1");
  IBFEM_TRY
  double t[2] = {0.0, 0.0};
  int best = 0;
  h->tune_cached = false;
  if (h->opt.precision != IBFEM_FP64 && h->tc_scheme() == 0) {
    const Setup& s = h->setup;
    int lg = 0;
    for (int64_t c = s.n_elem; c > 1; c >>= 1) ++lg;
    const std::array<int, 5> key = {h->opt.device, s.dim, s.p, s.ncomp, lg};
    bool hit = false;
    TuneChoice ch{};
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        ch = it->second;
        hit = true;
      }
    }
    if (!hit) {
      // time reps operator applications (the step's kernel in apply mode, on work vectors:
      // the state is untouched) for each tile shape and each cap on the resident CTAs per
      // SM (as many as fit, one), after two untimed ones
      cudaEvent_t e0, e1;
      check(cudaEventCreate(&e0), "event");
      check(cudaEventCreate(&e1), "event");
      double best_ms = 1e300;
      ch.ms[0] = ch.ms[1] = 1e300;
      for (int v = 0; v < 2; ++v) {
        h->set_tc_variant(v);
        for (int c : {0, 1}) {
          for (int i = 0; i < 2; ++i)
            check(launch_op_tc(h->dev, h->W, h->scratch, kModeApply, 0, v, h->stream, c), "autotune");
          check(cudaEventRecord(e0, h->stream), "event");
          for (int i = 0; i < reps; ++i)
            check(launch_op_tc(h->dev, h->W, h->scratch, kModeApply, 0, v, h->stream, c), "autotune");
          check(cudaEventRecord(e1, h->stream), "event");
          check(cudaEventSynchronize(e1), "event");
          float f = 0.f;
          check(cudaEventElapsedTime(&f, e0, e1), "event");
          const double m = (double)f / reps;
          ch.ms[v] = std::min(ch.ms[v], m);
          if (m < best_ms) {
            best_ms = m;
            ch.variant = v;
            ch.ctas = c;
          }
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune_cache[key] = ch;
    }
    h->set_tc_variant(ch.variant);
    if (h->tc_ctas != ch.ctas) {
      h->tc_ctas = ch.ctas;
      h->invalidate_graphs();
    }
    h->tune_cached = hit;
    best = ch.variant;
    t[0] = ch.ms[0];
    t[1] = ch.ms[1];
  } else if (h->opt.precision == IBFEM_EXACT64_TC) {
    best = h->tc_variant;   // one tile shape
  }
  if (variant) *variant = best;
  if (ms) {
    ms[0] = t[0];
    ms[1] = t[1];
  }
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_crit_dt(ibfem_t* h, int max_iter, double rtol, double* dt_crit, double* lambda_max,
                  int* iterations) {
  int rc = require_device(h);
  if (rc) return rc;
  if (max_iter < 1) return fail(IBFEM_ERR_ARG, "max_iter must be >= 1");
  IBFEM_TRY
  const Setup& s = h->setup;
  // start vector v_i = 1 + 0.5 sin(i) over kept DOFs, normalised
  std::vector<double> v(s.n_dof);
  double nrm = 0;
  const bool gen = h->consistent && h->imex;   // M = diag(M_L^dd) + consistent M^cc
  for (int64_t i = 0; i < s.n_dof; ++i) {
    v[i] = 1.0 + 0.5 * std::sin((double)i);
    if (h->imex && !gen) {
      int64_t lat = s.lat_of_kept[i / s.ncomp] * s.ncomp + i % s.ncomp;
      if (h->imex_host.c_of_dof[lat] >= 0) v[i] = 0.0;   // explicit (d) block only
    }
    nrm += v[i] * v[i];
  }
  nrm = std::sqrt(nrm);
  for (auto& x : v) x /= nrm;
  std::vector<double> lv;
  h->to_lattice(v.data(), lv);
  double* bufs[2] = {h->W, h->scratch};
  check(cudaMemcpyAsync(bufs[0], lv.data(), lv.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "start");
  double one = 1.0;
  double* inv_norm = h->scalars;
  check(cudaMemcpyAsync(inv_norm, &one, sizeof(double), cudaMemcpyHostToDevice, h->stream), "scal");
  std::vector<double> hist;
  double lam = 0, lam_old = 0;
  int it = 0, b = 0;
  bool have_old = false, converged = false;
  while (it < max_iter && !converged) {
    int chunk = std::min(kPowerChunk, max_iter - it);
    for (int c = 0; c < chunk; ++c) {
      if (gen) {
        // power iteration on G^{-1} K G^{-T}, G = diag(sqrt(M_L^dd)) + (c block) P^T L with
        // M^cc = P^T L L^T P: y = G^{-T} x, z = K y, w = G^{-1} z, lambda ~ x . w
        if (!h->pw[0]) {
          h->pw[0] = static_cast<double*>(h->dalloc(s.n_lat_dof * sizeof(double)));
          h->pw[1] = static_cast<double*>(h->dalloc(s.n_lat_dof * sizeof(double)));
        }
        double *y = h->pw[0], *z = h->pw[1];
        check(launch_scale_vec(s.n_lat_dof, h->dev.sinv, bufs[b], inv_norm, y, h->stream), "scale");
        check(launch_imex_tri(h->imex_dev, bufs[b], inv_norm, y, true, h->stream), "backward solve");
        OpInput yi{y, nullptr, nullptr};
        check(launch_cut_apply_fp64(h->dev, yi, false, h->stream), "cut_apply");
        check(launch_op_fp64(h->dev, yi, z, kModeApply, nullptr, h->stream), "apply");
        check(launch_scale_vec(s.n_lat_dof, h->dev.sinv, z, nullptr, bufs[1 - b], h->stream), "scale");
        check(launch_imex_tri(h->imex_dev, z, nullptr, bufs[1 - b], false, h->stream), "forward solve");
        check(launch_dot2(s.n_lat_dof, bufs[b], inv_norm, bufs[1 - b], h->partials, h->n_blocks, h->stream), "dot");
      } else {
        OpInput x{bufs[b], h->dev.sinv, inv_norm};
        check(launch_cut_apply_fp64(h->dev, x, false, h->stream), "cut_apply");
        check(launch_op_fp64(h->dev, x, bufs[1 - b], kModePower, h->partials, h->stream), "power");
      }
      check(launch_reduce_power(h->partials, h->n_blocks, h->lam_hist, inv_norm, c, h->stream), "reduce");
      b ^= 1;
    }
    hist.resize(chunk);
    check(cudaMemcpyAsync(hist.data(), h->lam_hist, chunk * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "hist");
    check(cudaStreamSynchronize(h->stream), "power sync");
    for (int c = 0; c < chunk; ++c) {
      ++it;
      lam = hist[c];
      if (have_old && std::fabs(lam - lam_old) <= rtol * std::fabs(lam)) {
        converged = true;
        break;
      }
      lam_old = lam;
      have_old = true;
    }
  }
  if (!(lam > 0) || !std::isfinite(lam)) throw std::runtime_error("power iteration produced a non-positive eigenvalue");
  if (lambda_max) *lambda_max = lam;
  if (dt_crit) *dt_crit = 2.0 / std::sqrt(lam);
  if (iterations) *iterations = it;
  return IBFEM_OK;
  IBFEM_CATCH
}

int ibfem_get_lumped_mass(ibfem_t* h, double* ml) {
  if (!h || !ml) return fail(IBFEM_ERR_ARG, "null argument");
  h->from_lattice(h->setup.ML, ml);
  return IBFEM_OK;
}

int ibfem_get_cut_cells(ibfem_t* h, int64_t* cells) {
  if (!h || !cells) return fail(IBFEM_ERR_ARG, "null argument");
  std::copy(h->setup.cut_cells.begin(), h->setup.cut_cells.end(), cells);
  return IBFEM_OK;
}

int ibfem_get_element(ibfem_t* h, int64_t cell, double* K, double* ml) {
  if (!h) return fail(IBFEM_ERR_ARG, "null handle");
  const Setup& s = h->setup;
  if (cell < 0 || cell >= s.n_elem || s.cls[cell] == kOutside) return fail(IBFEM_ERR_ARG, "cell is outside or out of range");
  const int nl = s.n_loc;
  if (s.cls[cell] == kCut) {
    int ci = s.cut_mat[s.cut_index[cell]];
    if (K) std::copy(&s.Kcut[(size_t)ci * nl * nl], &s.Kcut[(size_t)(ci + 1) * nl * nl], K);
    if (ml) std::copy(&s.mlcut[(size_t)ci * nl], &s.mlcut[(size_t)(ci + 1) * nl], ml);
  } else {
    if (K) std::copy(s.Kref.begin(), s.Kref.end(), K);
    if (ml) std::copy(s.mref.begin(), s.mref.end(), ml);
  }
  return IBFEM_OK;
}

int ibfem_get_element_mass(ibfem_t* h, int64_t cell, double* M) {
  if (!h || !M) return fail(IBFEM_ERR_ARG, "null argument");
  const Setup& s = h->setup;
  if (cell < 0 || cell >= s.n_elem || s.cls[cell] == kOutside) return fail(IBFEM_ERR_ARG, "cell is outside or out of range");
  const int nl = s.n_loc;
  if (s.cls[cell] == kCut) {
    if (s.Mcut.empty()) return fail(IBFEM_ERR_STATE, "consistent cut masses are kept by the IMEX and consistent-mass schemes only");
    const size_t ci = (size_t)s.cut_mat[s.cut_index[cell]];
    std::copy(&s.Mcut[ci * nl * nl], &s.Mcut[(ci + 1) * nl * nl], M);
  } else {
    std::fill(M, M + (size_t)nl * nl, 0.0);
    for (int i = 0; i < nl; ++i) M[(size_t)i * nl + i] = s.mref[i];
  }
  return IBFEM_OK;
}

}  // extern "C"
