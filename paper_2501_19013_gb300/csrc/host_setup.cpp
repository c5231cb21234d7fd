// Host construction of the spectral cell discretisation (library side).
//
// Sec. 2.2 (spatial discretisation, finite cell indicator, space-tree quadrature of cut
// cells), Sec. 2.4 (nodal lumping of uncut cells, HRZ lumping of cut cells), Sec. 2.5
// (eigenvalue stabilisation, Eq. epsilon_stabilization) of Buerchner et al.,
// arXiv 2501.19013.  Plane-strain elasticity and mass scaling are not defined in the
// paper; their textbook forms are used (isotropic Lame operator; cut-cell mass scaled by
// max(1, lambda_e / lambda_ref)).
//
// 1D rules come from the Golub-Welsch eigenvalue method: Gauss-Legendre nodes are the
// eigenvalues of the Legendre Jacobi matrix, the interior Gauss-Lobatto-Legendre nodes
// those of the Jacobi matrix of P^{(1,1)} (roots of P_p').
#include "host_setup.h"

#include <algorithm>
#include <limits>
#include <array>
#include <climits>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <stdexcept>
#include <thread>
#include <unordered_map>

namespace ibfem {

namespace {

// ------------------------------------------------------------------ 1D rules
// Symmetric tridiagonal Golub-Welsch: diag zero, off-diagonal b[k]; returns nodes and
// the squared first eigenvector components (times mu0 gives the weights).
void golub_welsch(int m, const std::vector<double>& off, std::vector<double>& x,
                  std::vector<double>& v0sq) {
  std::vector<double> A(m * m, 0.0), V(m * m), ev(m);
  for (int k = 0; k + 1 < m; ++k) {
    A[k * m + k + 1] = off[k];
    A[(k + 1) * m + k] = off[k];
  }
  if (!sym_eig(m, A.data(), ev.data(), V.data()))
    throw std::runtime_error("Golub-Welsch eigenproblem did not converge");
  x = ev;
  v0sq.resize(m);
  for (int j = 0; j < m; ++j) v0sq[j] = V[0 * m + j] * V[0 * m + j];
}

void gauss_rule(int m, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> off(std::max(m - 1, 0));
  for (int k = 1; k < m; ++k) off[k - 1] = k / std::sqrt(4.0 * k * k - 1.0);
  std::vector<double> v0;
  golub_welsch(m, off, x, v0);
  w.resize(m);
  for (int j = 0; j < m; ++j) w[j] = 2.0 * v0[j];
}

double legendre(int n, double x) {
  double a = 1.0, b = x;
  if (n == 0) return 1.0;
  for (int k = 1; k < n; ++k) {
    double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
    a = b;
    b = c;
  }
  return b;
}

void gll_rule(int p, std::vector<double>& x, std::vector<double>& w) {
  x.assign(p + 1, 0.0);
  x[0] = -1.0;
  x[p] = 1.0;
  if (p >= 2) {
    int m = p - 1;  // interior nodes: zeros of the Jacobi polynomial P^{(1,1)}_{p-1}
    std::vector<double> off(std::max(m - 1, 0));
    for (int k = 1; k < m; ++k) off[k - 1] = std::sqrt(k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
    std::vector<double> xi, v0;
    golub_welsch(m, off, xi, v0);
    for (int j = 0; j < m; ++j) x[j + 1] = xi[j];
  }
  w.resize(p + 1);
  for (int j = 0; j <= p; ++j) {
    double P = legendre(p, x[j]);
    w[j] = 2.0 / (p * (p + 1.0) * P * P);
  }
}

// 1D Lagrange values and derivatives at t for the nodes xs (product form).
void lagrange1d(const std::vector<double>& xs, double t, double* L, double* dL) {
  int m = (int)xs.size();
  for (int a = 0; a < m; ++a) {
    double val = 1.0, der = 0.0;
    for (int b = 0; b < m; ++b) {
      if (b == a) continue;
      double inv = 1.0 / (xs[a] - xs[b]);
      // d/dt of the running product (t - x_b) / (x_a - x_b)
      der = der * (t - xs[b]) * inv + val * inv;
      val *= (t - xs[b]) * inv;
    }
    L[a] = val;
    if (dL) dL[a] = der;
  }
}

// ------------------------------------------------------------------ geometry
struct Geo {
  const SetupInput* in;
  int d;
  // rotated box
  double half = 0, c[3] = {0, 0, 0}, T[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};

  explicit Geo(const SetupInput& inp) : in(&inp), d(inp.dim) {
    if (inp.geom.kind == 3) {
      const auto& s = inp.geom.shapes;
      half = 0.5 * s[0];
      for (int k = 0; k < 3; ++k) c[k] = s[1 + k];
      for (int k = 0; k < 9; ++k) T[k] = s[4 + k];
    }
  }

  bool physical_point(const double* x) const {
    const auto& g = in->geom;
    if (g.kind == 1) {
      int stride = d + 1;
      int cnt = (int)(g.shapes.size() / stride);
      for (int i = 0; i < cnt; ++i) {
        const double* s = &g.shapes[i * stride];
        double r2 = 0;
        for (int k = 0; k < d; ++k) r2 += (x[k] - s[k]) * (x[k] - s[k]);
        if (r2 < s[d] * s[d]) return false;
      }
      return true;
    }
    if (g.kind == 2) {
      int64_t idx = 0, stride = 1;
      for (int k = 0; k < d; ++k) {
        double rel = (x[k] - in->lo[k]) / (in->hi[k] - in->lo[k]) * g.vn[k];
        int64_t i = (int64_t)std::floor(rel);
        i = std::min<int64_t>(std::max<int64_t>(i, 0), g.vn[k] - 1);
        idx += i * stride;
        stride *= g.vn[k];
      }
      return g.voxels[idx] == 0;
    }
    if (g.kind == 3) {
      for (int a = 0; a < 3; ++a) {
        double loc = 0;
        for (int k = 0; k < 3; ++k) loc += (x[k] - c[k]) * T[k * 3 + a];
        if (std::fabs(loc) > half) return false;
      }
      return true;
    }
    return true;
  }

  // Box classification.  Voxel boxes are given by integer coordinates in units of
  // 1/(n_k 2^level) of the extended domain so that voxel ranges are exact.
  CellClass classify(const double* blo, const double* bhi, const int64_t* ilo,
                     int64_t denom_scale) const {
    const auto& g = in->geom;
    if (g.kind == 0) return kUncut;
    if (g.kind == 1) {
      int stride = d + 1;
      int cnt = (int)(g.shapes.size() / stride);
      bool cut = false;
      for (int i = 0; i < cnt; ++i) {
        const double* s = &g.shapes[i * stride];
        double dmin2 = 0, dmax2 = 0;
        for (int k = 0; k < d; ++k) {
          double gap = std::max(std::max(blo[k] - s[k], 0.0), s[k] - bhi[k]);
          dmin2 += gap * gap;
          double far = std::max(std::fabs(s[k] - blo[k]), std::fabs(s[k] - bhi[k]));
          dmax2 += far * far;
        }
        double r2 = s[d] * s[d];
        if (dmax2 <= r2) return kOutside;
        if (dmin2 < r2) cut = true;
      }
      return cut ? kCut : kUncut;
    }
    if (g.kind == 2) {
      // voxel index range [v0, v1) per axis from exact integer arithmetic:
      // box spans [ilo, ilo+1] in units of h/denom_scale of the cell grid.
      int64_t v0[3] = {0, 0, 0}, v1[3] = {1, 1, 1};
      for (int k = 0; k < d; ++k) {
        int64_t den = (int64_t)in->n[k] * denom_scale;
        int64_t a = ilo[k] * g.vn[k];
        int64_t b = (ilo[k] + 1) * g.vn[k];
        v0[k] = a / den;
        v1[k] = (b + den - 1) / den;
        v0[k] = std::min<int64_t>(std::max<int64_t>(v0[k], 0), g.vn[k] - 1);
        v1[k] = std::min<int64_t>(std::max<int64_t>(v1[k], v0[k] + 1), g.vn[k]);
      }
      bool any_void = false, any_solid = false;
      for (int64_t z = v0[2]; z < (d == 3 ? v1[2] : 1); ++z)
        for (int64_t y = v0[1]; y < v1[1]; ++y)
          for (int64_t x = v0[0]; x < v1[0]; ++x) {
            int64_t idx = x + (int64_t)g.vn[0] * (y + (int64_t)g.vn[1] * z);
            if (g.voxels[idx]) any_void = true; else any_solid = true;
            if (any_void && any_solid) return kCut;
          }
      return any_solid ? kUncut : kOutside;
    }
    // rotated box: separating axes between the aligned box and the cube
    double cb[3], hb[3];
    for (int k = 0; k < 3; ++k) {
      cb[k] = 0.5 * (blo[k] + bhi[k]);
      hb[k] = 0.5 * (bhi[k] - blo[k]);
    }
    double axes[15][3];
    int na = 0;
    for (int k = 0; k < 3; ++k) {
      for (int j = 0; j < 3; ++j) axes[na][j] = (j == k) ? 1.0 : 0.0;
      ++na;
    }
    for (int k = 0; k < 3; ++k) {
      for (int j = 0; j < 3; ++j) axes[na][j] = T[j * 3 + k];
      ++na;
    }
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) {
        double e[3] = {0, 0, 0};
        e[i] = 1.0;
        double t[3] = {T[0 * 3 + k], T[1 * 3 + k], T[2 * 3 + k]};
        double cr[3] = {e[1] * t[2] - e[2] * t[1], e[2] * t[0] - e[0] * t[2], e[0] * t[1] - e[1] * t[0]};
        double nrm = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        if (nrm > 1e-12) {
          for (int j = 0; j < 3; ++j) axes[na][j] = cr[j] / nrm;
          ++na;
        }
      }
    for (int a = 0; a < na; ++a) {
      const double* L = axes[a];
      double rb = 0, rc = 0, proj = 0;
      for (int k = 0; k < 3; ++k) {
        rb += hb[k] * std::fabs(L[k]);
        proj += (c[k] - cb[k]) * L[k];
      }
      for (int j = 0; j < 3; ++j) {
        double tl = T[0 * 3 + j] * L[0] + T[1 * 3 + j] * L[1] + T[2 * 3 + j] * L[2];
        rc += half * std::fabs(tl);
      }
      if (std::fabs(proj) >= rb + rc) return kOutside;
    }
    for (int corner = 0; corner < 8; ++corner) {
      double x[3];
      for (int k = 0; k < 3; ++k) x[k] = (corner >> k) & 1 ? bhi[k] : blo[k];
      if (!physical_point(x)) return kCut;
    }
    return kUncut;
  }
};

// ------------------------------------------------------------------ element integration
struct ElementIntegrator {
  const Setup* s;
  const SetupInput* in;
  std::vector<double> gx, gw;  // GL rule with p + 1 points

  ElementIntegrator(const Setup& st, const SetupInput& inp) : s(&st), in(&inp) {
    gauss_rule(st.p + 1, gx, gw);
  }

  // Accumulate K and M (n_loc x n_loc, full) over a tensor GL rule on the sub-box
  // [blo, bhi] of the cell [clo, clo + h]; alpha: constant (>= 0) or pointwise (< 0).
  void accumulate(const Geo& geo, const double* clo, const double* blo, const double* bhi,
                  double alpha_const, double* K, double* M) const {
    const int d = s->dim, m = s->nn1, nq1 = (int)gx.size();
    const int nnl = s->nn_loc, nc = s->ncomp, nl = s->n_loc;
    int nq = 1;
    for (int k = 0; k < d; ++k) nq *= nq1;
    std::vector<double> Lv(d * m), Ld(d * m), N(nnl), G(d * nnl);
    double lam = 0, mu = 0;
    if (s->ncomp == 2) {
      lam = in->E * in->nu / ((1 + in->nu) * (1 - 2 * in->nu));
      mu = in->E / (2 * (1 + in->nu));
    }
    for (int q = 0; q < nq; ++q) {
      double x[3] = {0, 0, 0}, w = 1.0;
      int qq = q;
      for (int k = 0; k < d; ++k) {
        int i = qq % nq1;
        qq /= nq1;
        double half = 0.5 * (bhi[k] - blo[k]);
        x[k] = blo[k] + (gx[i] + 1.0) * half;
        w *= gw[i] * half;
        double t = 2.0 * (x[k] - clo[k]) / s->h[k] - 1.0;
        lagrange1d(s->gll_x, t, &Lv[k * m], &Ld[k * m]);
        for (int a = 0; a < m; ++a) Ld[k * m + a] *= 2.0 / s->h[k];
      }
      double a = alpha_const >= 0 ? alpha_const : (geo.physical_point(x) ? 1.0 : in->alpha);
      double wa = w * a;
      if (wa == 0.0) continue;
      for (int j = 0; j < nnl; ++j) {
        int jj = j;
        double nv = 1.0, g[3] = {1.0, 1.0, 1.0};
        for (int k = 0; k < d; ++k) {
          int ak = jj % m;
          jj /= m;
          nv *= Lv[k * m + ak];
          for (int l = 0; l < d; ++l) g[l] *= (l == k ? Ld[k * m + ak] : Lv[k * m + ak]);
        }
        N[j] = nv;
        for (int l = 0; l < d; ++l) G[l * nnl + j] = g[l];
      }
      if (nc == 1) {
        double kc = in->rho * in->c * in->c * wa, mc = in->rho * wa;
        for (int i = 0; i < nnl; ++i)
          for (int j = i; j < nnl; ++j) {
            double gg = 0;
            for (int l = 0; l < d; ++l) gg += G[l * nnl + i] * G[l * nnl + j];
            K[i * nl + j] += kc * gg;
            M[i * nl + j] += mc * N[i] * N[j];
          }
      } else {
        // plane strain: K_(ia)(jb) = lam d_a N_i d_b N_j + mu d_b N_i d_a N_j
        //                            + mu delta_ab grad N_i . grad N_j
        double mc = in->rho * wa;
        for (int i = 0; i < nnl; ++i)
          for (int j = 0; j < nnl; ++j) {
            double gg = G[0 * nnl + i] * G[0 * nnl + j] + G[1 * nnl + i] * G[1 * nnl + j];
            for (int aa = 0; aa < 2; ++aa)
              for (int bb = 0; bb < 2; ++bb) {
                int r = 2 * i + aa, c = 2 * j + bb;
                if (c < r) continue;
                double v = lam * G[aa * nnl + i] * G[bb * nnl + j] +
                           mu * G[bb * nnl + i] * G[aa * nnl + j] + (aa == bb ? mu * gg : 0.0);
                K[r * nl + c] += wa * v;
                if (aa == bb) M[r * nl + c] += mc * N[i] * N[j];
              }
          }
      }
    }
  }

  static void symmetrize(int nl, double* A) {
    for (int i = 0; i < nl; ++i)
      for (int j = 0; j < i; ++j) A[i * nl + j] = A[j * nl + i];
  }

  // Space tree over cell `cell` with lower corner clo.
  void cut_cell(const Geo& geo, int64_t cell, const double* clo, double* K, double* M) const {
    const int d = s->dim;
    const int nl = s->n_loc;
    std::fill(K, K + nl * nl, 0.0);
    std::fill(M, M + nl * nl, 0.0);
    int64_t cidx[3] = {0, 0, 0};
    int64_t rem = cell;
    for (int k = 0; k < d; ++k) {
      cidx[k] = rem % s->n[k];
      rem /= s->n[k];
    }
    struct Node { int level; int64_t sub[3]; };
    std::vector<Node> stack;
    stack.push_back({0, {0, 0, 0}});
    const int depth = in->geom.quad_depth;
    while (!stack.empty()) {
      Node nd = stack.back();
      stack.pop_back();
      int64_t scale = (int64_t)1 << nd.level;
      double blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
      int64_t ilo[3] = {0, 0, 0};
      for (int k = 0; k < d; ++k) {
        double hs = s->h[k] / (double)scale;
        blo[k] = clo[k] + nd.sub[k] * hs;
        bhi[k] = blo[k] + hs;
        ilo[k] = cidx[k] * scale + nd.sub[k];
      }
      CellClass c = geo.classify(blo, bhi, ilo, scale);
      if (c == kUncut) {
        accumulate(geo, clo, blo, bhi, 1.0, K, M);
      } else if (c == kOutside) {
        accumulate(geo, clo, blo, bhi, in->alpha, K, M);
      } else if (nd.level >= depth) {
        accumulate(geo, clo, blo, bhi, -1.0, K, M);
      } else {
        // children pushed in reverse so that they are integrated in x-fastest order
        int nch = 1 << d;
        for (int ch = nch - 1; ch >= 0; --ch) {
          Node c2{nd.level + 1, {0, 0, 0}};
          for (int k = 0; k < d; ++k) c2.sub[k] = nd.sub[k] * 2 + ((ch >> k) & 1);
          stack.push_back(c2);
        }
      }
    }
    symmetrize(nl, K);
    symmetrize(nl, M);
  }
};

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& body) {
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  int nt = (int)std::min<int64_t>(hw, std::max<int64_t>(1, n / 16));
  if (nt <= 1) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  std::atomic<int64_t> next{0};
  const int64_t chunk = 16;
  std::exception_ptr err;
  std::atomic<bool> failed{false};
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (;;) {
        int64_t a = next.fetch_add(chunk);
        if (a >= n || failed.load()) break;
        try {
          body(a, std::min(n, a + chunk));
        } catch (...) {
          if (!failed.exchange(true)) err = std::current_exception();
          break;
        }
      }
    });
  for (auto& t : th) t.join();
  if (err) std::rethrow_exception(err);
}

}  // namespace

// ------------------------------------------------------------------ symmetric eigen
bool sym_eig(int n, double* A, double* evals, double* evecs) {
  // Householder reduction to tridiagonal form T = Q^T A Q, then implicit-shift QL.
  std::vector<double> Q(n * n, 0.0), diag(n), off(n, 0.0), v(n), pv(n);
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  for (int k = 0; k + 2 < n; ++k) {
    double nrm = 0;
    for (int i = k + 1; i < n; ++i) nrm += A[i * n + k] * A[i * n + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    double x0 = A[(k + 1) * n + k];
    double alpha = x0 > 0 ? -nrm : nrm;
    // v = x - alpha e1, normalised
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    for (int i = k + 1; i < n; ++i) v[i] = A[i * n + k];
    v[k + 1] -= alpha;
    double vn = 0;
    for (int i = k + 1; i < n; ++i) vn += v[i] * v[i];
    vn = std::sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = k + 1; i < n; ++i) v[i] /= vn;
    // A <- H A H with H = I - 2 v v^T: A - v w^T - w v^T, w = 2 A v - 2 (v^T A v) v
    for (int i = 0; i < n; ++i) {
      double acc = 0;
      for (int j = k + 1; j < n; ++j) acc += A[i * n + j] * v[j];
      pv[i] = 2.0 * acc;
    }
    double vpv = 0;
    for (int i = k + 1; i < n; ++i) vpv += v[i] * pv[i];
    for (int i = 0; i < n; ++i) pv[i] -= vpv * v[i];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) A[i * n + j] -= v[i] * pv[j] + pv[i] * v[j];
    // Q <- Q H
    for (int i = 0; i < n; ++i) {
      double acc = 0;
      for (int j = k + 1; j < n; ++j) acc += Q[i * n + j] * v[j];
      for (int j = k + 1; j < n; ++j) Q[i * n + j] -= 2.0 * acc * v[j];
    }
  }
  for (int i = 0; i < n; ++i) diag[i] = A[i * n + i];
  for (int i = 0; i + 1 < n; ++i) off[i] = A[(i + 1) * n + i];
  off[n - 1] = 0.0;
  // QL iterations on (diag, off); off[i] couples i and i + 1.
  const double tiny = 2.2204460492503131e-16;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m + 1 < n; ++m) {
        double dd = std::fabs(diag[m]) + std::fabs(diag[m + 1]);
        if (std::fabs(off[m]) <= tiny * dd) break;
      }
      if (m == l) break;
      if (++iter > 200) return false;
      double g = (diag[l + 1] - diag[l]) / (2.0 * off[l]);
      double r = std::hypot(g, 1.0);
      g = diag[m] - diag[l] + off[l] / (g + (g >= 0 ? r : -r));
      double sn = 1.0, cs = 1.0, p = 0.0;
      bool early = false;
      for (int i = m - 1; i >= l; --i) {
        double f = sn * off[i], b = cs * off[i];
        r = std::hypot(f, g);
        off[i + 1] = r;
        if (r == 0.0) {
          diag[i + 1] -= p;
          off[m] = 0.0;
          early = true;
          break;
        }
        sn = f / r;
        cs = g / r;
        g = diag[i + 1] - p;
        r = (diag[i] - g) * sn + 2.0 * cs * b;
        p = sn * r;
        diag[i + 1] = g + p;
        g = cs * r - b;
        for (int k = 0; k < n; ++k) {
          double t = Q[k * n + i + 1];
          Q[k * n + i + 1] = sn * Q[k * n + i] + cs * t;
          Q[k * n + i] = cs * Q[k * n + i] - sn * t;
        }
      }
      if (early) continue;
      diag[l] -= p;
      off[l] = g;
      off[m] = 0.0;
    }
  }
  // sort ascending
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return diag[a] < diag[b]; });
  for (int j = 0; j < n; ++j) {
    evals[j] = diag[order[j]];
    if (evecs)
      for (int i = 0; i < n; ++i) evecs[i * n + j] = Q[i * n + order[j]];
  }
  return true;
}

// ------------------------------------------------------------------ public helpers
int64_t lattice_node(const Setup& s, int64_t cell, int loc) {
  int64_t rem = cell, node = 0, stride = 1;
  int l = loc;
  for (int k = 0; k < s.dim; ++k) {
    int64_t ck = rem % s.n[k];
    rem /= s.n[k];
    int a = l % s.nn1;
    l /= s.nn1;
    node += (ck * s.p + a) * stride;
    stride *= s.lat[k];
  }
  return node;
}

int64_t locate_cell(const Setup& s, const double* x) {
  int64_t best = -1;
  int64_t base[3] = {0, 0, 0};
  for (int k = 0; k < s.dim; ++k) base[k] = (int64_t)std::floor((x[k] - s.lo[k]) / s.h[k]);
  int ncand = 1 << s.dim;
  for (int o = 0; o < ncand; ++o) {
    int64_t ck[3];
    bool ok = true;
    for (int k = 0; k < s.dim; ++k) {
      ck[k] = base[k] - ((o >> k) & 1);
      if (ck[k] < 0 || ck[k] >= s.n[k]) { ok = false; break; }
      double lo = s.lo[k] + ck[k] * s.h[k];
      if (x[k] < lo - 1e-14 || x[k] > lo + s.h[k] + 1e-14) { ok = false; break; }
    }
    if (!ok) continue;
    int64_t cell = 0, stride = 1;
    for (int k = 0; k < s.dim; ++k) {
      cell += ck[k] * stride;
      stride *= s.n[k];
    }
    if (s.cls[cell] == kOutside) continue;
    if (best < 0 || cell < best) best = cell;
  }
  return best;
}

void shape_values(const Setup& s, int64_t cell, const double* x, double* N) {
  int64_t rem = cell;
  std::vector<double> L(s.dim * s.nn1);
  for (int k = 0; k < s.dim; ++k) {
    int64_t ck = rem % s.n[k];
    rem /= s.n[k];
    double t = 2.0 * (x[k] - (s.lo[k] + ck * s.h[k])) / s.h[k] - 1.0;
    lagrange1d(s.gll_x, t, &L[k * s.nn1], nullptr);
  }
  for (int j = 0; j < s.nn_loc; ++j) {
    int jj = j;
    double v = 1.0;
    for (int k = 0; k < s.dim; ++k) {
      v *= L[k * s.nn1 + jj % s.nn1];
      jj /= s.nn1;
    }
    N[j] = v;
  }
}

double indicator(const SetupInput& in, const double* x) {
  Geo g(in);
  return g.physical_point(x) ? 1.0 : in.alpha;
}

void gauss_load(const Setup& s, const SetupInput& in, const double* xl, double sigma,
                std::vector<int64_t>& dofs, std::vector<double>& vals) {
  // kept cells within 8 sigma of x_l (f_s < 1.3e-14 beyond); each split into m^d subcells,
  // m = max(1, ceil(max_k h_k / sigma)), with (p + 4)-point Gauss-Legendre rules per axis
  Geo geo(in);
  const double reach = 8.0 * sigma;
  double hmax = 0.0;
  for (int k = 0; k < s.dim; ++k) hmax = std::max(hmax, s.h[k]);
  const int m = std::max(1, (int)std::ceil(hmax / sigma));
  std::vector<double> xg, wg;
  gauss_rule(s.p + 4, xg, wg);
  const int nq = (int)xg.size(), n1 = m * nq;   // points per axis and cell
  std::vector<double> px(3 * n1), pw(3 * n1), L(3 * (size_t)n1 * s.nn1);
  std::vector<double> acc(s.nn_loc);
  for (int64_t e = 0; e < s.n_elem; ++e) {
    if (s.cls[e] == kOutside) continue;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, gap2 = 0.0;
    int64_t rem = e;
    for (int k = 0; k < s.dim; ++k) {
      lo[k] = s.lo[k] + (rem % s.n[k]) * s.h[k];
      hi[k] = lo[k] + s.h[k];
      rem /= s.n[k];
      const double g = std::max(std::max(lo[k] - xl[k], xl[k] - hi[k]), 0.0);
      gap2 += g * g;
    }
    if (std::sqrt(gap2) > reach) continue;
    // composite points and weights per axis, and the 1D basis values at them
    for (int k = 0; k < s.dim; ++k)
      for (int a = 0; a < m; ++a) {
        const double sa = lo[k] + (hi[k] - lo[k]) * a / m, sb = lo[k] + (hi[k] - lo[k]) * (a + 1) / m;
        for (int q = 0; q < nq; ++q) {
          const int i = a * nq + q;
          px[k * n1 + i] = sa + (xg[q] + 1.0) * 0.5 * (sb - sa);
          pw[k * n1 + i] = wg[q] * 0.5 * (sb - sa);
          lagrange1d(s.gll_x, 2.0 * (px[k * n1 + i] - lo[k]) / s.h[k] - 1.0, &L[((size_t)k * n1 + i) * s.nn1], nullptr);
        }
      }
    std::fill(acc.begin(), acc.end(), 0.0);
    const int nz = s.dim == 3 ? n1 : 1;
    for (int iz = 0; iz < nz; ++iz)
      for (int iy = 0; iy < n1; ++iy)
        for (int ix = 0; ix < n1; ++ix) {
          const int idx[3] = {ix, iy, iz};
          double x[3] = {0, 0, 0}, w = in.rho, r2 = 0.0;
          for (int k = 0; k < s.dim; ++k) {
            x[k] = px[k * n1 + idx[k]];
            w *= pw[k * n1 + idx[k]];
            r2 += (x[k] - xl[k]) * (x[k] - xl[k]);
          }
          w *= std::exp(-0.5 * r2 / (sigma * sigma)) * (geo.physical_point(x) ? 1.0 : in.alpha);
          for (int j = 0; j < s.nn_loc; ++j) {
            int jj = j;
            double v = w;
            for (int k = 0; k < s.dim; ++k) {
              v *= L[((size_t)k * n1 + idx[k]) * s.nn1 + jj % s.nn1];
              jj /= s.nn1;
            }
            acc[j] += v;
          }
        }
    for (int l = 0; l < s.nn_loc; ++l) {
      if (acc[l] == 0.0) continue;
      for (int c = 0; c < s.ncomp; ++c) {
        dofs.push_back(lattice_node(s, e, l) * s.ncomp + c);
        vals.push_back(acc[l]);
      }
    }
  }
}

void edge_traction(const Setup& s, const SetupInput& in, double y0, double y1,
                   const double* t, std::vector<int64_t>& dofs, std::vector<double>& vals) {
  Geo geo(in);
  std::vector<double> gx, gw;
  gauss_rule(s.p + 1, gx, gw);
  std::vector<double> L(s.nn1);
  for (int ey = 0; ey < s.n[1]; ++ey) {
    int64_t cell = (int64_t)ey * s.n[0];
    if (s.cls[cell] == kOutside) continue;
    double ylo = s.lo[1] + ey * s.h[1], yhi = ylo + s.h[1];
    double a0 = std::max(ylo, y0), a1 = std::min(yhi, y1);
    if (a1 <= a0) continue;
    // only local nodes with x-index 0 are nonzero on the edge x = lo_x
    std::vector<double> integ(s.nn1, 0.0);
    for (size_t q = 0; q < gx.size(); ++q) {
      double y = a0 + (gx[q] + 1.0) * 0.5 * (a1 - a0);
      double w = gw[q] * 0.5 * (a1 - a0);
      double xp[3] = {s.lo[0], y, 0.0};
      double al = geo.physical_point(xp) ? 1.0 : in.alpha;
      lagrange1d(s.gll_x, 2.0 * (y - ylo) / s.h[1] - 1.0, L.data(), nullptr);
      for (int b = 0; b < s.nn1; ++b) integ[b] += w * al * L[b];
    }
    for (int b = 0; b < s.nn1; ++b) {
      int64_t node = lattice_node(s, cell, b * s.nn1);
      for (int c = 0; c < s.ncomp; ++c) {
        double v = integ[b] * t[c];
        if (v == 0.0) continue;
        dofs.push_back(node * s.ncomp + c);
        vals.push_back(v);
      }
    }
  }
}

// ------------------------------------------------------------------ build
Setup build_setup(const SetupInput& in) {
  Setup s;
  if (in.dim != 2 && in.dim != 3) throw std::invalid_argument("dim must be 2 or 3");
  if (in.p < 1 || in.p > 8) throw std::invalid_argument("p must be in 1..8");
  if (in.physics == 1 && in.dim != 2) throw std::invalid_argument("plane strain needs dim 2");
  s.dim = in.dim;
  s.p = in.p;
  s.ncomp = in.physics == 1 ? 2 : 1;
  s.nn1 = in.p + 1;
  s.nn_loc = 1;
  for (int k = 0; k < s.dim; ++k) s.nn_loc *= s.nn1;
  s.n_loc = s.nn_loc * s.ncomp;
  s.n_elem = 1;
  s.n_lat_nodes = 1;
  for (int k = 0; k < 3; ++k) {
    s.n[k] = k < s.dim ? in.n[k] : 1;
    if (s.n[k] < 1) throw std::invalid_argument("cells per axis must be >= 1");
    s.lo[k] = k < s.dim ? in.lo[k] : 0.0;
    s.h[k] = k < s.dim ? (in.hi[k] - in.lo[k]) / in.n[k] : 1.0;
    if (k < s.dim && !(s.h[k] > 0)) throw std::invalid_argument("empty extended box");
    s.lat[k] = k < s.dim ? (int64_t)s.n[k] * s.p + 1 : 1;
    s.n_elem *= s.n[k];
    s.n_lat_nodes *= s.lat[k];
  }
  s.n_lat_dof = s.n_lat_nodes * s.ncomp;
  gll_rule(s.p, s.gll_x, s.gll_w);
  Geo geo(in);

  // classification
  s.cls.assign(s.n_elem, kUncut);
  if (in.geom.kind != 0) {
    parallel_for(s.n_elem, [&](int64_t a, int64_t b) {
      for (int64_t e = a; e < b; ++e) {
        double blo[3], bhi[3];
        int64_t ilo[3] = {0, 0, 0}, rem = e;
        for (int k = 0; k < s.dim; ++k) {
          ilo[k] = rem % s.n[k];
          rem /= s.n[k];
          blo[k] = s.lo[k] + ilo[k] * s.h[k];
          bhi[k] = blo[k] + s.h[k];
        }
        s.cls[e] = geo.classify(blo, bhi, ilo, 1);
      }
    });
  }
  s.cut_index.assign(s.n_elem, -1);
  for (int64_t e = 0; e < s.n_elem; ++e) {
    if (s.cls[e] == kCut) {
      s.cut_index[e] = (int32_t)s.cut_cells.size();
      s.cut_cells.push_back(e);
    } else if (s.cls[e] == kUncut) {
      ++s.n_uncut;
    } else {
      ++s.n_outside;
    }
  }
  s.n_cut = (int64_t)s.cut_cells.size();
  if (s.n_cut + s.n_uncut == 0) throw std::domain_error("no cell intersects the physical domain");

  // node numbering: kept nodes in lattice order
  std::vector<uint8_t> used(s.n_lat_nodes, 0);
  for (int64_t e = 0; e < s.n_elem; ++e) {
    if (s.cls[e] == kOutside) continue;
    for (int l = 0; l < s.nn_loc; ++l) used[lattice_node(s, e, l)] = 1;
  }
  s.kept_of_lat.assign(s.n_lat_nodes, -1);
  for (int64_t i = 0; i < s.n_lat_nodes; ++i)
    if (used[i]) {
      s.kept_of_lat[i] = (int64_t)s.lat_of_kept.size();
      s.lat_of_kept.push_back(i);
    }
  s.n_kept_nodes = (int64_t)s.lat_of_kept.size();
  s.n_dof = s.n_kept_nodes * s.ncomp;

  // reference cell: GL stiffness, GLL lumped mass
  ElementIntegrator integ(s, in);
  const int nl = s.n_loc;
  s.Kref.assign(nl * nl, 0.0);
  {
    std::vector<double> Mgl(nl * nl, 0.0);   // GL mass of the full cell (not used by the SCM)
    double clo[3] = {s.lo[0], s.lo[1], s.lo[2]}, chi[3];
    for (int k = 0; k < 3; ++k) chi[k] = clo[k] + s.h[k];
    integ.accumulate(geo, clo, clo, chi, 1.0, s.Kref.data(), Mgl.data());
    ElementIntegrator::symmetrize(nl, s.Kref.data());
  }
  s.mref.assign(nl, 0.0);
  for (int j = 0; j < s.nn_loc; ++j) {
    int jj = j;
    double m = in.rho;
    for (int k = 0; k < s.dim; ++k) {
      m *= s.gll_w[jj % s.nn1] * 0.5 * s.h[k];
      jj /= s.nn1;
    }
    for (int c = 0; c < s.ncomp; ++c) s.mref[j * s.ncomp + c] = m;
  }
  auto lambda_max_lumped = [&](const double* K, const double* ml) {
    std::vector<double> A(nl * nl), ev(nl);
    for (int i = 0; i < nl; ++i)
      for (int j = 0; j < nl; ++j) A[i * nl + j] = K[i * nl + j] / std::sqrt(ml[i] * ml[j]);
    if (!sym_eig(nl, A.data(), ev.data(), nullptr)) throw std::runtime_error("eigensolver failed");
    return ev[nl - 1];
  };
  s.lambda_ref = lambda_max_lumped(s.Kref.data(), s.mref.data());
  // M^f of the eigenvalue stabilisation (Sec. 2.5): the mass of a cell inside the physical
  // domain as the SCM integrates it, i.e. with GLL quadrature (diagonal); its largest entry
  // scales M^s
  double mfull_max = *std::max_element(s.mref.begin(), s.mref.end());

  // distinct cut cells: with a voxel image holding a whole number r_k of voxels per cell and
  // axis (prod r_k <= 64), a cut cell's integrals depend only on its voxel block, so cells
  // with equal blocks share one set of matrices (computed for the first of them)
  std::vector<int64_t> rep;   // matrix index -> representative cut index
  s.cut_mat.assign(s.n_cut, 0);
  {
    const GeometryDesc& g = in.geom;
    bool blocks = g.kind == 2;
    int r[3] = {1, 1, 1}, nb = 1;
    for (int k = 0; blocks && k < s.dim; ++k) {
      blocks = g.vn[k] % s.n[k] == 0;
      r[k] = blocks ? g.vn[k] / s.n[k] : 1;
      nb *= r[k];
    }
    blocks = blocks && nb <= 64;
    std::unordered_map<uint64_t, int32_t> seen;
    for (int64_t ci = 0; ci < s.n_cut; ++ci) {
      if (!blocks) {
        s.cut_mat[ci] = (int32_t)rep.size();
        rep.push_back(ci);
        continue;
      }
      int64_t e = s.cut_cells[ci], rem = e, ic[3] = {0, 0, 0};
      for (int k = 0; k < s.dim; ++k) {
        ic[k] = rem % s.n[k];
        rem /= s.n[k];
      }
      uint64_t key = 0;
      int bit = 0;
      for (int c = 0; c < (s.dim == 3 ? r[2] : 1); ++c)
        for (int b = 0; b < r[1]; ++b)
          for (int a = 0; a < r[0]; ++a, ++bit) {
            int64_t vx = ic[0] * r[0] + a, vy = ic[1] * r[1] + b, vz = s.dim == 3 ? ic[2] * r[2] + c : 0;
            if (g.voxels[(size_t)((vz * g.vn[1] + vy) * g.vn[0] + vx)]) key |= 1ull << bit;
          }
      auto it = seen.find(key);
      if (it == seen.end()) {
        it = seen.emplace(key, (int32_t)rep.size()).first;
        rep.push_back(ci);
      }
      s.cut_mat[ci] = it->second;
    }
  }
  s.n_cut_mat = (int64_t)rep.size();

  // cut-cell matrices
  s.Kcut.assign((size_t)s.n_cut_mat * nl * nl, 0.0);
  s.mlcut.assign((size_t)s.n_cut_mat * nl, 0.0);
  if (in.need_consistent_mass) s.Mcut.assign((size_t)s.n_cut_mat * nl * nl, 0.0);
  parallel_for(s.n_cut_mat, [&](int64_t a, int64_t b) {
    std::vector<double> M(nl * nl), Ms(nl * nl), V(nl * nl), ev(nl);
    for (int64_t ci = a; ci < b; ++ci) {   // ci: matrix index
      int64_t e = s.cut_cells[rep[ci]];
      double clo[3] = {0, 0, 0};
      int64_t rem = e;
      for (int k = 0; k < s.dim; ++k) {
        clo[k] = s.lo[k] + (rem % s.n[k]) * s.h[k];
        rem /= s.n[k];
      }
      double* K = &s.Kcut[(size_t)ci * nl * nl];
      integ.cut_cell(geo, e, clo, K, M.data());
      // eigenvalue stabilisation M^e = M^o + eps M^s (Eq. epsilon_stabilization)
      if (in.stab == 1) {
        std::copy(M.begin(), M.end(), Ms.begin());
        if (!sym_eig(nl, Ms.data(), ev.data(), V.data())) throw std::runtime_error("EVS eigensolver failed");
        double thr = in.f_lambda * ev[nl - 1];
        std::fill(Ms.begin(), Ms.end(), 0.0);
        bool any = false;
        for (int j = 0; j < nl; ++j) {
          if (!(ev[j] < thr)) continue;
          any = true;
          for (int r = 0; r < nl; ++r) {
            double vr = V[r * nl + j];
            for (int c = 0; c < nl; ++c) Ms[r * nl + c] += vr * V[c * nl + j];
          }
        }
        if (any) {
          double mx = *std::max_element(Ms.begin(), Ms.end());
          double sc = in.eps * mfull_max / mx;
          for (int i = 0; i < nl * nl; ++i) M[i] += sc * Ms[i];
        }
      }
      // the consistent cut mass of the IMEX / consistent-mass schemes: M^o, plus eps M^s
      // with eigenvalue stabilisation
      if (in.need_consistent_mass) std::copy(M.begin(), M.end(), &s.Mcut[(size_t)ci * nl * nl]);
      // HRZ lumping: diagonal scaled to the element's total mass
      double total = 0, tr = 0;
      for (int i = 0; i < nl * nl; ++i) total += M[i];
      for (int i = 0; i < nl; ++i) tr += M[i * nl + i];
      double* ml = &s.mlcut[(size_t)ci * nl];
      for (int i = 0; i < nl; ++i) ml[i] = total * M[i * nl + i] / tr;
      if (in.stab == 2) {
        double lam = lambda_max_lumped(K, ml);
        double sc = std::max(1.0, lam / s.lambda_ref);
        for (int i = 0; i < nl; ++i) ml[i] *= sc;
      }
    }
  });

  // assembled lumped mass on the lattice
  s.ML.assign(s.n_lat_dof, 0.0);
  for (int64_t e = 0; e < s.n_elem; ++e) {
    if (s.cls[e] == kOutside) continue;
    const double* ml = s.cls[e] == kCut ? &s.mlcut[(size_t)s.cut_mat[s.cut_index[e]] * nl] : s.mref.data();
    for (int l = 0; l < s.nn_loc; ++l) {
      int64_t node = lattice_node(s, e, l);
      for (int c = 0; c < s.ncomp; ++c) s.ML[node * s.ncomp + c] += ml[l * s.ncomp + c];
    }
  }
  return s;
}

}  // namespace ibfem

// ====================================================================== IMEX (host)
namespace ibfem {

namespace {

// Supernode blocks of at most kMaxBlock rows: the GPU solves a block's dense diagonal part
// from a warp's 32 x 32 shared-memory copy; longer runs become a chain of blocks of rising
// height, whose couplings inside the run are off-block entries (solved row-parallel).
constexpr int64_t kMaxBlock = kImexSnMax;

// Records a run of `size` consecutive rows as supernodes starting at height h0; returns the
// height of its last block.
int push_blocks(int64_t size, int h0, std::vector<std::array<int64_t, 2>>& blocks) {
  int h = h0;
  for (int64_t done = 0; done < size; done += kMaxBlock, ++h)
    blocks.push_back({std::min(kMaxBlock, size - done), (int64_t)h});
  return h - 1;
}

// Geometric nested dissection of one connected vertex set: split along the longest axis
// at the median, take the vertices of the upper half adjacent to the lower half as the
// separator, order lower half, upper half, separator (recursively).  The leaf blocks and
// the separators are recorded as supernodes (size, height) in the same order; returns the
// height of the set's top supernode (-1 for an empty set).
int nested_dissection(std::vector<int64_t>& verts, const std::vector<int64_t>& Ap,
                      const std::vector<int64_t>& Ai, const std::vector<std::array<int64_t, 3>>& xyz,
                      std::vector<int32_t>& tag, int32_t& next_tag, std::vector<int64_t>& out,
                      std::vector<std::array<int64_t, 2>>& blocks) {
  const size_t kLeaf = 24;
  if (verts.empty()) return -1;
  auto leaf = [&]() {
    out.insert(out.end(), verts.begin(), verts.end());
    return push_blocks((int64_t)verts.size(), 0, blocks);
  };
  if (verts.size() <= kLeaf) return leaf();
  int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
  for (int64_t v : verts)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], xyz[v][k]);
      hi[k] = std::max(hi[k], xyz[v][k]);
    }
  int axis = 0;
  for (int k = 1; k < 3; ++k)
    if (hi[k] - lo[k] > hi[axis] - lo[axis]) axis = k;
  if (hi[axis] == lo[axis]) return leaf();
  std::sort(verts.begin(), verts.end(), [&](int64_t a, int64_t b) {
    return xyz[a][axis] != xyz[b][axis] ? xyz[a][axis] < xyz[b][axis] : a < b;
  });
  int64_t split = xyz[verts[verts.size() / 2]][axis];
  if (split == xyz[verts[0]][axis]) split += 1;  // keep both halves non-empty
  int32_t tA = next_tag++;
  std::vector<int64_t> A, B, S;
  for (int64_t v : verts)
    if (xyz[v][axis] < split) {
      A.push_back(v);
      tag[v] = tA;
    }
  for (int64_t v : verts) {
    if (xyz[v][axis] < split) continue;
    bool sep = false;
    for (int64_t p = Ap[v]; p < Ap[v + 1] && !sep; ++p)
      if (tag[Ai[p]] == tA) sep = true;
    (sep ? S : B).push_back(v);
  }
  if (A.empty() || (B.empty() && S.size() == verts.size())) return leaf();
  const int hA = nested_dissection(A, Ap, Ai, xyz, tag, next_tag, out, blocks);
  const int hB = nested_dissection(B, Ap, Ai, xyz, tag, next_tag, out, blocks);
  if (S.empty()) return std::max(hA, hB);
  out.insert(out.end(), S.begin(), S.end());
  return push_blocks((int64_t)S.size(), 1 + std::max(hA, hB), blocks);
}

// The sparse Cholesky factorisation below (elimination tree with path compression over
// ancestors, row patterns as reaches in that tree, up-looking factorisation one row of L at
// a time) is the published algorithm of T. A. Davis, "Direct Methods for Sparse Linear
// Systems", SIAM 2006, Ch. 4 (etree, ereach, up-looking Cholesky), in this library's data
// layout: L kept by columns with the diagonal first, plus its CSR by rows.

// Elimination tree of a symmetric matrix given by its full CSR pattern.
void etree(int64_t n, const std::vector<int64_t>& Ap, const std::vector<int64_t>& Ai,
           std::vector<int64_t>& parent) {
  std::vector<int64_t> anc(n, -1);
  parent.assign(n, -1);
  for (int64_t k = 0; k < n; ++k)
    for (int64_t p = Ap[k]; p < Ap[k + 1]; ++p) {
      int64_t j = Ai[p];
      while (j != -1 && j < k) {
        int64_t nx = anc[j];
        anc[j] = k;
        if (nx == -1) parent[j] = k;
        j = nx;
      }
    }
}

// Nonzero pattern of row k of L (columns < k) in topological order: s[top..n).
int64_t row_pattern(int64_t k, const std::vector<int64_t>& Ap, const std::vector<int64_t>& Ai,
                    const std::vector<int64_t>& parent, std::vector<int64_t>& s,
                    std::vector<int64_t>& mark, std::vector<int64_t>& path) {
  int64_t n = (int64_t)s.size(), top = n;
  mark[k] = k;
  for (int64_t p = Ap[k]; p < Ap[k + 1]; ++p) {
    int64_t j = Ai[p];
    if (j >= k) continue;
    int64_t len = 0;
    while (mark[j] != k) {
      path[len++] = j;
      mark[j] = k;
      j = parent[j];
    }
    while (len > 0) s[--top] = path[--len];
  }
  return top;
}

}  // namespace

bool sparse_cholesky(int64_t n, const std::vector<int64_t>& Ap, const std::vector<int64_t>& Ai,
                     const std::vector<double>& Ax, SparseChol& out, std::string& err) {
  // Up-looking factorisation A = L L^T, one row of L at a time; L kept by columns (CSC),
  // diagonal first in each column, which is the CSR of L^T used by the backward solve.
  std::vector<int64_t> parent, s(n), mark(n, -1), path(n);
  etree(n, Ap, Ai, parent);
  std::vector<int64_t> cnt(n, 1);
  for (int64_t k = 0; k < n; ++k) {
    int64_t top = row_pattern(k, Ap, Ai, parent, s, mark, path);
    for (int64_t t = top; t < n; ++t) cnt[s[t]]++;
  }
  std::vector<int64_t> Cp(n + 1, 0);
  for (int64_t j = 0; j < n; ++j) Cp[j + 1] = Cp[j] + cnt[j];
  std::vector<int64_t> Ci(Cp[n]);
  std::vector<double> Cx(Cp[n]);
  std::vector<int64_t> fill(n);
  for (int64_t j = 0; j < n; ++j) fill[j] = Cp[j] + 1;
  std::vector<double> x(n, 0.0);
  std::fill(mark.begin(), mark.end(), -1);
  for (int64_t k = 0; k < n; ++k) {
    int64_t top = row_pattern(k, Ap, Ai, parent, s, mark, path);
    double d = 0.0;
    for (int64_t p = Ap[k]; p < Ap[k + 1]; ++p) {
      int64_t j = Ai[p];
      if (j < k) x[j] = Ax[p];
      else if (j == k) d = Ax[p];
    }
    for (int64_t t = top; t < n; ++t) {
      int64_t i = s[t];
      double lki = x[i] / Cx[Cp[i]];
      x[i] = 0.0;
      for (int64_t p = Cp[i] + 1; p < fill[i]; ++p) x[Ci[p]] -= Cx[p] * lki;
      d -= lki * lki;
      Ci[fill[i]] = k;
      Cx[fill[i]] = lki;
      fill[i]++;
    }
    if (!(d > 0.0)) {
      err = "matrix is not positive definite at row " + std::to_string(k);
      return false;
    }
    Ci[Cp[k]] = k;
    Cx[Cp[k]] = std::sqrt(d);
  }
  out.n = n;
  out.Up = Cp;
  out.Ui = Ci;
  out.Ux = Cx;
  // CSR of L (rows), diagonal last
  std::vector<int64_t> rc(n, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Cp[j]; p < Cp[j + 1]; ++p) rc[Ci[p]]++;
  out.Lp.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) out.Lp[i + 1] = out.Lp[i] + rc[i];
  out.Li.assign(out.Lp[n], 0);
  out.Lx.assign(out.Lp[n], 0.0);
  std::vector<int64_t> pos(out.Lp.begin(), out.Lp.end() - 1);
  for (int64_t j = 0; j < n; ++j)   // columns in increasing order -> diagonal lands last
    for (int64_t p = Cp[j]; p < Cp[j + 1]; ++p) {
      int64_t i = Ci[p];
      out.Li[pos[i]] = j;
      out.Lx[pos[i]] = Cx[p];
      pos[i]++;
    }
  return true;
}

void imex_partition(const Setup& s, ImexData& d) {
  const int nl = s.n_loc, nc = s.ncomp;
  d.c_of_dof.assign(s.n_lat_dof, -1);
  std::vector<uint8_t> isc(s.n_lat_dof, 0);
  for (int64_t ci = 0; ci < s.n_cut; ++ci) {
    int64_t cell = s.cut_cells[ci];
    for (int l = 0; l < s.nn_loc; ++l) {
      int64_t node = lattice_node(s, cell, l);
      for (int c = 0; c < nc; ++c) isc[node * nc + c] = 1;
    }
  }
  d.c_dof.clear();
  for (int64_t g = 0; g < s.n_lat_dof; ++g)
    if (isc[g]) {
      d.c_of_dof[g] = (int64_t)d.c_dof.size();
      d.c_dof.push_back(g);
    }
  d.n_c = (int64_t)d.c_dof.size();
  // cells touching the c-set
  d.ccells.clear();
  std::vector<int64_t> loc_dof(nl);
  for (int64_t e = 0; e < s.n_elem; ++e) {
    if (s.cls[e] == kOutside) continue;
    bool any = false;
    for (int l = 0; l < s.nn_loc && !any; ++l)
      if (isc[lattice_node(s, e, l) * nc]) any = true;
    if (any) d.ccells.push_back(e);
  }
  // pattern of S over c indices: union of c-c couplings of the c-cells
  std::vector<std::vector<int64_t>> rows(d.n_c);
  for (int64_t e : d.ccells) {
    for (int l = 0; l < s.nn_loc; ++l)
      for (int c = 0; c < nc; ++c) loc_dof[l * nc + c] = d.c_of_dof[lattice_node(s, e, l) * nc + c];
    bool cut = s.cls[e] == kCut;
    for (int a = 0; a < nl; ++a) {
      if (loc_dof[a] < 0) continue;
      for (int b = 0; b < nl; ++b) {
        if (loc_dof[b] < 0) continue;
        if (!cut && s.Kref[(size_t)a * nl + b] == 0.0 && a != b) continue;
        rows[loc_dof[a]].push_back(loc_dof[b]);
      }
    }
  }
  d.Sp.assign(d.n_c + 1, 0);
  for (int64_t i = 0; i < d.n_c; ++i) {
    auto& r = rows[i];
    r.push_back(i);
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    d.Sp[i + 1] = d.Sp[i] + (int64_t)r.size();
  }
  d.Si.resize(d.Sp[d.n_c]);
  for (int64_t i = 0; i < d.n_c; ++i) std::copy(rows[i].begin(), rows[i].end(), d.Si.begin() + d.Sp[i]);
  rows.clear();
  // values of M^cc (consistent cut mass + nodal GLL mass of uncut cells) and K^cc
  d.Mx.assign(d.Si.size(), 0.0);
  d.Kx.assign(d.Si.size(), 0.0);
  auto slot = [&](int64_t i, int64_t j) {
    auto b = d.Si.begin() + d.Sp[i], en = d.Si.begin() + d.Sp[i + 1];
    return (int64_t)(std::lower_bound(b, en, j) - d.Si.begin());
  };
  for (int64_t e : d.ccells) {
    for (int l = 0; l < s.nn_loc; ++l)
      for (int c = 0; c < nc; ++c) loc_dof[l * nc + c] = d.c_of_dof[lattice_node(s, e, l) * nc + c];
    bool cut = s.cls[e] == kCut;
    const double* K = cut ? &s.Kcut[(size_t)s.cut_mat[s.cut_index[e]] * nl * nl] : s.Kref.data();
    const double* M = cut ? &s.Mcut[(size_t)s.cut_mat[s.cut_index[e]] * nl * nl] : nullptr;
    for (int a = 0; a < nl; ++a) {
      if (loc_dof[a] < 0) continue;
      for (int b = 0; b < nl; ++b) {
        if (loc_dof[b] < 0) continue;
        double kv = K[(size_t)a * nl + b];
        double mv = cut ? M[(size_t)a * nl + b] : (a == b ? s.mref[a] : 0.0);
        if (kv == 0.0 && mv == 0.0) continue;
        int64_t p = slot(loc_dof[a], loc_dof[b]);
        d.Kx[p] += kv;
        d.Mx[p] += mv;
      }
    }
  }
  // ordering: connected components (BFS), nested dissection inside each
  std::vector<std::array<int64_t, 3>> xyz(d.n_c);
  for (int64_t i = 0; i < d.n_c; ++i) {
    int64_t node = d.c_dof[i] / nc, rem = node;
    for (int k = 0; k < 3; ++k) {
      xyz[i][k] = k < s.dim ? rem % s.lat[k] : 0;
      if (k < s.dim) rem /= s.lat[k];
    }
  }
  std::vector<int32_t> comp(d.n_c, -1), tag(d.n_c, -1);
  int32_t next_tag = 0;
  d.perm.clear();
  d.comp_ptr.assign(1, 0);
  d.sn_start.clear();
  d.sn_size.clear();
  d.sn_height.clear();
  std::vector<std::array<int64_t, 2>> blocks;
  int64_t sn_row = 0;
  std::vector<int64_t> queue;
  for (int64_t r = 0; r < d.n_c; ++r) {
    if (comp[r] >= 0) continue;
    int32_t cid = (int32_t)d.comp_ptr.size() - 1;
    queue.assign(1, r);
    comp[r] = cid;
    for (size_t q = 0; q < queue.size(); ++q) {
      int64_t v = queue[q];
      for (int64_t p = d.Sp[v]; p < d.Sp[v + 1]; ++p)
        if (comp[d.Si[p]] < 0) {
          comp[d.Si[p]] = cid;
          queue.push_back(d.Si[p]);
        }
    }
    blocks.clear();
    nested_dissection(queue, d.Sp, d.Si, xyz, tag, next_tag, d.perm, blocks);
    for (auto& b : blocks) {
      d.sn_start.push_back(sn_row);
      d.sn_size.push_back((int32_t)b[0]);
      d.sn_height.push_back((int32_t)b[1]);
      sn_row += b[0];
    }
    d.comp_ptr.push_back((int32_t)d.perm.size());
  }
  d.iperm.assign(d.n_c, 0);
  for (int64_t r = 0; r < d.n_c; ++r) d.iperm[d.perm[r]] = r;
  // residual gather lists (permuted rows): entries slot * n_loc + loc over the c-cells
  std::vector<std::vector<int32_t>> g(d.n_c);
  for (size_t sl = 0; sl < d.ccells.size(); ++sl) {
    int64_t e = d.ccells[sl];
    for (int l = 0; l < s.nn_loc; ++l)
      for (int c = 0; c < nc; ++c) {
        int64_t ci = d.c_of_dof[lattice_node(s, e, l) * nc + c];
        if (ci >= 0) g[d.iperm[ci]].push_back((int32_t)(sl * nl + l * nc + c));
      }
  }
  d.g_ptr.assign(d.n_c + 1, 0);
  for (int64_t r = 0; r < d.n_c; ++r) d.g_ptr[r + 1] = d.g_ptr[r] + (int64_t)g[r].size();
  d.g_idx.clear();
  for (auto& v : g) d.g_idx.insert(d.g_idx.end(), v.begin(), v.end());
}

static void permuted(const ImexData& d, const std::vector<double>& vals, std::vector<int64_t>& P,
                     std::vector<int64_t>& I, std::vector<double>& X) {
  P.assign(d.n_c + 1, 0);
  for (int64_t r = 0; r < d.n_c; ++r) P[r + 1] = P[r] + (d.Sp[d.perm[r] + 1] - d.Sp[d.perm[r]]);
  I.resize(P[d.n_c]);
  X.resize(P[d.n_c]);
  std::vector<std::pair<int64_t, double>> row;
  for (int64_t r = 0; r < d.n_c; ++r) {
    int64_t i = d.perm[r];
    row.clear();
    for (int64_t p = d.Sp[i]; p < d.Sp[i + 1]; ++p) row.push_back({d.iperm[d.Si[p]], vals[p]});
    std::sort(row.begin(), row.end());
    for (size_t q = 0; q < row.size(); ++q) {
      I[P[r] + q] = row[q].first;
      X[P[r] + q] = row[q].second;
    }
  }
}

bool imex_factor(const Setup& s, double beta_dt2, ImexData& d, std::string& err) {
  (void)s;
  std::vector<double> Sx(d.Mx.size());
  for (size_t p = 0; p < Sx.size(); ++p) Sx[p] = d.Mx[p] + beta_dt2 * d.Kx[p];
  std::vector<int64_t> P, I;
  std::vector<double> X;
  permuted(d, Sx, P, I, X);
  if (!sparse_cholesky(d.n_c, P, I, X, d.chol, err)) return false;
  d.beta_dt2 = beta_dt2;
  // block solve data: each supernode's dense diagonal block of L, and where each row's
  // entries leave its block (the rows of L and of L^T are sorted by column)
  const SparseChol& L = d.chol;
  const size_t nsn = d.sn_start.size();
  d.sn_doff.assign(nsn + 1, 0);
  for (size_t q = 0; q < nsn; ++q) d.sn_doff[q + 1] = d.sn_doff[q] + (int64_t)d.sn_size[q] * d.sn_size[q];
  d.sn_D.assign((size_t)d.sn_doff[nsn], 0.0);
  d.sn_DT.assign((size_t)d.sn_doff[nsn], 0.0);
  d.f_off_end.assign(d.n_c, 0);
  d.b_off_beg.assign(d.n_c, 0);
  std::vector<double> Ls;
  for (size_t q = 0; q < nsn; ++q) {
    const int64_t st = d.sn_start[q], w = d.sn_size[q], en = st + w;
    Ls.assign((size_t)w * w, 0.0);
    for (int64_t r = st; r < en; ++r) {
      int64_t p = L.Lp[r];
      while (p < L.Lp[r + 1] && L.Li[p] < st) ++p;
      d.f_off_end[r] = p;
      for (; p < L.Lp[r + 1]; ++p) Ls[(size_t)(r - st) * w + (L.Li[p] - st)] = L.Lx[p];
      int64_t pb = L.Up[r];
      while (pb < L.Up[r + 1] && L.Ui[pb] < en) ++pb;
      d.b_off_beg[r] = pb;
    }
    // the dense block itself (substitution within it is backward stable, unlike an
    // explicit inverse), row-major and transposed, with 1 / L_jj in the diagonal slots
    double* D = &d.sn_D[(size_t)d.sn_doff[q]];
    double* DT = &d.sn_DT[(size_t)d.sn_doff[q]];
    for (int64_t i = 0; i < w; ++i)
      for (int64_t j = 0; j <= i; ++j) {
        const double v = i == j ? 1.0 / Ls[(size_t)i * w + i] : Ls[(size_t)i * w + j];
        D[i * w + j] = v;
        DT[j * w + i] = v;
      }
  }
  // supernodes by height of the dissection tree over all components (the GPU solves every
  // supernode of one height per launch)
  int hmax = -1;
  for (size_t q = 0; q < nsn; ++q) hmax = std::max(hmax, d.sn_height[q]);
  d.gh_sn_ptr.assign(1, 0);
  d.gh_sn.clear();
  for (int h = 0; h <= hmax; ++h) {
    for (size_t q = 0; q < nsn; ++q)
      if (d.sn_height[q] == h) d.gh_sn.push_back((int32_t)q);
    d.gh_sn_ptr.push_back((int32_t)d.gh_sn.size());
  }
  // work split of the off-block sums, per direction: the tpr threads of a row take its
  // entries in turn, and a supernode gets g CTAs, each with the same fraction of every row,
  // g chosen so that no thread sums more than kImexThreadEntries entries (its loads are
  // issued together, before the CTA waits); partial sums of split supernodes at pbase (32
  // per CTA).
  //
  // Waits: with the elimination tree of L (parent(j) = the first row below the diagonal in
  // column j), an entry L_ij != 0 (i > j) makes i an ancestor of j, and the path from j up
  // to i climbs in row order.  So in the forward sweep a supernode needs only the supernodes
  // of the rows whose parent lies in it (every other row it reads is below one of those on
  // a tree path, finished before them), and in the backward sweep only the supernodes of
  // its rows' parents.  CTAs take supernodes by height of the dissection tree (forward
  // upwards, backward downwards; the chains of every component start at once) if that order
  // is topological for the waits, else by index (always topological: a wait is on a lower
  // index forward, a higher one backward): every wait is on a supernode taken earlier.
  std::vector<int32_t> sn_of(d.n_c, 0);
  for (size_t q = 0; q < nsn; ++q)
    for (int64_t r = d.sn_start[q]; r < d.sn_start[q] + d.sn_size[q]; ++r) sn_of[r] = (int32_t)q;
  std::vector<std::vector<int32_t>> fdep(nsn), bdep(nsn);
  for (int64_t j = 0; j < d.n_c; ++j) {
    if (L.Up[j + 1] - L.Up[j] < 2) continue;          // a root: no entry below the diagonal
    const int64_t par = L.Ui[L.Up[j] + 1];
    const int32_t a = sn_of[j], b = sn_of[par];
    if (a == b) continue;
    fdep[b].push_back(a);
    bdep[a].push_back(b);
  }
  for (int dir = 0; dir < 2; ++dir) {
    ImexSplit& sp = dir == 0 ? d.fsplit : d.bsplit;
    sp.g.assign(nsn, 1);
    sp.tpr.assign(nsn, 32);
    sp.pbase.assign(nsn, 0);
    int64_t parts = 0;
    for (size_t q = 0; q < nsn; ++q) {
      int64_t lng = 0;
      for (int64_t r = d.sn_start[q]; r < d.sn_start[q] + d.sn_size[q]; ++r)
        lng = std::max(lng, dir == 0 ? d.f_off_end[r] - L.Lp[r] : L.Up[r + 1] - d.b_off_beg[r]);
      int tpr = 32;
      while (tpr > 8 && tpr * d.sn_size[q] > 256) tpr >>= 1;
      const int64_t per_cta = kImexThreadEntries * tpr;
      const int64_t g = std::min<int64_t>(kImexMaxSplit, std::max<int64_t>(1, (lng + per_cta - 1) / per_cta));
      sp.g[q] = (int32_t)g;
      sp.tpr[q] = tpr;
      if (g > 1) {
        sp.pbase[q] = parts;
        parts += g * 32;
      }
    }
    sp.n_parts = parts;
    auto& deps = dir == 0 ? fdep : bdep;
    sp.dep_ptr.assign(1, 0);
    sp.dep.clear();
    for (size_t q = 0; q < nsn; ++q) {
      std::vector<int32_t>& v = deps[q];
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
      sp.dep.insert(sp.dep.end(), v.begin(), v.end());
      sp.dep_ptr.push_back((int32_t)sp.dep.size());
    }
    // order: by height (forward ascending, backward descending), ties by index
    sp.order.resize(nsn);
    for (size_t q = 0; q < nsn; ++q) sp.order[q] = (int32_t)q;
    std::stable_sort(sp.order.begin(), sp.order.end(), [&](int32_t a, int32_t b) {
      return dir == 0 ? d.sn_height[a] < d.sn_height[b] : d.sn_height[a] > d.sn_height[b];
    });
    if (dir == 1) {
      // descending index within a height
      size_t k0 = 0;
      while (k0 < nsn) {
        size_t k1 = k0;
        while (k1 < nsn && d.sn_height[sp.order[k1]] == d.sn_height[sp.order[k0]]) ++k1;
        std::reverse(sp.order.begin() + k0, sp.order.begin() + k1);
        k0 = k1;
      }
    }
    std::vector<int32_t> pos(nsn, 0);
    for (size_t k = 0; k < nsn; ++k) pos[sp.order[k]] = (int32_t)k;
    bool topo = true;
    for (size_t q = 0; q < nsn && topo; ++q)
      for (int32_t k = sp.dep_ptr[q]; k < sp.dep_ptr[q + 1]; ++k)
        if (pos[sp.dep[k]] >= pos[q]) {
          topo = false;
          break;
        }
    if (!topo)
      for (size_t q = 0; q < nsn; ++q) sp.order[q] = (int32_t)(dir == 0 ? q : nsn - 1 - q);
  }
  return true;
}

bool imex_check_schedule(const Setup& s, const ImexData& part, double beta_dt2, uint64_t seed,
                         int64_t& violations, double& rel_err, std::string& err) {
  ImexData d = part;
  if (!imex_factor(s, beta_dt2, d, err)) return false;
  const SparseChol& L = d.chol;
  const int64_t n = d.n_c;
  const size_t nsn = d.sn_start.size();
  violations = 0;
  rel_err = 0.0;
  if (n == 0) return true;
  // the supernodes cover the rows once, in order, each within the GPU's block size
  std::vector<int32_t> sn_of(n, -1);
  int64_t next = 0;
  for (size_t q = 0; q < nsn; ++q) {
    if (d.sn_start[q] != next || d.sn_size[q] < 1 || d.sn_size[q] > kImexSnMax) ++violations;
    for (int64_t r = d.sn_start[q]; r < d.sn_start[q] + d.sn_size[q] && r < n; ++r) sn_of[r] = (int32_t)q;
    next = d.sn_start[q] + d.sn_size[q];
  }
  if (next != n) ++violations;
  if (violations) return true;
  // a deterministic generator for the right-hand side and the schedules (splitmix64)
  auto rnd = [&seed]() {
    seed += 0x9e3779b97f4a7c15ULL;
    uint64_t z = seed;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
  };
  std::vector<double> b(n), y(n), x(n);
  for (int64_t r = 0; r < n; ++r) b[r] = (double)(rnd() >> 11) * 0x1.0p-53 - 0.5;
  // plain substitution: L y = b by rows (diagonal last), L^T x = y by rows of L^T (diagonal first)
  for (int64_t r = 0; r < n; ++r) {
    double a = b[r];
    for (int64_t p = L.Lp[r]; p < L.Lp[r + 1] - 1; ++p) a -= L.Lx[p] * y[L.Li[p]];
    y[r] = a / L.Lx[L.Lp[r + 1] - 1];
  }
  for (int64_t r = n - 1; r >= 0; --r) {
    double a = y[r];
    for (int64_t p = L.Up[r] + 1; p < L.Up[r + 1]; ++p) a -= L.Ux[p] * x[L.Ui[p]];
    x[r] = a / L.Ux[L.Up[r]];
  }
  std::vector<double> cur, in = b;
  for (int dir = 0; dir < 2; ++dir) {
    const bool fwd = dir == 0;
    const ImexSplit& sp = fwd ? d.fsplit : d.bsplit;
    // the ticket order is topological for the waits
    std::vector<int64_t> pos(nsn, -1);
    for (size_t k = 0; k < sp.order.size(); ++k) pos[sp.order[k]] = (int64_t)k;
    for (size_t q = 0; q < nsn; ++q) {
      if (pos[q] < 0) ++violations;
      for (int32_t k = sp.dep_ptr[q]; k < sp.dep_ptr[q + 1]; ++k)
        if (pos[sp.dep[k]] >= pos[q]) ++violations;
      // the work split: partial sums in range, at most kImexThreadEntries per thread
      const int64_t g = sp.g[q];
      if (g < 1 || g > kImexMaxSplit || (g > 1 && (sp.pbase[q] % 32 != 0 || sp.pbase[q] + 32 * g > sp.n_parts)))
        ++violations;
      for (int64_t r = d.sn_start[q]; r < d.sn_start[q] + d.sn_size[q]; ++r) {
        const int64_t len = fwd ? d.f_off_end[r] - L.Lp[r] : L.Up[r + 1] - d.b_off_beg[r];
        if (g < kImexMaxSplit && ((len + g - 1) / g + sp.tpr[q] - 1) / sp.tpr[q] > kImexThreadEntries) ++violations;
      }
    }
    // random asynchronous schedules of ready supernodes; a row not yet final holds NaN, so a
    // read that the waits do not cover poisons the result and is counted
    cur.assign(n, std::numeric_limits<double>::quiet_NaN());
    std::vector<char> done(nsn, 0);
    size_t n_done = 0;
    std::vector<int32_t> ready, run;
    std::vector<std::pair<int64_t, double>> writes;
    while (n_done < nsn) {
      ready.clear();
      for (size_t q = 0; q < nsn; ++q) {
        if (done[q]) continue;
        bool ok = true;
        for (int32_t k = sp.dep_ptr[q]; k < sp.dep_ptr[q + 1] && ok; ++k) ok = done[sp.dep[k]] != 0;
        if (ok) ready.push_back((int32_t)q);
      }
      if (ready.empty()) {   // a cycle of waits
        ++violations;
        return true;
      }
      run.clear();
      for (int32_t q : ready)
        if (rnd() % 3 == 0) run.push_back(q);
      if (run.empty()) run.push_back(ready[rnd() % ready.size()]);
      writes.clear();
      for (int32_t q : run) {   // every supernode of a round reads before any of them writes
        const int64_t st = d.sn_start[q];
        const int wd = d.sn_size[q];
        double T[kImexSnMax];
        for (int i = 0; i < wd; ++i) {
          const int64_t r = st + i;
          const int64_t p0 = fwd ? L.Lp[r] : d.b_off_beg[r], p1 = fwd ? d.f_off_end[r] : L.Up[r + 1];
          double acc = 0.0;
          for (int64_t p = p0; p < p1; ++p) {
            const int64_t c = fwd ? L.Li[p] : L.Ui[p];
            if (c >= st && c < st + wd) ++violations;   // an in-block entry listed off-block
            if (std::isnan(cur[c])) ++violations;
            acc += (fwd ? L.Lx[p] : L.Ux[p]) * cur[c];
          }
          T[i] = in[r] - acc;
        }
        const double* M = (fwd ? d.sn_DT.data() : d.sn_D.data()) + d.sn_doff[q];
        for (int jj = 0; jj < wd; ++jj) {
          const int j = fwd ? jj : wd - 1 - jj;
          const double xj = T[j] * M[(size_t)j * wd + j];
          T[j] = xj;
          for (int l = 0; l < wd; ++l)
            if (fwd ? l > j : l < j) T[l] -= M[(size_t)j * wd + l] * xj;
        }
        for (int i = 0; i < wd; ++i) writes.push_back({st + i, T[i]});
      }
      for (const auto& w : writes) cur[w.first] = w.second;
      for (int32_t q : run) done[q] = 1;
      n_done += run.size();
    }
    const std::vector<double>& ref = fwd ? y : x;
    double e2 = 0.0, r2 = 0.0;
    for (int64_t r = 0; r < n; ++r) {
      e2 += (cur[r] - ref[r]) * (cur[r] - ref[r]);
      r2 += ref[r] * ref[r];
    }
    rel_err = std::max(rel_err, r2 > 0.0 ? std::sqrt(e2 / r2) : std::sqrt(e2));
    in = cur;   // the backward sweep solves with the forward result
  }
  return true;
}

bool imex_mass_solve(const ImexData& d, const std::vector<double>& b, std::vector<double>& a,
                     std::string& err) {
  std::vector<int64_t> P, I;
  std::vector<double> X;
  permuted(d, d.Mx, P, I, X);
  SparseChol c;
  if (!sparse_cholesky(d.n_c, P, I, X, c, err)) return false;
  std::vector<double> y(d.n_c);
  for (int64_t r = 0; r < d.n_c; ++r) y[r] = b[d.perm[r]];
  for (int64_t r = 0; r < d.n_c; ++r) {
    double acc = y[r];
    for (int64_t p = c.Lp[r]; p + 1 < c.Lp[r + 1]; ++p) acc -= c.Lx[p] * y[c.Li[p]];
    y[r] = acc / c.Lx[c.Lp[r + 1] - 1];
  }
  for (int64_t r = d.n_c - 1; r >= 0; --r) {
    double acc = y[r];
    for (int64_t p = c.Up[r] + 1; p < c.Up[r + 1]; ++p) acc -= c.Ux[p] * y[c.Ui[p]];
    y[r] = acc / c.Ux[c.Up[r]];
  }
  a.assign(d.n_c, 0.0);
  for (int64_t r = 0; r < d.n_c; ++r) a[d.perm[r]] = y[r];
  return true;
}

}  // namespace ibfem
