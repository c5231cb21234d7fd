// Host-side construction of the spectral-cell discretisation (library side).
//
// Everything here runs once per problem, before any time step: cell classification,
// space-tree quadrature of cut cells, element matrices with the finite cell indicator,
// eigenvalue stabilisation, HRZ lumping, mass scaling, the lumped mass on the node
// lattice, loads, observers and the IMEX partition with its Cholesky factor.  The
// result is a set of flat arrays in the device layout (node lattice, x fastest,
// components interleaved) that the runtime uploads.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace ibfem {

enum CellClass : uint8_t { kOutside = 0, kCut = 1, kUncut = 2 };

struct GeometryDesc {
  int kind = 0;                 // IBFEM_GEOM_*
  std::vector<double> shapes;   // holes: (c..., r); rotated box: (edge, c[3], T[9])
  std::vector<uint8_t> voxels;  // x fastest
  int vn[3] = {1, 1, 1};
  int quad_depth = 0;
};

struct SetupInput {
  int dim = 2;
  int n[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  int p = 2;
  int physics = 0;  // 0 scalar, 1 plane strain
  double rho = 1, c = 1, E = 1, nu = 0.3;
  double alpha = 1e-5;
  int stab = 0;     // 0 none, 1 EVS, 2 mass scaling
  double eps = 0, f_lambda = 1e-2;
  GeometryDesc geom;
  bool need_consistent_mass = false;  // IMEX: keep the consistent cut mass
};

struct Setup {
  // grid
  int dim = 2, p = 2, ncomp = 1, nn1 = 3, nn_loc = 9, n_loc = 9;
  int n[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, h[3] = {1, 1, 1};
  int64_t lat[3] = {1, 1, 1};   // lattice nodes per axis
  int64_t n_lat_nodes = 0, n_lat_dof = 0, n_elem = 0;
  // classification
  std::vector<uint8_t> cls;          // per cell
  std::vector<int32_t> cut_index;    // per cell, -1 unless cut
  std::vector<int64_t> cut_cells;    // cut index -> cell
  int64_t n_uncut = 0, n_cut = 0, n_outside = 0;
  // numbering
  std::vector<int64_t> kept_of_lat;  // lattice node -> kept node or -1
  std::vector<int64_t> lat_of_kept;  // kept node -> lattice node
  int64_t n_kept_nodes = 0, n_dof = 0;
  // matrices
  std::vector<double> Kref;          // n_loc^2
  std::vector<double> mref;          // n_loc, GLL lumped
  double lambda_ref = 0;
  // cut-cell matrices, one set per distinct cut cell: cut cells of a voxel geometry whose
  // voxel sub-images are equal have equal integrals and share one set
  std::vector<int32_t> cut_mat;      // cut index -> matrix index
  int64_t n_cut_mat = 0;
  std::vector<double> Kcut;          // n_cut_mat * n_loc^2, row-major, symmetric
  std::vector<double> Mcut;          // n_cut_mat * n_loc^2 consistent (alpha) mass (if kept)
  std::vector<double> mlcut;         // n_cut_mat * n_loc lumped (HRZ [+EVS] [x scale])
  std::vector<double> ML;            // lattice dof -> assembled lumped mass (0 = dead)
  // 1D GLL data
  std::vector<double> gll_x, gll_w;
};

// Throws std::runtime_error with a message on failure; `code` receives an IBFEM_ERR_*.
Setup build_setup(const SetupInput& in);

// Shape functions of cell `cell` at physical point x: writes nn_loc values.
void shape_values(const Setup& s, int64_t cell, const double* x, double* N);

// Cell containing x (lowest kept index among the closed boxes), or -1.
int64_t locate_cell(const Setup& s, const double* x);

// Lattice node index of local node `loc` of `cell`.
int64_t lattice_node(const Setup& s, int64_t cell, int loc);

// alpha^FCM at a point (1 inside the physical domain).
double indicator(const SetupInput& in, const double* x);

// Volumetric Gaussian load of the benchmark (Sec. 3.1): int alpha^FCM rho f_s N_i over the
// kept cells, f_s = exp(-|x - xl|^2 / (2 sigma^2)); (lattice dof, value) pairs.
void gauss_load(const Setup& s, const SetupInput& in, const double* xl, double sigma,
                std::vector<int64_t>& dofs, std::vector<double>& vals);

// Edge-traction load on x = lo_x, y in [y0, y1]: returns (lattice dof, value) pairs.
void edge_traction(const Setup& s, const SetupInput& in, double y0, double y1,
                   const double* t, std::vector<int64_t>& dofs, std::vector<double>& vals);

// Symmetric eigen-decomposition (Householder tridiagonalisation + implicit QL).
// A is n x n row-major (destroyed); evals ascending; evecs (row-major, column j =
// eigenvector j) if non-null.  Returns false if QL fails to converge.
bool sym_eig(int n, double* A, double* evals, double* evecs);

// Simplicial sparse Cholesky of a symmetric positive definite CSR matrix (full pattern)
// after the given symmetric permutation.  Produces L in CSR (rows, strictly lower part
// plus diagonal last in each row) and level sets for the forward solve.
struct SparseChol {
  int64_t n = 0;
  std::vector<int64_t> Lp, Li;       // CSR of L (lower), diagonal stored last per row
  std::vector<double> Lx;
  std::vector<int64_t> Up, Ui;       // CSR of L^T (upper), diagonal first per row
  std::vector<double> Ux;
};
bool sparse_cholesky(int64_t n, const std::vector<int64_t>& Ap, const std::vector<int64_t>& Ai,
                     const std::vector<double>& Ax, SparseChol& out, std::string& err);

// IMEX partition (Sec. 2.6, Algorithm 2): the c-set (DOFs with support in a cut cell),
// the consistent M^cc and K^cc on it, and the Cholesky factor of S = M^cc + beta dt^2 K^cc
// in a fill-reducing order (connected components, then geometric nested dissection), with
// the supernodes of that order for the block triangular solves.
// Off-block entries of one row that one thread of the GPU block solve sums (the host picks
// the CTAs per supernode so that no thread has more), and the most CTAs one supernode's
// sums are split over (beyond that the threads loop).
constexpr int64_t kImexThreadEntries = 8;
constexpr int64_t kImexMaxSplit = 256;
// Rows of a supernode at most (the GPU solves its dense diagonal block in one warp).
constexpr int kImexSnMax = 32;

// One direction's sweep of the block solve (forward: L y = b; backward: L^T x = y): the
// split of each supernode's off-block sums over CTAs, the supernodes each one waits for, and
// the order in which CTAs take the supernodes (a topological order of those waits).
struct ImexSplit {
  std::vector<int32_t> g;        // per supernode: CTAs
  std::vector<int32_t> tpr;      // per supernode: threads per row (256 / wd rounded down to
                                 // a power of two, at most 32)
  std::vector<int64_t> pbase;    // per supernode split over g > 1 CTAs: first partial sum
  int64_t n_parts = 0;           // partial sums of all split supernodes
  std::vector<int32_t> dep_ptr, dep;   // per supernode: the supernodes it waits for
  std::vector<int32_t> order;    // supernodes in the order their CTAs are taken
};

struct ImexData {
  int64_t n_c = 0;
  std::vector<int64_t> c_dof;          // c index -> lattice DOF (lattice order)
  std::vector<int64_t> c_of_dof;       // lattice DOF -> c index or -1
  std::vector<int64_t> ccells;         // kept cells with at least one c-DOF
  // symmetric pattern of S over c indices (CSR, full) and the two value arrays
  std::vector<int64_t> Sp, Si;
  std::vector<double> Mx, Kx;
  // ordering: permuted row r -> c index, components as contiguous row ranges
  std::vector<int64_t> perm, iperm;
  std::vector<int32_t> comp_ptr;
  // residual gather: permuted row r -> entries (slot * n_loc + loc) into the c-cell products
  std::vector<int64_t> g_ptr;
  std::vector<int32_t> g_idx;
  // factor of S (rebuilt per dt)
  SparseChol chol;
  double beta_dt2 = 0.0;
  // supernodes of the nested-dissection order (dt-independent): contiguous row ranges (the
  // leaf blocks and the separators), each depending only on the supernodes below it in the
  // dissection tree; height 0 for a leaf, one above its highest child for a separator
  std::vector<int64_t> sn_start;
  std::vector<int32_t> sn_size, sn_height;
  // block solve data (rebuilt with the factor): per supernode its dense diagonal block of L
  // (w x w, row-major, zeros above the diagonal, 1 / L_jj on it) and its transpose, at
  // sn_doff; per row the end of its off-block part in the CSR of L (forward) and the start of
  // its off-block part in the CSR of L^T (backward)
  std::vector<int64_t> sn_doff;
  std::vector<double> sn_D, sn_DT;
  std::vector<int64_t> f_off_end, b_off_beg;
  // the supernodes grouped by height over all components (the GPU solves one height of every
  // component per launch), and the split of their off-block sums over CTAs per direction
  std::vector<int32_t> gh_sn_ptr, gh_sn;
  ImexSplit fsplit, bsplit;
};
// Build the partition and the pattern (dt-independent part).
void imex_partition(const Setup& s, ImexData& d);
// Factor S = M^cc + beta_dt2 K^cc; returns false (with message) if S is not positive definite.
bool imex_factor(const Setup& s, double beta_dt2, ImexData& d, std::string& err);
// Host check of the GPU block solve's schedule for S = M^cc + beta_dt2 K^cc (the partition
// is copied and factored anew): supernode cover and size, topological ticket order, the
// work split's bounds, and both sweeps replayed over random asynchronous orders of ready
// supernodes (rows not yet final are NaN) against plain substitution.  Counts violations
// and returns the larger relative error of the two sweeps; false if S is not positive
// definite.
bool imex_check_schedule(const Setup& s, const ImexData& part, double beta_dt2, uint64_t seed,
                         int64_t& violations, double& rel_err, std::string& err);
// Solve M^cc a = b (b and a in c-index order) with a Cholesky factor of M^cc.
bool imex_mass_solve(const ImexData& d, const std::vector<double>& b, std::vector<double>& a,
                     std::string& err);

}  // namespace ibfem
