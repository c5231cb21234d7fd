/*
 * ibfem.h -- C ABI of the GB300 immersed-boundary explicit wave solver.
 *
 * The library advances the semi-discrete wave equation M Psi'' + K Psi = F (Sec. 2.2,
 * Eq. semi of Buerchner et al., arXiv 2501.19013) on a uniform Cartesian grid of
 * tensor-product GLL spectral elements of order p, where cells cut by the immersed
 * boundary carry the finite cell indicator alpha^FCM (Eq. weak_form_extended).  One
 * time step of the explicit scheme is the central-difference update (Eq. cdm)
 *
 *     u^{k+1} = 2 u^k - u^{k-1} + dt^2 M_L^{-1} (F^k - K u^k),
 *
 * with K applied element by element on the GPU (no global matrix) and M_L the lumped
 * mass.  The semi-explicit variant is the Newmark IMEX scheme of Algorithm 2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status: IBFEM_OK (0) or a negative IBFEM_ERR_* code.
 *    On error a human-readable message is available from ibfem_last_error() (per
 *    thread) and the handle stays valid unless stated otherwise.
 *  - Host arrays passed in are copied before the call returns; the caller keeps
 *    ownership.  Output arrays are caller-allocated host memory of the stated size.
 *  - Vectors in the ABI ("kept-DOF order") are indexed by the kept DOFs: the global node
 *    lattice has (n_k p + 1) nodes per axis, numbered lexicographically with x fastest;
 *    nodes that belong to at least one kept (not entirely fictitious) cell are numbered
 *    in lattice order; the ncomp components of a node are consecutive.
 *  - Device memory belongs to the handle.  It is obtained through options->dev_alloc
 *    (e.g. the PyTorch caching allocator) when given, else cudaMalloc.
 *  - ibfem_step only enqueues work on the handle's stream; ibfem_sample, ibfem_get_state,
 *    ibfem_crit_dt, ibfem_sync and the other "read" calls synchronise that stream.
 *  - Handles are not thread-safe; distinct handles may be used from distinct threads.
 *  - Every call that works on the device also returns ARG for a null handle, STATE for
 *    a host_only handle or a batch member (ibfem_info and ibfem_destroy excepted), CUDA
 *    when a CUDA call fails and OOM when an allocation fails; the per-function "Errors"
 *    lists add what is particular to the call.
 *  - Entry points marked "library" (lifetime, diagnostics, timing, batching, tile shape,
 *    deferred upload) serve the GPU runtime; the paper, a one-process CPU study, has no
 *    counterpart for them.
 */
#ifndef IBFEM_H
#define IBFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define IBFEM_OK 0
#define IBFEM_ERR_ARG (-1)       /* invalid argument or unsupported combination        */
#define IBFEM_ERR_OOM (-2)       /* device or host allocation failed                   */
#define IBFEM_ERR_CUDA (-3)      /* a CUDA runtime call failed                         */
#define IBFEM_ERR_DIVERGED (-4)  /* a non-finite value appeared in the state           */
#define IBFEM_ERR_TIMEOUT (-5)   /* a bounded device wait gave up                      */
#define IBFEM_ERR_GEOMETRY (-6)  /* geometry leaves no kept cell / point not in domain */
#define IBFEM_ERR_EIG (-7)       /* a host eigen/Cholesky factorisation failed         */
#define IBFEM_ERR_STATE (-8)     /* call order (e.g. step before set_dt)               */

/* ---- enumerations ---------------------------------------------------------------- */
enum { IBFEM_GEOM_NONE = 0,     /* no immersed boundary: every cell is uncut            */
       IBFEM_GEOM_HOLES = 1,    /* circles (2D) / spheres (3D) of fictitious material   */
       IBFEM_GEOM_VOXELS = 2,   /* voxel image, 1 = void (fictitious), 0 = solid        */
       IBFEM_GEOM_ROTATED_BOX = 3 /* physical domain = rotated cube (Sec. 3.1)          */ };
enum { IBFEM_STAB_NONE = 0, IBFEM_STAB_EVS = 1, IBFEM_STAB_MASS_SCALING = 2 };
enum { IBFEM_SCALAR = 0, IBFEM_ELASTIC_PLANE_STRAIN = 1 };
/* Time integration: IBFEM_CDM, Eq. cdm with the lumped mass; IBFEM_IMEX, Algorithm 2
 * (Newmark beta = 1/4, gamma = 1/2 on the DOFs of cut cells, CDM on the rest);
 * IBFEM_CDM_CONSISTENT, the central-difference method with the consistent mass of the cut
 * cells (the paper's "SCM con." CDM): Algorithm 2 with beta = 0, i.e. the DOFs of cut cells
 * are advanced explicitly through a solve with their consistent (EVS-stabilised when
 * eps > 0) mass block M^cc.  IMEX and the consistent-mass CDM take precision IBFEM_FP64,
 * IBFEM_EXACT64_TC or IBFEM_EXACT_TC (the explicit part on that kernel; the solves are
 * FP64); ibfem_create returns IBFEM_ERR_ARG for the others. */
enum { IBFEM_CDM = 0, IBFEM_IMEX = 1, IBFEM_CDM_CONSISTENT = 2 };
/* Precision of the element contractions.  The integrator state (u^k, u^{k-1}), the
 * central-difference update, the IMEX solves and the power iteration are FP64 always. */
enum { IBFEM_FP64 = 0,          /* FP64 contractions on the CUDA cores                      */
       IBFEM_EXACT_TC = 1,      /* tcgen05 kind::f16, balanced 8-bit digit slices of u and
                                   K_ref (BF16) accumulated exactly per level (10 MMA chains),
                                   level 0 summed error-free: about 32 significant bits      */
       IBFEM_BF16X3_TC = 2,     /* tcgen05 kind::f16, BF16 hi/lo splits, 3 passes, FP32 acc. */
       IBFEM_BF16_TC = 3,       /* tcgen05 kind::f16, one BF16 pass, FP32 accumulation      */
       IBFEM_EXACT64_TC = 4     /* FP64-grade: tcgen05 kind::f16, seven balanced 8-bit digit
                                   slices of u and K_ref (one exponent for K_ref), all levels
                                   s + t <= 6 (28 MMA chains) exact, integer node sums, K u
                                   rounded once in FP64; cut cells by the FP64 cut kernel    */ };
enum { IBFEM_SRC_NONE = 0,
       IBFEM_SRC_POINT = 1,          /* params: x, y[, z] [, dir_x, dir_y] (elastic)   */
       IBFEM_SRC_EDGE_TRACTION = 2,  /* params: y0, y1, t_x[, t_y]; edge x = lo_x (2D) */
       IBFEM_SRC_GAUSS = 3           /* params: x_l[dim], sigma (volumetric Gaussian)  */ };

/* ---- structures ------------------------------------------------------------------ */
typedef struct ibfem_s ibfem_t;

typedef struct {
    int dim;          /* 2 or 3                                                        */
    int n[3];         /* cells per axis (n[2] ignored in 2D)                           */
    double lo[3];     /* extended-domain box                                           */
    double hi[3];
} ibfem_grid;

typedef struct {
    int kind;                 /* IBFEM_GEOM_*                                          */
    int count;                /* HOLES: number of circles/spheres                      */
    const double* shapes;     /* HOLES: count x (cx, cy[, cz], r);
                                 ROTATED_BOX: (edge, cx, cy, cz, T00..T22 row-major),
                                 T maps the cube frame to global axes (x = c + T x')   */
    const uint8_t* voxels;    /* VOXELS: vn[0]*vn[1]*vn[2] bytes, x fastest, 1 = void  */
    int vn[3];                /* VOXELS: voxels per axis spanning [lo, hi]             */
    int quad_depth;           /* space-tree depth for cut cells (>= 0)                 */
} ibfem_geometry;

typedef struct {
    int kind;                 /* IBFEM_STAB_*                                          */
    double eps;               /* EVS: epsilon of Eq. epsilon_stabilization             */
    double f_lambda;          /* EVS: small-eigenvalue threshold fraction              */
} ibfem_stab;

typedef struct {
    int physics;              /* IBFEM_SCALAR or IBFEM_ELASTIC_PLANE_STRAIN (2D only)  */
    double rho, c;            /* density, wave speed (scalar)                          */
    double E, nu;             /* Young's modulus, Poisson ratio (elastic)              */
    int scheme;               /* IBFEM_CDM, IBFEM_IMEX or IBFEM_CDM_CONSISTENT         */
    int precision;            /* IBFEM_FP64 / _EXACT_TC / _BF16X3_TC / _BF16_TC / _EXACT64_TC */
    void* stream;             /* cudaStream_t to run on, NULL = the legacy stream      */
    void* (*dev_alloc)(size_t bytes, void* ctx);  /* optional device allocator         */
    void (*dev_free)(void* ptr, void* ctx);
    void* alloc_ctx;
    int device;               /* CUDA device ordinal, made current inside every call   */
    int host_only;            /* 1: build the host discretisation only (no device use);
                                 only ibfem_info/get_lumped_mass/get_cut_cells/
                                 get_element are then valid -- for checks without a GPU */
} ibfem_options;

typedef struct {
    int64_t n_dof;            /* kept DOFs                                             */
    int64_t n_lattice_dof;    /* DOFs of the full node lattice (device layout)         */
    int64_t n_elem, n_uncut, n_cut, n_outside;
    int64_t n_c;              /* IMEX: DOFs treated implicitly (0 for CDM)             */
    int64_t nnz_L;            /* IMEX: nonzeros of the Cholesky factor                 */
    int32_t n_levels;         /* IMEX: heights of the nested-dissection tree, the
                                 longest chain of waits in one triangular sweep       */
    int32_t n_loc;            /* DOFs per element                                      */
    int32_t ncomp;
    int32_t precision;
    int64_t step;             /* steps taken since set_initial / set_state             */
    double t, dt;
    double lambda_ref;        /* lambda_max(K_ref, M_ref) of one uncut cell            */
    size_t device_bytes;      /* device memory held by the handle; for a host_only
                                 handle the bytes ibfem_upload would allocate            */
    int64_t n_cut_matrices;   /* distinct cut-cell matrix sets: equal to n_cut, or fewer
                                 for voxel images with whole voxels per cell, where cut
                                 cells with equal voxel blocks share one set             */
    int32_t tile_variant;     /* tensor-core tile shape in use (0 full, 1 small)       */
    int32_t tile[3];          /* cells per tile and axis of the tensor-core kernel     */
    size_t shared_device_bytes; /* part of device_bytes held jointly with the handle's
                                 clones (or its source): geometry, cut-cell and
                                 reference matrices; freed with the last of them          */
    int32_t tc_ctas_per_sm;   /* cap on the exact kernel's resident CTAs per SM (0: as
                                 many as fit), set by ibfem_autotune                     */
    int32_t autotune_cached;  /* 1 if the last ibfem_autotune reused a cached choice     */
} ibfem_info_t;

/* ---- lifetime -------------------------------------------------------------------- */

/* Build the discretisation (Sec. 2.2-2.6) on the host and upload it.
 *  grid, p (1..6), geometry (NULL = none), alpha (indicator value in the fictitious
 *  domain, Eq. weak_form_extended), stab (NULL = none), opt (NULL = scalar, rho = c = 1,
 *  CDM, FP64, default stream and allocator).  *out receives the new handle.
 *  Errors: ARG (bad sizes/combination), GEOMETRY (no kept cell), EIG (a cut-cell
 *  eigenproblem or the IMEX factorisation failed), OOM, CUDA.                          */
int ibfem_create(const ibfem_grid* grid, int p, const ibfem_geometry* geometry,
                 double alpha, const ibfem_stab* stab, const ibfem_options* opt,
                 ibfem_t** out);
/* Library.  Several loads on one discretisation (shared-geometry multi-source runs).  *out
 * receives a new handle on the same grid, geometry, material, scheme, precision and
 * tile shape as `src`, whose device geometry, cut-cell matrices, reference stiffness
 * and tensor-core K_ref image it shares instead of holding a copy; it owns its state,
 * load, observers, counters and dt^2 / M_L.  The clone starts at rest with no load and
 * no observers, with src's dt if src has one (set_dt on either changes only that
 * handle).  Each handle keeps the shared arrays alive: `src` may be destroyed first.
 * A clone steps alone or as a member of a batch like any handle, and gives the results
 * of a handle created from scratch on the same inputs, bit for bit.  `src` may be a
 * batch member (nothing of its state is read).
 * Errors: ARG (null argument; src solves a c-set, i.e. IMEX or the consistent-mass CDM
 * with cut cells), STATE (src is host_only), OOM, CUDA.                               */
int ibfem_clone(ibfem_t* src, ibfem_t** out);
/* Library.  Free every resource of the handle (NULL is accepted; waits for the handle's
 * queued work, and for its batch's if it is a member).  Arrays shared with clones are
 * freed with the last handle that uses them.  Always returns IBFEM_OK.                 */
int ibfem_destroy(ibfem_t* h);
/* Library.  Message of the last failed call on this thread ("" if none).  Valid until
 * the next failing call on the same thread.                                             */
const char* ibfem_last_error(void);
/* Library.  Fill *out with the handle's sizes, counts, step, time and device footprint
 * (the fields of ibfem_info_t).  Host data only: no synchronisation, valid for host_only
 * handles and batch members.  Errors: ARG (null h or out).                              */
int ibfem_info(const ibfem_t* h, ibfem_info_t* out);

/* ---- problem data ---------------------------------------------------------------- */

/* Load F^k = F_s * f_t(t_k) with the Ricker wavelet of Eq. source_time (centre
 * frequency f_e).  kind/params as in IBFEM_SRC_*.  A point source contributes
 * alpha^FCM(x_s) rho N_i(x_s) (times the direction for elasticity); an edge traction
 * contributes the boundary integral of alpha^FCM N_i t; the Gaussian load of the
 * benchmark (Sec. 3.1) contributes int alpha^FCM rho f_s N_i over the kept cells with
 * f_s = exp(-|x - x_l|^2 / (2 sigma^2)) (Eq. weak_form_extended, load term), integrated on
 * cells within 8 sigma of x_l split into ceil(h / sigma)^dim subcells with (p + 4)^dim
 * Gauss-Legendre points each.  Errors: ARG, GEOMETRY.                                   */
int ibfem_set_source(ibfem_t* h, int kind, const double* params, int nparams, double f_e);

/* Observer points (Sec. 3.2): npts x dim coordinates.  Each step records
 * Psi(x_i, t_k) = sum_j N_j(x_i) u_j^k (all components) into a device ring of
 * `capacity` rows; ibfem_sample returns them.  Resets the ring.  Errors: ARG, GEOMETRY. */
int ibfem_set_observers(ibfem_t* h, int npts, const double* xyz, int64_t capacity);

/* Initial state Psi_0, Psi'_0 (host, kept-DOF order, n_dof each; NULL = zero).  The
 * start-up value u^{-1} = u^0 - dt v^0 + dt^2/2 M_L^{-1}(F^0 - K u^0) is formed on the
 * device: the initialisation of Algorithm 1 with beta = 0 (the paper leaves the CDM
 * start-up open); IMEX: its d-part, plus Psi''_0 = (M^cc)^{-1}(F^c_0 - K^c u_0) on the
 * c-part (Algorithm 2 initialisation).  Resets the step count and the observer ring.
 * Errors: STATE (set_dt not called).                                                    */
int ibfem_set_initial(ibfem_t* h, const double* u0, const double* v0);

/* Critical step dt_crit = 2 / sqrt(lambda_max(K, M_L)) (Sec. 2.3) by power iteration on
 * M_L^{-1/2} K M_L^{-1/2}: start v_i = 1 + 0.5 sin(i) over kept DOFs, stop when
 * |lambda_k - lambda_{k-1}| <= rtol lambda_k or after max_iter products.  For IMEX the
 * iteration runs on the explicit (d) block.  Any of the outputs may be NULL.           */
int ibfem_crit_dt(ibfem_t* h, int max_iter, double rtol, double* dt_crit,
                  double* lambda_max, int* iterations);

/* Set the step size dt of Eq. cdm (> 0, finite).  Rescales dt^2 M_L^{-1} on the device
 * and, for IMEX, refactors S = M^cc + beta dt^2 K^cc (Algorithm 2, beta = 1/4) on the
 * host.  Errors: ARG (dt not positive), EIG (factorisation failed).                     */
int ibfem_set_dt(ibfem_t* h, double dt);

/* ---- time stepping --------------------------------------------------------------- */

/* Enqueue n time steps (n >= 0) on the handle's stream: Eq. cdm (IBFEM_CDM), Algorithm 2
 * (IBFEM_IMEX) or Algorithm 2 with beta = 0 (IBFEM_CDM_CONSISTENT), replaying a captured
 * CUDA graph of the per-step kernels.  Asynchronous: divergence and device timeouts are
 * reported by the next synchronising call.  Errors: ARG (n < 0), STATE (no initial state:
 * call set_initial or set_state first).                                                  */
int ibfem_step(ibfem_t* h, int64_t n);

/* Same as ibfem_step, but every kernel is launched directly with a pair of CUDA events
 * around it on the handle's stream (no graph).  When flush_bytes > 0, flush_buf (device
 * memory of at least flush_bytes; each half larger than the L2 cache) evicts the L2 cache
 * before every step, outside the timed events: its first half is overwritten with
 * cudaMemsetAsync and its second half is then read by a kernel, so that the write-back of
 * the dirty lines (the memset's and the previous step's) happens before the step and the
 * step starts with the cache holding clean lines of unrelated data.  ms[0] accumulates the device time of
 * whole steps (first kernel start to last kernel end), ms[1 + k] that of kernel k (at most
 * max_slots values; names from ibfem_kernel_name); *n_slots receives the slot count.
 * Synchronises.  Library: meant for benchmarks and profiles.
 * Errors: ARG (n < 0, null ms with max_slots > 0, null flush_buf with flush_bytes > 0),
 * STATE (no initial state).                                                             */
int ibfem_step_timed(ibfem_t* h, int64_t n, void* flush_buf, size_t flush_bytes, double* ms,
                     int max_slots, int* n_slots);
/* Library.  Name of kernel slot `slot` of ibfem_step_timed ("" if out of range or for a
 * null handle); the string lives as long as the library.                               */
const char* ibfem_kernel_name(const ibfem_t* h, int slot);

/* Library.  Synchronise the stream; report a tensor-core kernel whose bounded wait (an
 * mbarrier of the MMA or of the K_ref copy) gave up as IBFEM_ERR_TIMEOUT, and a non-finite
 * state (a run beyond the stability limit of Sec. 2.3) as IBFEM_ERR_DIVERGED.  The flags
 * stay set (the state is no longer trustworthy).                                        */
int ibfem_sync(ibfem_t* h);

/* Observer series (Sec. 3.2) recorded since set_observers/set_initial, oldest first: up
 * to max_rows rows of npts*ncomp doubles (row r = time t_{k0+r}).  The last row is the
 * current state Psi(t_k).  *rows receives the count.  Synchronises.
 * Errors: ARG (null out or rows, max_rows < 0), DIVERGED, TIMEOUT (as ibfem_sync).     */
int ibfem_sample(ibfem_t* h, int64_t max_rows, double* out, int64_t* rows);

/* State of the integrator (host, kept-DOF order, n_dof each; either pointer may be NULL).
 * Synchronises.  CDM (Eq. cdm): u = u^k, u_prev = u^{k-1}.  IMEX (Algorithm 2): u_prev
 * holds u^{k-1} on d and Psi'^k on c.                                                    */
int ibfem_get_state(ibfem_t* h, double* u, double* u_prev);
/* Restore a state previously read by ibfem_get_state (the pair of Eq. cdm, or of
 * Algorithm 2 for IMEX) together with its step index (the load f_t(t_k) of the next step
 * follows from it).  Continuing from it is bitwise equal
 * to not having stopped.  Errors: ARG (null u or u_prev, step < 0), STATE (no dt).       */
int ibfem_set_state(ibfem_t* h, const double* u, const double* u_prev, int64_t step);

/* ---- inspection (used by the parity tests) ---------------------------------------- */

/* y = K x (K of Eq. semi, applied element by element: the shared reference matrix in
 * uncut cells, the space-tree integrated K^e in cut cells, Sec. 2.2), x and y host
 * vectors in kept-DOF order.  Synchronises.  Errors: ARG (null x or y).                   */
int ibfem_apply_operator(ibfem_t* h, const double* x, double* y);
/* Assembled lumped mass diagonal M_L of Eq. cdm (Sec. 2.4: GLL in uncut cells, HRZ
 * diagonal scaling of the (stabilised) cut-cell mass), kept-DOF order, n_dof doubles.
 * Host data.  Errors: ARG (null argument).                                               */
int ibfem_get_lumped_mass(ibfem_t* h, double* ml);
/* Flat indices (x fastest) of the cut cells (Sec. 2.2: cells the immersed boundary
 * crosses), n_cut int64 values in ascending order.  Host data.  Errors: ARG (null).      */
int ibfem_get_cut_cells(ibfem_t* h, int64_t* cells);
/* Element stiffness (n_loc x n_loc, row-major) used for cell `cell`: the shared reference
 * matrix for uncut cells, the alpha^FCM-weighted space-tree integral for cut cells (Sec.
 * 2.2, Eq. weak_form_extended); optional lumped diagonal (n_loc, Sec. 2.4).  Host data.
 * Errors: ARG (cell outside or out of range).                                            */
int ibfem_get_element(ibfem_t* h, int64_t cell, double* K, double* ml);
/* Consistent element mass (n_loc x n_loc, row-major) of cell `cell` as the consistent-mass
 * schemes use it: for a cut cell the alpha-integrated space-tree mass M^o (Sec. 2.2), plus
 * eps M^s under eigenvalue stabilisation (Eq. epsilon_stabilization); for an uncut cell
 * the GLL-quadrature mass, which is diagonal (Sec. 2.4).  Host data only (valid for
 * host_only handles).  Errors: ARG (null M, cell outside or out of range), STATE (a cut
 * cell of a handle with scheme IBFEM_CDM, which keeps only the lumped cut masses).       */
int ibfem_get_element_mass(ibfem_t* h, int64_t cell, double* M);

/* ---- tile shape -------------------------------------------------------------------- */

/* The exact tensor-core kernel exists with two tile shapes: variant 0 fills the 128 rows
 * of one MMA with the halo'd tile (2D: 8x8 cells for n_loc >= 32, else 15x7; 3D: 4x4x4),
 * variant 1 is smaller (2D: 5x5 or 7x7; 3D: 3x3x3): more tiles for small problems and, in
 * 3D, less shared memory per CTA.  ibfem_set_tile_variant picks one; ibfem_autotune times
 * reps operator applications (the state is untouched) for each tile shape and each cap on
 * the persistent launch's resident CTAs per SM (as many as fit, or one), keeps the fastest
 * pair, and returns its tile shape and the best time of each shape (ms per application) in
 * ms[2].  The choice is cached per (device, dim, p, ncomp, log2 of the cell count) for the
 * life of the process: a later handle of the same class takes it without timing
 * (ibfem_info reports the cap and whether the cache answered).  The FP64 path and the BF16
 * schemes have variant 0 only (ibfem_autotune then returns 0 and zero times); the
 * FP64-grade path has one tile shape (returned, zero times).
 * Results of the two variants agree within the exact scheme's accuracy (the digit
 * exponent is per tile), not bitwise.  This is a part of this library; the paper has no
 * counterpart.  Errors: ARG, STATE (batch member), CUDA.                                  */
int ibfem_set_tile_variant(ibfem_t* h, int variant);
int ibfem_autotune(ibfem_t* h, int reps, int* variant, double* ms);

/* ---- deferred upload ----------------------------------------------------------------- */

/* Move a handle created with host_only = 1 onto its device: the buffers, the K_ref image
 * and the tables that ibfem_create uploads for a device handle (its options are those given
 * at creation).  Before the call, ibfem_info(h).device_bytes is the number of bytes this
 * call allocates (sources, observers and the IMEX factor come on top), so a caller can
 * admit work by device-memory footprint before any allocation happens.  This is a part of
 * this library; the paper has no counterpart.
 * Errors: STATE (not host_only), ARG (no kernel for the shape/precision), OOM, CUDA; on an
 * error the handle stays host_only and holds no device memory.                          */
int ibfem_upload(ibfem_t* h);

/* ---- batched stepping (continuous batching) ------------------------------------------ */

/* A batch advances many independent handles together: per shape class (dim, p, ncomp)
 * one persistent tensor-core launch per time step covers the tiles of every member, the
 * classes run concurrently, and chunks of 32 steps are replayed as CUDA graphs.  Members
 * join and leave between chunks.  Each member performs exactly the arithmetic of
 * ibfem_step on its own (same kernel code per tile, Eq. cdm), so its results do not depend
 * on the other members.  This is a part of this library; the paper has no counterpart.
 *
 * Members must be device handles with precision IBFEM_EXACT_TC and scheme IBFEM_CDM, with
 * dt and the initial state set.  While a handle is a member, every other call on it returns
 * IBFEM_ERR_STATE, except ibfem_info and ibfem_destroy (which first waits for the batch's
 * queued work and takes the handle out).  A batch is used from one thread at a time.     */
typedef struct ibfem_batch_s ibfem_batch_t;

/* New empty batch on `device`; `stream` (cudaStream_t, NULL = a private stream) carries
 * its work.  Errors: ARG (null out), CUDA.                                              */
int ibfem_batch_create(void* stream, int device, ibfem_batch_t** out);

/* Admit handle h for n_steps (>= 1) more steps.  The batch's work starts after everything
 * already queued on h's stream.  The K_ref image is shared with members whose image is
 * byte-identical.  Errors: ARG (wrong precision/scheme/device, n_steps < 1), STATE (host_only,
 * not initialised, already a member), CUDA.                                               */
int ibfem_batch_add(ibfem_batch_t* b, ibfem_t* h, int64_t n_steps);

/* Enqueue n batched steps (asynchronous).  A member whose budget runs out inside the n
 * steps stops there exactly (its tiles are skipped afterwards) and becomes "finished":
 * it leaves the batch, and its own stream is ordered after the batch work queued so far,
 * so that ibfem_sample / get_state on it see its final state.  Errors: ARG (null batch,
 * n < 0), CUDA.                                                                         */
int ibfem_batch_run(ibfem_batch_t* b, int64_t n);

/* Hand back up to max_done finished handles (in completion order) in done[]; *n_done
 * receives their count.  The handles are ordinary handles again (the caller owns them).
 * Errors: ARG (null b or n_done, or null done with max_done > 0).                         */
int ibfem_batch_poll(ibfem_batch_t* b, ibfem_t** done, int max_done, int* n_done);

/* Members still stepping, finished members not yet polled, batched steps enqueued (any
 * output may be NULL).  Errors: ARG (null batch).                                        */
int ibfem_batch_status(const ibfem_batch_t* b, int* n_active, int* n_finished, int64_t* steps_enqueued);

/* Block until at most max_pending enqueued chunks (ibfem_batch_run calls are split into
 * chunks of up to 32 steps) are still unfinished on the GPU: the back-pressure of a
 * serving loop, so that new members are not queued behind a long backlog.  Errors: ARG, CUDA. */
int ibfem_batch_wait(ibfem_batch_t* b, int max_pending);

/* Wait for the batch's queued work.  Errors: CUDA.                                       */
int ibfem_batch_sync(ibfem_batch_t* b);

/* Wait for the queued work, release members still in the batch (at the step their device
 * counter reached) and free the batch (NULL is accepted).  Always returns IBFEM_OK.       */
int ibfem_batch_destroy(ibfem_batch_t* b);

/* ---- failure detection ---------------------------------------------------------------- */

/* Library runtime diagnostic (the paper has no counterpart): enqueues on the handle's stream
 * one wait of the kind the tensor-core kernel uses for its MMA completions, on an mbarrier
 * that nothing arrives on (no MMA or copy in flight), limited to `polls` try_wait calls.
 * The wait runs out, records the timeout in the handle's device flag word and returns, so
 * the next ibfem_sync / ibfem_sample returns IBFEM_ERR_TIMEOUT while the CUDA context stays
 * usable; ibfem_set_initial / ibfem_set_state clear the record.  Asynchronous.
 * Errors: ARG (polls outside [1, 2^24]), STATE (host-only handle), CUDA (launch). */
int ibfem_check_bounded_wait(ibfem_t* h, int polls);

/* Host check of the schedule of the GPU's block triangular solves (the c-set solve of
 * Algorithm 2, Sec. 2.6, and of the consistent-mass CDM): factors S = M^cc + beta_dt2 K^cc
 * on the host (a copy; the handle's factor is untouched) and checks what the GPU sweeps
 * rely on: supernodes that cover the rows in order with at most 32 rows each, ticket
 * orders that are topological for the waits (edges of the elimination tree between
 * supernodes), partial-sum slots in range and at most 8 entries per thread; then it replays
 * the forward (L y = b) and the backward (L^T x = y) sweep over random asynchronous orders
 * of ready supernodes, rows not yet final set to NaN, against plain substitution, for a
 * right-hand side drawn from `seed`.  Runs on the host only (host_only handles too).
 *   violations  out: broken invariants plus reads of rows not yet final (0 when sound)
 *   rel_err     out: the larger relative L2 error of the two sweeps against substitution
 * Errors: ARG (null pointers, beta_dt2 < 0, S not positive definite), STATE (a handle
 * without a c-set: scheme IBFEM_CDM, or no cut cells). */
int ibfem_check_solve_schedule(ibfem_t* h, double beta_dt2, uint64_t seed, int64_t* violations,
                               double* rel_err);

/* ---- allocation-free operator ----------------------------------------------------- */

/* y = K x on the node lattice, for callers that cannot allocate device memory: an
 * application whose own fixed pool or arena owns the GPU memory, or a latency-critical
 * loop where cudaMalloc/cudaFree (which may synchronise the device) are off-limits.  This
 * is an addition of this library; the paper has no counterpart.
 *
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library routine).  Its
 * only scratch, the products K^e x_e of the cut cells, lives in a static device array of
 * 2^19 doubles (4 MiB) that every GPU loading the library holds until the process exits.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress,
 * with the device current) and keeps it for the life of the process; make that first call
 * before any stream capture, and do not call this entry point after cudaDeviceReset (or
 * anything else that unloads the module), since the kept address would then be stale.  All calls
 * share the array and it keeps the last call's contents; every entry a call reads is
 * written by the same call first, so nothing needs clearing.  Calls whose kernels overlap
 * on the GPU (different streams, or different threads) race on the array: serialise them.
 *
 * Arguments (all pointers are device memory owned by the caller, read-only except y):
 *   dim, p, ncomp   2 or 3; GLL order; 1 (scalar) or 2 (plane strain, dim 2)
 *   n_cells[dim]    cells per axis; the lattice has n_cells[k] p + 1 nodes per axis
 *   cell_class      one byte per cell, x fastest: 0 outside, 1 cut, 2 uncut
 *   cut_index       int32 per cell: index into the cut list, -1 if not cut
 *   cut_cells       n_cut int64: cell of each cut index
 *   K_ref           n_loc x n_loc reference stiffness of an uncut cell (n_loc = (p+1)^dim ncomp)
 *   K_cut           n_cut x n_loc x n_loc stiffness of the cut cells (symmetric, row-major)
 *   x, y            lattice vectors, node-major with ncomp interleaved; y is overwritten
 *   stream          cudaStream_t (NULL = legacy stream); the call only enqueues work
 * Errors: IBFEM_ERR_ARG for a null pointer, an unsupported (dim, p, ncomp) or
 * n_cut * n_loc above 2^19 (message names the sizes); IBFEM_ERR_CUDA for a launch error. */
int ibfem_apply_operator_noalloc(int dim, int p, int ncomp, const int n_cells[3],
                                 const uint8_t* cell_class, const int32_t* cut_index,
                                 const int64_t* cut_cells, int64_t n_cut,
                                 const double* K_ref, const double* K_cut,
                                 const double* x, double* y, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IBFEM_H */
