"""FP64 CPU oracle for the immersed-boundary (finite/spectral cell) explicit wave solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.  It
shares no code with the CUDA library (``paper_2501_19013_gb300``); both are fed the same
seeded inputs from ``paper_2501_19013_gb300.workloads``, which holds no solver arithmetic.

The oracle is a plain, slow, readable restatement of Buerchner et al., "On the efficiency
of explicit and semi-explicit immersed boundary finite element methods for wave
propagation problems" (arXiv 2501.19013).  Every function cites the section or equation
it follows.  The global stiffness is *assembled* as a sparse matrix (the paper's own
"global matrix times vector" formulation, Sec. 3 computation times), whereas the CUDA
path applies K element by element without any global matrix.

Modules
-------
basis        GLL / Gauss-Legendre points, 1D Lagrange polynomials (Sec. 2.2)
geometry     cell classification against holes, voxels, a rotated box (Sec. 2.2, 3.1)
quadrature   space-tree (quadtree/octree) quadrature of cut cells (Sec. 1, 2.2)
elements     element stiffness and mass matrices with alpha^FCM (Eq. weak_form_extended)
stabilization eigenvalue stabilisation, HRZ lumping, mass scaling (Sec. 2.4, 2.5)
discretization DOF numbering, global assembly, loads, observers
integrators  CDM (Eq. cdm), Newmark (Algorithm 1), Newmark IMEX (Algorithm 2)
eigen        critical time step (Sec. 2.3): dense and power-iteration lambda_max

Parity pins are listed per function; functions without an independent pin say so.
"""
