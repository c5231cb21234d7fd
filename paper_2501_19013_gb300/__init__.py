"""GB300 (sm_103a) implementation of the explicit / semi-explicit immersed-boundary
(finite / spectral cell) wave solver hot path: the central-difference step with an
element-by-element operator, its IMEX variant and the critical-time-step iteration.

The compute path is the CUDA library ``libibfem.so`` (C ABI in ``include/ibfem.h``);
``paper_2501_19013_gb300.ibfem`` is its ctypes binding and loads the library on first
use (ImportError if it has not been built -- there is no fallback).
``workloads`` generates the seeded synthetic inputs.
"""
