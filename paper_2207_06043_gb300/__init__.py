"""GB300-native coupled lattice-Boltzmann / dynamic-immersed-boundary solver.

The compute path is the CUDA library ``libibl.so`` (C ABI in ``include/ibl.h``),
reached through :mod:`paper_2207_06043_gb300.binding`.  ``geometry`` and
``meshes`` generate seeded inputs; ``workloads`` assembles the standard cases.
Importing this package does not load the CUDA library; the binding raises an
error when the library has not been built.
"""
