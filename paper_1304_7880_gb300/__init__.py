"""WDLB on GB300: the per-timestep Weighted Density Lattice Boltzmann update
(Marini Bettolo Marconi & Melchionna, arXiv:1304.7880) as hand-written sm_103a
CUDA kernels behind a C ABI (``include/wdlb.h``).

Submodules:
  ``wdlb``   ctypes binding of the C ABI (argument marshalling only).
  ``build``  compiles ``csrc/`` into the in-tree ``_build/libwdlb.so``.
  ``synth``  seeded synthetic inputs (no method arithmetic).
"""
