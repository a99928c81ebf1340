"""GB300-native (sm_103a) RKL2 super-time-stepping and BE+PCG solves of frozen-coefficient
parabolic operators on spherical grids (Caplan, Mikic, Linker & Lionello, arXiv:1610.01265).

The compute path is the C-ABI library built from ``csrc/`` (see ``include/rklpcg.h``);
this package holds its thin ctypes binding and the seeded synthetic-input generator.
"""
