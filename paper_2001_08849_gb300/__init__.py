"""GB300-native FS-FEM-T4: smoothed stiffness operator, CSR assembly and
Jacobi-PCG / mixed-precision solves in sm_103a CUDA behind a C ABI
(include/sfem.h, lib/libsfem.so).

`paper_2001_08849_gb300.sfem` is the ctypes binding; importing it requires
the built library (see `paper_2001_08849_gb300.build`).
"""
