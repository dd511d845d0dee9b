"""GB300-native systolic Yee FDTD (arxiv 2502.20610).

The compute path is the CUDA library libfdtd.so (C ABI, include/fdtd.h);
`fdtd` is its thin ctypes binding and `workloads` the seeded input
generators.  Importing the package does not load the library; creating a
simulation does, and fails loudly if it is missing.
"""
