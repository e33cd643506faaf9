"""GB300-native IPComp: interpolation-based progressive lossy compression
(arXiv 2502.04093) as sm_103a CUDA kernels behind a C ABI (include/ipc.h).

``ipc`` is the ctypes binding of libipcomp.so; ``build`` compiles it;
``synth`` draws the seeded synthetic workloads.
"""
