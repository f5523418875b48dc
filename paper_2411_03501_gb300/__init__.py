"""GB300-native explicit Hamilton-Jacobi level-set integrator (LevelSetPy,
arXiv 2411.03501): fused sm_103a CUDA stage kernels behind a C ABI
(``include/lsp.h``), with a thin ctypes binding (``binding``).

Submodules: ``binding`` (the C ABI, loaded on first call; there is no CPU
fallback), ``workloads`` (seeded synthetic inputs), ``build`` (nvcc build).
"""
