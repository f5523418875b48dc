// FP32 adjoint stage and loss kernels.
#define LSP_REAL float
#include "adjoint.inl"
