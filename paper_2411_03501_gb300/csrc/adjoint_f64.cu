// FP64 adjoint stage and loss kernels.
#define LSP_REAL double
#include "adjoint.inl"
