// FP64 instantiations of the generic stage kernels.
#define LSP_REAL double
#include "dispatch.inl"
