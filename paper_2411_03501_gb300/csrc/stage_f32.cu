// FP32 instantiations of the generic stage kernels.
#define LSP_REAL float
#include "dispatch.inl"
