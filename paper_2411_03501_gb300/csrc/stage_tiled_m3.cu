// FP32 tiled stage kernels, 3 CTAs of 256 threads per SM.
#define LSP_MINB 3
#include "stage_tiled.inl"
