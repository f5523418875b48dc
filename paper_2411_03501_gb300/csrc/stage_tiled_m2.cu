// FP32 tiled stage kernels, 2 CTAs of 256 threads per SM.
#define LSP_MINB 2
#include "stage_tiled.inl"
