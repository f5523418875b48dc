// FP32 tiled stage kernels, 4 CTAs of 256 threads per SM.
#define LSP_MINB 4
#include "stage_tiled.inl"
