// Face-shared ENO stage kernel, runs of 4 nodes, 128 registers (Tile.pair = 3).
#define LSP_RUN_R 4
#define LSP_RUN_MINB 2
#include "stage_run.inl"
