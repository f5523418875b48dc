// Face-shared ENO stage kernel, runs of 2 nodes, 80 registers (Tile.pair = 4).
#define LSP_RUN_R 2
#define LSP_RUN_MINB 3
#include "stage_run.inl"
