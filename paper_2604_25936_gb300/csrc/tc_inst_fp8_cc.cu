// Tensor-core T-MLP kernel instantiations: FP8 e4m3 operands, SAND queries on raw coordinates with the
// exit-layer-1 rows on two CUDA-core warps.
#define SAND_INST_MODE TC_FP8
#define SAND_INST_VAR 3
#include "tc_inst_body.cuh"
