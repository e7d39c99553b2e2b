// Tensor-core T-MLP kernel instantiations: fp16 operands, SAND queries on raw coordinates with the
// exit-layer-1 rows on two CUDA-core warps.
#define SAND_INST_MODE TC_F16
#define SAND_INST_VAR 3
#include "tc_inst_body.cuh"
