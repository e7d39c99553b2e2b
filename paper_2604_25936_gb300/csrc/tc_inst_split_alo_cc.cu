// Tensor-core T-MLP kernel instantiations: the float32 mode at width 336 with A_lo in shared memory, SAND query with CUDA core warps variant.
#define SAND_INST_MODE TC_SPLIT16
#define SAND_INST_VAR 7
#include "tc_inst_body.cuh"
