// Tensor-core T-MLP kernel instantiations: the float32 mode (3 x fp16 split), SAND queries on raw coordinates with the
// exit-layer-1 rows on two CUDA-core warps.
#define SAND_INST_MODE TC_SPLIT16
#define SAND_INST_VAR 3
#include "tc_inst_body.cuh"
