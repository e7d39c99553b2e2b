// Tensor-core T-MLP kernel instantiations: the bf16 mode.
#define SAND_INST_MODE TC_BF16
#define SAND_INST_VAR 0
#include "tc_inst_body.cuh"
