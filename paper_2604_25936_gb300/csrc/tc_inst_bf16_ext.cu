// Tensor-core T-MLP kernel instantiations: the bf16 mode, extended outputs (all tails, dynamic exit).
#define SAND_INST_MODE TC_BF16
#define SAND_INST_VAR 1
#include "tc_inst_body.cuh"
