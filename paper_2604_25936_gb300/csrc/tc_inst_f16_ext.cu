// Tensor-core T-MLP kernel instantiations: the fp16 mode, extended outputs (all tails, dynamic exit).
#define SAND_INST_MODE TC_F16
#define SAND_INST_VAR 1
#include "tc_inst_body.cuh"
