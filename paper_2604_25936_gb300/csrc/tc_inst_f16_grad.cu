// Tensor-core T-MLP kernel instantiations: the fp16 mode, value and input gradient.
#define SAND_INST_MODE TC_F16
#define SAND_INST_VAR 2
#include "tc_inst_body.cuh"
