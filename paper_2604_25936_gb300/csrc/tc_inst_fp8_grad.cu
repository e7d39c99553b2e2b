// Tensor-core T-MLP kernel instantiations: the FP8 (e4m3) mode, value and input gradient.
#define SAND_INST_MODE TC_FP8
#define SAND_INST_VAR 2
#include "tc_inst_body.cuh"
