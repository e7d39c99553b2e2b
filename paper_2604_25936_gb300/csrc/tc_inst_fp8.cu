// Tensor-core T-MLP kernel instantiations: the FP8 (e4m3) mode.
#define SAND_INST_MODE TC_FP8
#define SAND_INST_VAR 0
#include "tc_inst_body.cuh"
