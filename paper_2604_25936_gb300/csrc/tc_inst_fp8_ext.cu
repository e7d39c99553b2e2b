// Tensor-core T-MLP kernel instantiations: the FP8 (e4m3) mode, extended outputs (all tails, dynamic exit).
#define SAND_INST_MODE TC_FP8
#define SAND_INST_VAR 1
#include "tc_inst_body.cuh"
