// Tensor-core T-MLP kernel instantiations: the float32 mode (3 x fp16 split).
#define SAND_INST_MODE TC_SPLIT16
#define SAND_INST_VAR 0
#include "tc_inst_body.cuh"
