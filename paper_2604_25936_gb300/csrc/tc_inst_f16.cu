// Tensor-core T-MLP kernel instantiations: the fp16 mode.
#define SAND_INST_MODE TC_F16
#define SAND_INST_EXT false
#include "tc_inst_body.cuh"
