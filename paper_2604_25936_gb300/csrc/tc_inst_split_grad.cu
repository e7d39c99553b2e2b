// Tensor-core T-MLP kernel instantiations: the float32 mode (3 x fp16 split), value and input gradient.
#define SAND_INST_MODE TC_SPLIT16
#define SAND_INST_VAR 2
#include "tc_inst_body.cuh"
