// Tensor-core T-MLP kernel instantiations: the float32 mode at width 336 with A_lo in shared memory, extended output variant.
#define SAND_INST_MODE TC_SPLIT16
#define SAND_INST_VAR 5
#include "tc_inst_body.cuh"
