// Instantiation of the kernels and launchers for population storage LB_BF16_SHIFTED (the
// two-node step and the adjoint launchers are instantiated in step_bf16_shifted_pair.cu
// and step_bf16_shifted_adjoint.cu, so that the three compile in parallel).
#define LBC_OPS_SKIP_PAIR
#define LBC_OPS_SKIP_ADJOINT
#include "ops.cuh"

template struct lbc::Ops<LB_BF16_SHIFTED>;
