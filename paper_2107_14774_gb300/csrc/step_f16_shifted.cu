// Instantiation of the kernels and launchers for population storage LB_F16_SHIFTED (the
// two-node step and the adjoint launchers are instantiated in step_f16_shifted_pair.cu
// and step_f16_shifted_adjoint.cu, so that the three compile in parallel).
#define LBC_OPS_SKIP_PAIR
#define LBC_OPS_SKIP_ADJOINT
#include "ops.cuh"

template struct lbc::Ops<LB_F16_SHIFTED>;
