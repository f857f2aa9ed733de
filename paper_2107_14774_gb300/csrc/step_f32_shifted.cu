// Instantiation of the kernels and launchers for population storage LB_F32_SHIFTED (the
// two-node step and the adjoint launchers are instantiated in step_f32_shifted_pair.cu
// and step_f32_shifted_adjoint.cu, so that the three compile in parallel).
#define LBC_OPS_SKIP_PAIR
#define LBC_OPS_SKIP_ADJOINT
#include "ops.cuh"

template struct lbc::Ops<LB_F32_SHIFTED>;
