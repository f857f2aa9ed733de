// Instantiation of the kernels and launchers for population storage LB_F64 (the
// adjoint launchers are instantiated in step_f64_adjoint.cu).
#define LBC_OPS_SKIP_ADJOINT
#include "ops.cuh"

template struct lbc::Ops<LB_F64>;
