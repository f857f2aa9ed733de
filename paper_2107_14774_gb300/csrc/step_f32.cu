// Instantiation of the kernels and launchers for population storage LB_F32.
#include "ops.cuh"

template struct lbc::Ops<LB_F32>;
