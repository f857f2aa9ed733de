// Instantiation of the two-node step launcher (and its kernels) for population
// storage LB_F16_SHIFTED.
#include "ops.cuh"

template cudaError_t lbc::Ops<LB_F16_SHIFTED>::step_pair(const lbc::LaunchArgs &, const void *, void *);
