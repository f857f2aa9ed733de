// Instantiation of the two-node step launcher (and its kernels) for population
// storage LB_BF16_SHIFTED.
#include "ops.cuh"

template cudaError_t lbc::Ops<LB_BF16_SHIFTED>::step_pair(const lbc::LaunchArgs &, const void *, void *);
