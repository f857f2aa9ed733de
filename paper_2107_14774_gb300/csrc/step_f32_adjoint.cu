// Instantiation of the adjoint launchers (and their kernels) for population
// storage LB_F32.
#include "ops.cuh"

template cudaError_t lbc::Ops<LB_F32>::adjoint_seed(const lbc::LaunchArgs &, const void *, void *, void *, double *);
template cudaError_t lbc::Ops<LB_F32>::adjoint_step(const lbc::LaunchArgs &, const void *, const void *, void *, void *,
                                                 double *);
template cudaError_t lbc::Ops<LB_F32>::collide_vjp(const lbc::LaunchArgs &, const void *, const void *, const void *,
                                                void *, void *, long long, double *);
