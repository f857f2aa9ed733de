"""torch.autograd.Function around the hand-written adjoint of liblbcuboid.

``kinetic_energy_rollout(force, omegas, rho0, u0, T, K, **lattice)`` returns the mean
kinetic energy J after T fused steps started from f^eq(rho0, u0), driven by the
per-node body force ``force`` [3, nz, ny, nx] with relaxation rates ``omegas`` =
(omega_nu, omega_xi).  Its backward gives dJ/dforce and dJ/domegas from the
discrete adjoint (lb_adjoint_ke: transposed streaming plus the per-node VJP of the
collision, with checkpoint-and-recompute every K steps).  The gradient is computed
in the same C-ABI call as the forward rollout.
"""
from __future__ import annotations

import torch

from .lattice import Lattice


class KineticEnergyRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, force, omegas, rho0, u0, T, K, lattice_kwargs):
        shape = tuple(force.shape[1:])
        nz, ny, nx = shape
        lat = Lattice(nx, ny, nz, **lattice_kwargs)
        try:
            w = omegas.detach().double().cpu()
            lat.set_rates(float(w[0]), float(w[1]))
            lat.set_force_field(force.detach())
            lat.init(rho0, u0)
            J, dJdF, dJdw = lat.adjoint_ke(T, K)
        finally:
            lat.close()
        ctx.save_for_backward(dJdF.to(force.dtype), torch.tensor(dJdw, dtype=omegas.dtype, device=omegas.device))
        return torch.tensor(J, dtype=force.dtype, device=force.device)

    @staticmethod
    def backward(ctx, gJ):
        dJdF, dJdw = ctx.saved_tensors
        return gJ * dJdF, gJ * dJdw, None, None, None, None, None


def kinetic_energy_rollout(force, omegas, rho0, u0, T, K, **lattice_kwargs):
    """Mean kinetic energy after T steps; differentiable in force and omegas."""
    return KineticEnergyRollout.apply(force, omegas, rho0, u0, T, K, lattice_kwargs)
