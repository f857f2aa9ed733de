"""Pulsatile duct of Sec. 5.2 on the GPU: a time-dependent uniform body force set
through lb_set_force between steps, checked against the FP64 oracle step by step and
against the Fourier-series solution on the paper's three cuboid grids."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_time_dependent_force_parity_fp64(oracle_mod):
    """A force that changes at every step (walls on y and z): FP64 storage within 1e-12
    of the oracle given the same force sequence."""
    from paper_2107_14774_gb300 import Lattice
    n, r, s = (12, 16, 10), 0.5, 1.0
    lat = Lattice(*n, r_y=r, r_z=s, nu=0.03, storage="f64", walls="yz")
    p = lat.params
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          corr=oracle_mod.CORR_LOCAL, walls="yz")
    rho, u = synth.solenoidal_random(*n, r, s, 2.0, 0.01, seed=5)
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    f = o.init(rho, u)
    for k in range(40):
        F = (1e-4 * np.cos(0.2 * k), 3e-5 * np.sin(0.1 * k), -2e-5 * (k % 3))
        lat.set_force(F).step(1)
        o.set_force(F)
        f = o.step(f)
    fg = lat.populations().cpu().numpy()
    assert np.linalg.norm(fg - f) / np.linalg.norm(f) < 1e-12
    lat.close()


@pytest.mark.parametrize("ny,nz,r,s,Wo", [
    (80, 40, 0.5, 1.0, 3.09),
    (80, 80, 0.5, 0.5, 3.09),
    (160, 80, 0.25, 0.5, 3.09),
    (80, 40, 0.5, 1.0, 6.25),
])
def test_pulsatile_duct_paper_grids(ny, nz, r, s, Wo):
    """2a = 40, Fm = 1e-5, T = 10000 (Sec. 5.2), FP32 storage on an nx = 40 slab.
    Started from the series at t = 0 (equilibrium populations), one period is run and
    u_x is compared with the series at each quarter period; the relative L2 error is
    normalised by the local oscillation amplitude."""
    from paper_2107_14774_gb300 import Lattice
    from tests.analytic import pulsatile_duct
    nx, a, Fm, T = 40, 20.0, 1e-5, 10000
    om = 2 * np.pi / T
    nu = a * a * om / (Wo * Wo)
    lat = Lattice(nx, ny, nz, r_y=r, r_z=s, nu=nu, storage="f32", walls="yz", force=(Fm, 0.0, 0.0))
    Z, Y = np.meshgrid((np.arange(nz) + 0.5) * s - a, (np.arange(ny) + 0.5) * r - a, indexing="ij")
    amp = np.abs(pulsatile_duct(Y, Z, 0.0, a, Fm, om, nu) + 1j * pulsatile_duct(Y, Z, T / 4, a, Fm, om, nu))
    u0 = np.zeros((3, nz, ny, nx))
    u0[0] = pulsatile_duct(Y, Z, 0.0, a, Fm, om, nu)[:, :, None]
    lat.init(torch.ones((nz, ny, nx), dtype=torch.float64).cuda(), torch.from_numpy(u0).cuda())
    n, errs = 0, []
    for q in range(1, 5):
        while n < q * T // 4:
            lat.set_force((Fm * np.cos(om * n), 0.0, 0.0)).step(1)
            n += 1
        lat.set_force((Fm * np.cos(om * n), 0.0, 0.0))
        _, u = lat.moments()
        u = u.cpu().numpy().astype(np.float64)
        ua = pulsatile_duct(Y, Z, float(n), a, Fm, om, nu)
        errs.append(np.linalg.norm(u[0].mean(axis=2) - ua) / np.linalg.norm(amp))
        assert np.abs(u[0] - u[0][:, :, :1]).max() < 1e-6 * amp.max()   # x-invariant
        assert np.abs(u[1:]).max() < 1e-4 * amp.max()                   # no secondary flow
    print("pulsatile", (ny, nz, r, s, Wo), ["%.4f" % e for e in errs])
    assert max(errs) < 0.01
    lat.close()
