"""The differentiable torch reference (oracle/torch_ref.py) against the C oracle and
against central finite differences of the C oracle.  CPU only."""
import numpy as np
import pytest
import torch

import synth
from oracle import torch_ref as tr


@pytest.mark.parametrize("corr", ["none", "lowmach", "local"])
@pytest.mark.parametrize("r,s,cs2", [(0.5, 2.0, 1 / 12), (1.0, 0.5, 0.1), (0.406, 1.3, 0.04)])
def test_collision_matches_c_oracle(oracle_mod, corr, r, s, cs2):
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=1.55, omega_xi=1.2, corr=getattr(oracle_mod, "CORR_" + corr.upper()))
    fs = synth.random_populations(5, seed=31)
    F = 1e-3 * np.random.default_rng(1).standard_normal((5, 3))
    got = tr.collide(torch.from_numpy(fs.T.copy()), torch.from_numpy(F.T.copy()), r, s, cs2, 1.55, 1.2, corr).numpy()
    want = np.stack([o.collide_node(f, Fi) for f, Fi in zip(fs, F)], 1)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-14)


def test_run_matches_c_oracle_with_walls_and_force_field(oracle_mod):
    n, r, s, cs2 = (6, 5, 4), 0.5, 1.0, 0.04
    rho, u = synth.solenoidal_random(*n, r, s, 2.0, 0.02, seed=5)
    ff = synth.force_field(*n, 1e-4, seed=6)
    wn, wb = 1.4, 1.1
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=cs2, omega_nu=wn, omega_xi=wb, walls="yz", force_field=ff)
    f0 = o.init(rho, u)
    want = o.run(f0, 5)
    N = np.prod(n)
    got = tr.run(torch.from_numpy(f0.reshape(27, N)), torch.from_numpy(ff.reshape(3, N)), r, s, cs2, wn, wb, 5, n,
                 walls="yz").numpy().reshape(want.shape)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
    feq = tr.equilibrium(torch.from_numpy(rho.reshape(N)), torch.from_numpy(u.reshape(3, N)), r, s, cs2)
    np.testing.assert_allclose(feq.numpy().reshape(f0.shape), f0, rtol=1e-12)


def test_autograd_gradient_matches_finite_differences_of_c_oracle(oracle_mod):
    """dJ/domega_nu, dJ/domega_xi and a directional dJ/dF of the mean kinetic energy
    after T steps (torch autograd) against central differences of the C oracle."""
    n, r, s, cs2, T = (6, 4, 5), 1.0, 0.5, 1 / 12, 6
    N = int(np.prod(n))
    rho, u = synth.solenoidal_random(*n, r, s, 2.0, 0.03, seed=8)
    ff = synth.force_field(*n, 1e-4, seed=9)
    v = synth.random_direction((3,) + n[::-1], np.linalg.norm(ff), seed=10)

    def J_c(wn, wb, F):
        o = oracle_mod.Oracle(*n, r=r, s=s, cs2=cs2, omega_nu=wn, omega_xi=wb, force_field=F)
        f = o.run(o.init(rho, u), T)
        rr, uu = o.moments(f)
        return float((0.5 * rr * (uu ** 2).sum(0)).mean())

    wn0, wb0 = 1.6, 1.2
    f0 = torch.from_numpy(oracle_mod.Oracle(*n, r=r, s=s, cs2=cs2).init(rho, u).reshape(27, N))
    w = torch.tensor([wn0, wb0], dtype=torch.float64, requires_grad=True)
    F = torch.from_numpy(ff.reshape(3, N).copy()).requires_grad_(True)
    J = tr.mean_kinetic_energy(tr.run(f0, F, r, s, cs2, w[0], w[1], T, n), F, r, s)
    J.backward()
    h = 1e-4
    d_wn = (J_c(wn0 + h, wb0, ff) - J_c(wn0 - h, wb0, ff)) / (2 * h)
    d_wb = (J_c(wn0, wb0 + h, ff) - J_c(wn0, wb0 - h, ff)) / (2 * h)
    eps = 1e-2
    d_F = (J_c(wn0, wb0, ff + eps * v) - J_c(wn0, wb0, ff - eps * v)) / (2 * eps)
    assert w.grad[0].item() == pytest.approx(d_wn, rel=1e-6)
    assert w.grad[1].item() == pytest.approx(d_wb, rel=1e-6)
    assert float((F.grad.numpy() * v.reshape(3, N)).sum()) == pytest.approx(d_F, rel=1e-6)
    assert J.item() == pytest.approx(J_c(wn0, wb0, ff), rel=1e-12)
