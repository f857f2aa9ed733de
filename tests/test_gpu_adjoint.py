"""The hand-written adjoint (through the C ABI) against torch autograd of the FP64
torch reference (oracle/torch_ref.py) and against central finite differences."""
import numpy as np
import pytest
import torch

import synth
from oracle import torch_ref as tr

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 2e-4)])
@pytest.mark.parametrize("corr", ["none", "lowmach", "local"])
@pytest.mark.parametrize("r,s,cs2", [(1.0, 0.5, 1 / 12), (0.5, 2.0, 1 / 12), (0.406, 1.3, 0.04)])
def test_per_node_vjp_matches_autograd(storage, tol, corr, r, s, cs2):
    from paper_2107_14774_gb300 import Lattice
    n = 300
    wn, wb = 1.55, 1.2
    lat = Lattice(1, 1, 1, r_y=r, r_z=s, nu=0.01, cs2=cs2, storage=storage, corr=corr)
    lat.set_rates(wn, wb)
    rng = np.random.default_rng(3)
    rho = 1 + 0.01 * rng.standard_normal(n)
    u = 0.04 * rng.standard_normal((3, n))
    feq = tr.equilibrium(torch.from_numpy(rho), torch.from_numpy(u), r, s, cs2)
    f = (feq * (1 + 0.02 * torch.from_numpy(rng.standard_normal((27, n))))).detach()
    F = torch.from_numpy(1e-4 * rng.standard_normal((3, n)))
    lam = torch.from_numpy(rng.standard_normal((27, n)))
    fb, Fb, wbar = lat.collide_vjp(f.cuda(), F.cuda(), lam.cuda())
    lat.close()
    fr = f.clone().requires_grad_(True)
    Fr = F.clone().requires_grad_(True)
    w = torch.tensor([wn, wb], dtype=torch.float64, requires_grad=True)
    (tr.collide(fr, Fr, r, s, cs2, w[0], w[1], corr) * lam).sum().backward()
    assert rel(fb.cpu(), fr.grad) < tol
    assert rel(Fb.cpu(), Fr.grad) < tol
    assert rel(wbar, w.grad) < tol


def _tiny_setup(n, r, s, seed=8):
    rho, u = synth.solenoidal_random(*n, r, s, 2.0, 0.03, seed=seed)
    ff = synth.force_field(*n, 1e-4, seed=seed + 1)
    return rho, u, ff


@pytest.mark.parametrize("storage,tol", [("f64", 1e-9), ("f32", 1e-3)])
@pytest.mark.parametrize("walls,corr", [("", "local"), ("y", "local"), ("yz", "lowmach"), ("", "none")])
def test_adjoint_rollout_matches_autograd(storage, tol, walls, corr):
    """8x6x4 lattice (r=1, s=0.5), T=20 steps, checkpoint every K=5: J, dJ/dF and
    dJ/domega from the GPU adjoint against torch autograd through the FP64 reference."""
    from paper_2107_14774_gb300 import kinetic_energy_rollout
    n, r, s, cs2, T, K = (8, 6, 4), 1.0, 0.5, 1 / 12, 20, 5
    N = int(np.prod(n))
    rho, u, ff = _tiny_setup(n, r, s)
    dt = torch.float64 if storage == "f64" else torch.float32
    F = torch.from_numpy(ff).to("cuda", dt).requires_grad_(True)
    w = torch.tensor([1.6, 1.2], dtype=dt, device="cuda", requires_grad=True)
    J = kinetic_energy_rollout(F, w, torch.from_numpy(rho), torch.from_numpy(u), T, K, r_y=r, r_z=s, cs2=cs2,
                               storage=storage, corr=corr, walls=walls)
    J.backward()
    f0 = tr.equilibrium(torch.from_numpy(rho.reshape(N)), torch.from_numpy(u.reshape(3, N)), r, s, cs2)
    Fr = torch.from_numpy(ff.reshape(3, N).copy()).requires_grad_(True)
    wr = torch.tensor([1.6, 1.2], dtype=torch.float64, requires_grad=True)
    Jr = tr.mean_kinetic_energy(tr.run(f0, Fr, r, s, cs2, wr[0], wr[1], T, n, walls=walls, corr=corr), Fr, r, s)
    Jr.backward()
    assert abs(J.item() / Jr.item() - 1) < (1e-12 if storage == "f64" else 1e-5)
    assert rel(F.grad.cpu().reshape(3, N), Fr.grad) < tol
    assert rel(w.grad.cpu(), wr.grad) < tol


def test_adjoint_leaves_state_after_T_steps():
    from paper_2107_14774_gb300 import Lattice
    n = (16, 8, 8)
    rho, u, ff = _tiny_setup(n, 1.0, 0.5)
    a = Lattice(*n, r_y=1.0, r_z=0.5, nu=0.01)
    b = Lattice(*n, r_y=1.0, r_z=0.5, nu=0.01)
    for lat in (a, b):
        lat.set_force_field(torch.from_numpy(ff).cuda())
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    a.adjoint_ke(13, 4)
    b.step(13)
    assert torch.equal(a.get_state(), b.get_state()) and a.time_step == 13
    assert a.objective_ke() == pytest.approx(b.objective_ke(), rel=1e-15)
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("walls", ["", "y"])
def test_adjoint_independent_of_checkpoint_interval(storage, walls):
    """Every checkpoint interval K gives the same J, dJ/dF and dJ/domega bit for bit: the
    adjoint steps read the same states in the same order whether they were kept (K = 1
    keeps every state resident and recomputes nothing) or recomputed from a checkpoint
    (K >= T recomputes the whole run from the initial state); and every K leaves the
    state lb_step(T) leaves."""
    from paper_2107_14774_gb300 import Lattice
    n, T = (16, 8, 8), 13
    rho, u, ff = _tiny_setup(n, 1.0, 0.5)

    def fresh():
        lat = Lattice(*n, r_y=1.0, r_z=0.5, nu=0.01, storage=storage, walls=walls)
        lat.set_force_field(torch.from_numpy(ff).cuda())
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        return lat
    ref = fresh()
    ref.step(T)
    state_T = ref.get_state().cpu()
    ref.close()
    out = {}
    for K in (1, 3, 5, 13, 20):
        lat = fresh()
        J, g, w = lat.adjoint_ke(T, K)
        assert torch.equal(lat.get_state().cpu(), state_T) and lat.time_step == T, K
        out[K] = (J, g.cpu(), w)
        lat.close()
    J1, g1, w1 = out[1]
    for K, (J, g, w) in out.items():
        assert J == J1 and torch.equal(g, g1) and w == w1, K


def test_adjoint_128x64x64_against_central_differences():
    """Adjoint case 128x64x64 periodic, r_z=0.5, FP32, mean kinetic energy after T=500
    steps, checkpoint every 50; u0 from the solenoidal generator at u_rms=0.01 (seed 4),
    F i.i.d. N(0, (1e-5)^2) (seed 44).  The FP32 adjoint against central differences
    of the FP64 forward: dJ/domega_nu, dJ/domega_xi (h = 1e-3 relative), the directional
    derivative along a seeded v with |v| = |F| (h = 1e-3), and 16 single components."""
    from paper_2107_14774_gb300 import Lattice
    n, r, s, nu, T, K = (128, 64, 64), 1.0, 0.5, 0.01, 500, 50
    rho, u = synth.solenoidal_random(*n, r, s, 4.0, 0.01, seed=4)
    ff = synth.force_field(*n, 1e-5, seed=44)
    v = synth.random_direction(ff.shape, np.linalg.norm(ff), seed=45)
    rho_t, u_t = torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()

    lat = Lattice(*n, r_y=r, r_z=s, nu=nu, storage="f32")
    wn0, wb0 = lat.params["omega_nu"], lat.params["omega_xi"]
    lat.set_force_field(torch.from_numpy(ff).cuda())
    lat.init(rho_t, u_t)
    J32, dJdF, dJdw = lat.adjoint_ke(T, K)
    dJdF = dJdF.double().cpu().numpy()
    lat.close()

    ref = Lattice(*n, r_y=r, r_z=s, nu=nu, storage="f64")

    def J64(wn, wb, F):
        ref.set_rates(wn, wb)
        ref.set_force_field(torch.from_numpy(F).cuda())
        ref.init(rho_t, u_t).step(T)
        return ref.objective_ke()

    J0 = J64(wn0, wb0, ff)
    assert J32 == pytest.approx(J0, rel=1e-4)
    h = 1e-3
    d_wn = (J64(wn0 * (1 + h), wb0, ff) - J64(wn0 * (1 - h), wb0, ff)) / (2 * h * wn0)
    d_wb = (J64(wn0, wb0 * (1 + h), ff) - J64(wn0, wb0 * (1 - h), ff)) / (2 * h * wb0)
    d_v = (J64(wn0, wb0, ff + h * v) - J64(wn0, wb0, ff - h * v)) / (2 * h)
    print(f"adjoint 128x64x64: J {J32:.6e} vs {J0:.6e}; dJ/dwn {dJdw[0]:.6e} vs FD {d_wn:.6e}; "
          f"dJ/dwb {dJdw[1]:.6e} vs {d_wb:.6e}; <dJ/dF,v> {(dJdF * v).sum():.6e} vs {d_v:.6e}")
    assert dJdw[0] == pytest.approx(d_wn, rel=1e-4)
    assert dJdw[1] == pytest.approx(d_wb, rel=1e-4)
    assert float((dJdF * v).sum()) == pytest.approx(d_v, rel=1e-4)
    rng = np.random.default_rng(46)
    eps = 1e-5
    worst = 0.0
    for _ in range(16):
        c, k, j, i = (int(rng.integers(0, m)) for m in (3, n[2], n[1], n[0]))
        e = np.zeros_like(ff)
        e[c, k, j, i] = eps
        d = (J64(wn0, wb0, ff + e) - J64(wn0, wb0, ff - e)) / (2 * eps)
        worst = max(worst, abs(dJdF[c, k, j, i] - d) / abs(d))
    print(f"adjoint 128x64x64: worst single-component relative error {worst:.2e}")
    assert worst < 1e-4
    ref.close()


def test_lb_adjoint_matches_lb_adjoint_ke():
    """lb_adjoint (the entry point without J) returns the same gradients as lb_adjoint_ke."""
    import ctypes
    from paper_2107_14774_gb300 import Lattice
    from paper_2107_14774_gb300._lib import check
    n = (16, 8, 8)
    rho, u = synth.solenoidal_random(*n, 1.0, 0.5, 2.0, 0.01, seed=8)
    lat = Lattice(*n, r_y=1.0, r_z=0.5, nu=0.02, storage="f64")
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    _, g1, w1 = lat.adjoint_ke(20, 5)
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    g2 = torch.empty_like(g1)
    dw = (ctypes.c_double * 2)()
    check(lat.lib.lb_adjoint(lat.ctx, 20, 5, g2.data_ptr(), dw))
    assert torch.equal(g1, g2) and (dw[0], dw[1]) == w1
    lat.close()
