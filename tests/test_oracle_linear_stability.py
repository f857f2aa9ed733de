"""Linear stability of the update about the rest state, from the FP64 oracle (a von Neumann
analysis).  The collision is linearised at f = f^eq(1, 0) by central differences; streaming
multiplies population a by exp(-i k.e_a); the spectral radius of the product over a grid of
wavevectors k says whether small perturbations of the rest state grow.

The case is the lattice of the Sec. 7 stability study (Figs. 8 and 9): r = 0.5, s = 1,
c_s^2 = 0.08, every rate other than omega_nu and omega_xi equal to one.  The first test pins
the linearised collision to what relaxing moments at given rates means; the others record
where the grid-anisotropy corrections of App. D (Eqs. 38-40, 44-49, 63), in the reading the
oracle implements, move the stability limit."""
import itertools

import numpy as np
import pytest

import oracle

EX = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1])
EY = np.array([0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1])
EZ = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1])
R, S, CS2 = 0.5, 1.0, 0.08


def jacobian(omega_nu, omega_xi, corr, r=R, s=S, cs2=CS2, u0=(0.0, 0.0, 0.0), model="central"):
    """d(post-collision f)/d(pre-collision f) at the equilibrium of density 1 and velocity u0
    (the rest state by default), by central differences."""
    o = oracle.Oracle(1, 1, 1, r=r, s=s, cs2=cs2, omega_nu=omega_nu, omega_xi=omega_xi, corr=corr, model=model)
    f0 = o.equilibrium(1.0, u0)
    eps = 1e-7
    cols = []
    for b in range(27):
        d = np.zeros(27)
        d[b] = eps
        cols.append((o.collide_node(f0 + d) - o.collide_node(f0 - d)) / (2 * eps))
    return np.stack(cols, axis=1)


def spectral_radius(omega_nu, omega_xi, corr, nk=12, r=R, s=S, cs2=CS2, u0=(0.0, 0.0, 0.0), model="central"):
    """Largest |eigenvalue| of the linearised step over an nk^3 grid of wavevectors
    (cell centres of [-pi, pi)^3, so k = 0 and its conserved modes are left out)."""
    J = jacobian(omega_nu, omega_xi, corr, r, s, cs2, u0, model)
    ks = np.linspace(-np.pi, np.pi, nk, endpoint=False) + np.pi / nk
    worst = 0.0
    for kx, ky, kz in itertools.product(ks, ks, ks):
        phase = np.exp(-1j * (kx * EX + ky * EY + kz * EZ))
        worst = max(worst, float(np.abs(np.linalg.eigvals(phase[:, None] * J)).max()))
    return worst


@pytest.mark.parametrize("omega_nu,omega_xi", [(1.5, 1.0), (1.9, 0.5), (1.3, 1.4)])
def test_uncorrected_collision_relaxes_at_the_given_rates(omega_nu, omega_xi):
    """Without corrections the linearised collision at rest relaxes each moment at its own
    rate (App. D): eigenvalue 1 for mass and the three momenta, 1 - omega_nu for the five
    deviatoric second-order moments, 1 - omega_xi for their trace, 0 for the 17 higher
    moments (all relaxed at one)."""
    ev = np.sort(np.linalg.eigvals(jacobian(omega_nu, omega_xi, oracle.CORR_NONE)).real)
    want = np.sort([1.0] * 4 + [1.0 - omega_nu] * 5 + [1.0 - omega_xi] + [0.0] * 17)
    assert np.allclose(ev, want, atol=1e-7)


@pytest.mark.parametrize("omega_nu", [1.5, 1.9, 1.95])
@pytest.mark.parametrize("omega_xi", [0.5, 1.0, 1.4])
def test_uncorrected_rest_state_is_linearly_stable(omega_nu, omega_xi):
    assert spectral_radius(omega_nu, omega_xi, oracle.CORR_NONE) <= 1.0 + 1e-9


def test_corrections_raise_the_effective_shear_rate_independently_of_omega_xi():
    """With the corrections the normal-stress differences relax faster than omega_nu: at
    c_s^2 = 0.08 the lattice's own second moments along x and z (c^2/3 = 1/3) exceed c_s^2
    and the correction takes the excess away.  The fastest mode's rate, 1 - (smallest
    eigenvalue), is 1.890 at omega_nu = 1.5 and 1.991 at 1.95, whatever omega_xi."""
    for omega_nu, want in ((1.5, 1.8904), (1.95, 1.9911)):
        rates = [1.0 - np.linalg.eigvals(jacobian(omega_nu, wb, oracle.CORR_LOCAL)).real.min()
                 for wb in (0.5, 1.0, 1.4)]
        assert np.allclose(rates, want, atol=5e-4), rates
        assert min(rates) > omega_nu


def test_corrected_rest_state_loses_stability_near_omega_nu_1_9():
    """With the corrections the rest state itself turns linearly unstable at omega_nu = 1.9
    for omega_xi = 0.5 and at 1.95 for every omega_xi of Fig. 9; a lower omega_xi gives the
    larger growth rate there."""
    for wb in (0.5, 1.0, 1.4):
        assert spectral_radius(1.8, wb, oracle.CORR_LOCAL) < 1.0
    assert spectral_radius(1.9, 0.5, oracle.CORR_LOCAL) > 1.003
    assert spectral_radius(1.9, 1.0, oracle.CORR_LOCAL) < 1.0
    rho = [spectral_radius(1.95, wb, oracle.CORR_LOCAL) for wb in (0.5, 1.0, 1.4)]
    assert min(rho) > 1.005 and rho[0] > rho[1] > rho[2]


@pytest.mark.parametrize("cs2", [1.0 / 3.0, 0.08])
@pytest.mark.parametrize("corr", [oracle.CORR_NONE, oracle.CORR_LOCAL])
def test_cubic_lattice_rest_stability_does_not_depend_on_omega_xi(corr, cs2):
    """On the cubic lattice (r = s = 1) the least-damped mode of the rest state is the same for
    omega_xi = 0.5, 1 and 1.4, with or without the corrections, and stable at omega_nu = 1.98."""
    rho = [spectral_radius(1.98, wb, corr, r=1.0, s=1.0, cs2=cs2) for wb in (0.5, 1.0, 1.4)]
    assert max(rho) - min(rho) < 1e-9 and max(rho) < 1.0


def test_cuboid_lattice_low_omega_xi_destabilises_the_uncorrected_rest_state():
    """On the r = 0.5 lattice of Sec. 7 the bulk mode couples to the grid anisotropy: without
    any corrections the rest state at omega_nu = 1.98 is unstable for omega_xi = 0.5 and
    stable for omega_xi = 1 and 1.4 -- a larger bulk viscosity destabilises it."""
    assert spectral_radius(1.98, 0.5, oracle.CORR_NONE) > 1.002
    assert spectral_radius(1.98, 1.0, oracle.CORR_NONE) < 1.0
    assert spectral_radius(1.98, 1.4, oracle.CORR_NONE) < 1.0


@pytest.mark.parametrize("omega_nu,u", [(1.7, 0.2), (1.8, 0.15)])
def test_central_moments_stay_stable_in_a_uniform_flow_where_raw_moments_do_not(omega_nu, u):
    """Sec. 7 (Fig. 8) in linear form: about a uniform flow along x on the r = 0.5 lattice the
    central-moment scheme (3DCCM) is stable at speeds where the raw-moment scheme (3DCRM) with
    the same corrected equilibria is not."""
    central = spectral_radius(omega_nu, 1.0, oracle.CORR_LOCAL, u0=(u, 0.0, 0.0), model="central")
    raw = spectral_radius(omega_nu, 1.0, oracle.CORR_LOCAL, u0=(u, 0.0, 0.0), model="raw")
    assert central < 1.0 < raw
