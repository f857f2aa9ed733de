"""Pins of the oracle's raw-moment scheme (3DCRM: the cuboid raw-moment formulation of
Sec. 3.1 with the corrected equilibria of the central scheme, compared in Sec. 7)."""
import numpy as np
import pytest

import synth
from tests.analytic import raw_equilibria_eq10, fit_decay_rate


def _names(o):
    m, n, p = o.moment_exponents()
    return [f"{a}{b}{c}" for a, b, c in zip(m, n, p)]


def _rand_f(o, rng, u_scale=0.05):
    w = o.equilibrium(1.0, np.zeros(3))
    return w * (1.0 + 0.3 * rng.standard_normal(27)) + o.equilibrium(1.0, u_scale * rng.standard_normal(3)) - w


def _raw_moments(f, r, s, names):
    e = np.array([[1.0], [r], [s]]) * _vel()
    return {nm: float(np.sum(f * e[0] ** int(nm[0]) * e[1] ** int(nm[1]) * e[2] ** int(nm[2]))) for nm in names}


def _vel():
    import oracle
    return oracle.Oracle.velocities().astype(float)


def test_raw_equilibrium_matches_eq10(oracle_mod):
    o = oracle_mod.Oracle(cs2=0.07)
    rho, u = 1.021, np.array([0.03, -0.045, 0.02])
    m = o.raw_equilibrium(rho, u)
    want = raw_equilibria_eq10(rho, u, 0.07)
    for j, nm in enumerate(_names(o)):
        assert m[j] == pytest.approx(want[nm], rel=1e-14, abs=1e-18), nm


@pytest.mark.parametrize("corr", ["NONE", "LOWMACH", "LOCAL", "FULL"])
def test_raw_factored_equals_definitional(oracle_mod, corr):
    """S P f ... P^-1 S^-1 against moments taken with the cuboid velocities (Eq. 3b) and
    an LU solve back: two independent routes through the raw-moment scheme."""
    rng = np.random.default_rng(21)
    kw = dict(r=0.5, s=1.3, cs2=0.07, omega_nu=1.6, omega_xi=1.2, corr=getattr(oracle_mod, "CORR_" + corr),
              model="raw")
    a = oracle_mod.Oracle(form=0, **kw)
    b = oracle_mod.Oracle(form=1, **kw)
    for _ in range(10):
        f = _rand_f(a, rng)
        F, g = 1e-3 * rng.standard_normal(3), 1e-2 * rng.standard_normal(3)
        np.testing.assert_allclose(a.collide_node(f, F, g), b.collide_node(f, F, g), rtol=1e-11, atol=1e-14)


def test_raw_collision_conserves_mass_and_adds_force(oracle_mod):
    rng = np.random.default_rng(22)
    r, s = 0.5, 0.8
    o = oracle_mod.Oracle(r=r, s=s, cs2=0.06, omega_nu=1.7, omega_xi=0.9, model="raw")
    e = np.array([[1.0], [r], [s]]) * o.velocities()
    for _ in range(10):
        f = _rand_f(o, rng)
        F = 1e-3 * rng.standard_normal(3)
        ft = o.collide_node(f, F)
        assert ft.sum() == pytest.approx(f.sum(), rel=1e-14)
        np.testing.assert_allclose(e @ ft, e @ f + F, rtol=0, atol=1e-15)


def test_raw_equals_central_at_rest(oracle_mod):
    """With zero momentum and no force the frame transformation F(0) is the identity, so
    the raw and the central scheme coincide (Sec. 7: they differ only by the mappings
    involving F(u))."""
    rng = np.random.default_rng(23)
    kw = dict(r=0.406, s=1.3, cs2=0.05, omega_nu=1.8, omega_xi=1.1)
    oc = oracle_mod.Oracle(**kw)
    orw = oracle_mod.Oracle(model="raw", **kw)
    opp = [int(np.flatnonzero((oc.velocities() == -oc.velocities()[:, [a]]).all(axis=0))[0]) for a in range(27)]
    for _ in range(5):
        g = _rand_f(oc, rng)
        f = 0.5 * (g + g[opp])                      # symmetric: zero momentum
        np.testing.assert_allclose(orw.collide_node(f), oc.collide_node(f), rtol=1e-13, atol=1e-16)
    # away from rest they differ
    f = _rand_f(oc, rng, u_scale=0.08)
    assert np.abs(orw.collide_node(f) - oc.collide_node(f)).max() > 1e-8


def test_raw_equilibrium_is_fixed_point_and_higher_moments_are_eq10(oracle_mod):
    """f^eq(rho, u) is left unchanged without a force; for any input the post-collision
    raw moments of order >= 3 are the raw equilibria of Eq. 10 (rates 1) and those of
    order 1 equal rho u + F/2."""
    rng = np.random.default_rng(24)
    r, s, cs2 = 0.5, 1.3, 0.07
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=1.5, omega_xi=1.0, model="raw")
    u = np.array([0.04, -0.02, 0.03])
    feq = o.equilibrium(0.98, u)
    np.testing.assert_allclose(o.collide_node(feq), feq, rtol=1e-13, atol=1e-16)
    names = _names(o)
    for _ in range(5):
        f = _rand_f(o, rng)
        F = 1e-3 * rng.standard_normal(3)
        e = np.array([[1.0], [r], [s]]) * o.velocities()
        rho = f.sum()
        uu = (e @ f + F / 2) / rho
        mt = _raw_moments(o.collide_node(f, F), r, s, names)
        want = raw_equilibria_eq10(rho, uu, cs2)
        for nm in names:
            if sum(int(c) for c in nm) >= 3:
                assert mt[nm] == pytest.approx(want[nm], rel=1e-11, abs=1e-15), nm
        for i, nm in enumerate(("100", "010", "001")):
            assert mt[nm] == pytest.approx(rho * uu[i] + F[i] / 2, rel=1e-12, abs=1e-16)


@pytest.mark.parametrize("r,s,cs2,nu,n,fa,ga", [
    (1.0, 0.5, 1 / 12, 0.05, (1, 1, 32), 0, 2),
    (0.5, 2.0, 1 / 12, 0.02, (16, 32, 4), 2, 1),
])
def test_raw_shear_wave_decays_at_eq53_viscosity(oracle_mod, r, s, cs2, nu, n, fa, ga):
    """The raw-moment scheme carries the same transport coefficients (Eq. 53)."""
    wn, _ = oracle_mod.omega_from_viscosity(nu, cs2 / 3, cs2)
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=cs2, omega_nu=wn, omega_xi=1.0, model="raw")
    rho, u, k2 = synth.shear_wave(*n, r, s, 1e-3, fa, ga)
    f = o.init(rho, u)
    ts, amps = [], []
    for t in range(0, 401, 40):
        if t:
            f = o.run(f, 40)
        _, uu = o.moments(f)
        ts.append(t)
        amps.append(float(np.sum(uu * u) / np.sum(u * u)))
    assert fit_decay_rate(ts[1:], amps[1:]) / (k2 * nu) == pytest.approx(1.0, abs=5e-3)


@pytest.mark.parametrize("corr", ["NONE", "LOCAL", "FULL"])
def test_raw_and_central_agree_up_to_second_order(oracle_mod, corr):
    """The two schemes relax the same second-order non-equilibrium moments (raw and
    central ones coincide, Sec. 2.6) with sources that are binomial transforms of each
    other (Eq. 11 vs Eq. 11c), so their post-collision raw moments of order <= 2 are
    equal for any state and force; they differ above second order."""
    rng = np.random.default_rng(25)
    r, s = 0.5, 1.3
    kw = dict(r=r, s=s, cs2=0.07, omega_nu=1.6, omega_xi=1.2, corr=getattr(oracle_mod, "CORR_" + corr))
    oc = oracle_mod.Oracle(**kw)
    orw = oracle_mod.Oracle(model="raw", **kw)
    names = _names(oc)
    low = [nm for nm in names if sum(int(c) for c in nm) <= 2]
    high = [nm for nm in names if sum(int(c) for c in nm) >= 3]
    for _ in range(10):
        f = _rand_f(oc, rng, u_scale=0.08)
        F, g = 1e-3 * rng.standard_normal(3), 1e-2 * rng.standard_normal(3)
        mc = _raw_moments(oc.collide_node(f, F, g), r, s, names)
        mr = _raw_moments(orw.collide_node(f, F, g), r, s, names)
        for nm in low:
            assert mr[nm] == pytest.approx(mc[nm], rel=1e-12, abs=1e-16), nm
        assert max(abs(mr[nm] - mc[nm]) for nm in high) > 1e-9
