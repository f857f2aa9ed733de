"""Pins of the oracle's per-node collision (App. D) against invariants and special
cases fixed by the mathematics.  CPU only."""
import numpy as np
import pytest

import synth

MODES = ["NONE", "LOWMACH", "LOCAL", "FULL"]


def _mode(oracle_mod, name):
    return getattr(oracle_mod, "CORR_" + name)


def _cuboid_e(o, r, s):
    return o.velocities().astype(float) * np.array([[1.0], [r], [s]])


def _central(f, ec, u, m, n, p):
    return np.sum(f * (ec[0] - u[0]) ** m * (ec[1] - u[1]) ** n * (ec[2] - u[2]) ** p)


CASES = [(0.5, 2.0, 1 / 12), (1.0, 0.5, 0.10), (0.25, 1.0, 1 / 48), (0.406, 1.3, 0.04), (1.0, 1.0, 1 / 3)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("r,s,cs2", CASES)
def test_definitional_equals_factored(oracle_mod, mode, r, s, cs2):
    """Eq. 3a + LU (definitional) and P, S, F(u), F(-u), S^-1, P^-1 (Sec. 3.2) agree."""
    kw = dict(r=r, s=s, cs2=cs2, omega_nu=1.63, omega_xi=1.21, corr=_mode(oracle_mod, mode))
    o0, o1 = oracle_mod.Oracle(form=0, **kw), oracle_mod.Oracle(form=1, **kw)
    fs = synth.random_populations(6, seed=11)
    rng = np.random.default_rng(5)
    for f in fs:
        F = 1e-3 * rng.standard_normal(3)
        g = 1e-2 * rng.standard_normal(3)
        a, b = o0.collide_node(f, F, g), o1.collide_node(f, F, g)
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-13 * np.abs(a).max())


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("r,s,cs2", CASES[:4])
def test_mass_and_momentum_conservation(oracle_mod, mode, r, s, cs2):
    """Collision conserves mass and adds the body force to the momentum:
    sum f~ = sum f, sum f~ e = sum f e + F (k~_000 = k_000; k~_100 = F/2 with u
    carrying F/2; App. D with omega_1 = 1)."""
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=1.4, omega_xi=0.9, corr=_mode(oracle_mod, mode))
    ec = _cuboid_e(o, r, s)
    rng = np.random.default_rng(2)
    for f in synth.random_populations(5, seed=3):
        F = 1e-3 * rng.standard_normal(3)
        ft = o.collide_node(f, F, 1e-2 * rng.standard_normal(3))
        assert ft.sum() == pytest.approx(f.sum(), rel=1e-14)
        np.testing.assert_allclose(ec @ ft, ec @ f + F, rtol=0, atol=2e-15 * np.abs(f).sum())


@pytest.mark.parametrize("mode", MODES)
def test_equilibrium_is_fixed_point(oracle_mod, mode):
    """At F = 0 the Maxwellian-matched equilibrium (Eq. 9/10) is left unchanged: its
    non-equilibrium moments vanish, hence so do the recovered strain rates and the
    corrections."""
    o = oracle_mod.Oracle(r=0.5, s=0.5, cs2=1 / 12, omega_nu=1.78, omega_xi=1.0, corr=_mode(oracle_mod, mode))
    feq = o.equilibrium(1.02, [0.03, -0.02, 0.01])
    np.testing.assert_allclose(o.collide_node(feq), feq, rtol=1e-13, atol=1e-16)


def test_unit_rates_give_equilibrium(oracle_mod):
    """omega_nu = omega_xi = 1 and no corrections: every moment is replaced by its
    equilibrium, so f~ = f^eq(rho, u) for any f (F = 0)."""
    o = oracle_mod.Oracle(r=0.5, s=2.0, cs2=1 / 12, omega_nu=1.0, omega_xi=1.0, corr=oracle_mod.CORR_NONE)
    ec = _cuboid_e(o, 0.5, 2.0)
    for f in synth.random_populations(4, seed=8):
        rho = f.sum()
        u = ec @ f / rho
        np.testing.assert_allclose(o.collide_node(f), o.equilibrium(rho, u), rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("r,s,cs2", CASES[:3])
def test_relaxation_structure_of_central_moments(oracle_mod, r, s, cs2):
    """Without corrections, the central moments of f~ (computed here from the definition,
    Eq. 3a) are: k~_110 = (1-w_nu) k_110, deviatoric k~_2d = (1-w_nu) k_2d, trace
    k~_2s - 3 cs2 rho = (1-w_xi)(k_2s - 3 cs2 rho), k~_100 = F/2, third order 0,
    k~_220 = cs2^2 rho, k~_211 = 0, k~_222 = cs2^3 rho (App. D)."""
    wn, wb = 1.37, 0.83
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=wn, omega_xi=wb, corr=oracle_mod.CORR_NONE)
    ec = _cuboid_e(o, r, s)
    F = np.array([2e-4, -1e-4, 3e-4])
    for f in synth.random_populations(3, seed=21):
        rho = f.sum()
        u = (ec @ f + F / 2) / rho
        ft = o.collide_node(f, F)
        k = lambda m, n, p: _central(f, ec, u, m, n, p)
        kt = lambda m, n, p: _central(ft, ec, u, m, n, p)
        tol = 1e-13
        for (m, n, p) in [(1, 1, 0), (1, 0, 1), (0, 1, 1)]:
            assert kt(m, n, p) == pytest.approx((1 - wn) * k(m, n, p), abs=tol)
        assert kt(2, 0, 0) - kt(0, 2, 0) == pytest.approx((1 - wn) * (k(2, 0, 0) - k(0, 2, 0)), abs=tol)
        assert kt(2, 0, 0) - kt(0, 0, 2) == pytest.approx((1 - wn) * (k(2, 0, 0) - k(0, 0, 2)), abs=tol)
        tr = lambda g: g(2, 0, 0) + g(0, 2, 0) + g(0, 0, 2) - 3 * cs2 * rho
        assert tr(kt) == pytest.approx((1 - wb) * tr(k), abs=tol)
        for i, e in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
            assert kt(*e) == pytest.approx(F[i] / 2, abs=tol)
        for e in [(1, 2, 0), (1, 0, 2), (2, 1, 0), (0, 1, 2), (2, 0, 1), (0, 2, 1), (1, 1, 1),
                  (2, 1, 1), (1, 2, 1), (1, 1, 2), (1, 2, 2), (2, 1, 2), (2, 2, 1)]:
            assert kt(*e) == pytest.approx(0.0, abs=tol), e
        for e in [(2, 2, 0), (2, 0, 2), (0, 2, 2)]:
            assert kt(*e) == pytest.approx(cs2 ** 2 * rho, abs=tol)
        assert kt(2, 2, 2) == pytest.approx(cs2 ** 3 * rho, abs=tol)


def test_strain_rates_solve_the_3x3_system(oracle_mod):
    """The closed form of Eq. 49 (App. D) solves the linear system of Eq. 48 whose
    coefficients are those of Eq. 47 / App. D; checked with a library solver."""
    r, s, cs2, wn, wb = 0.5, 0.8, 0.06, 1.55, 1.1
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=wn, omega_xi=wb)
    rng = np.random.default_rng(4)
    for _ in range(5):
        rho = 1 + 0.01 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        gr = 0.01 * rng.standard_normal(3)
        k = 0.01 * rng.standard_normal(27)
        ex = o.moment_exponents()
        idx = {"%d%d%d" % tuple(ex[:, j]): j for j in range(27)}
        k[idx["200"]] += cs2 * rho; k[idx["020"]] += cs2 * rho; k[idx["002"]] += cs2 * rho
        d = o.strain_rates(k, rho, u, gr, aliasing=True)
        ux, uy, uz = u
        A, B, C = 0.5 * (3 * cs2 - 1) * ux, 0.5 * (3 * cs2 - r * r) * uy, 0.5 * (3 * cs2 - s * s) * uz
        k2s = k[idx["200"]] + k[idx["020"]] + k[idx["002"]]
        R = np.array([k[idx["200"]] - k[idx["020"]] - A * gr[0] + B * gr[1],
                      k[idx["200"]] - k[idx["002"]] - A * gr[0] + C * gr[2],
                      k2s - 3 * cs2 * rho - A * gr[0] - B * gr[1] - C * gr[2]])
        cx = lambda w: (-2 * cs2 / w + 0.5 * (3 * cs2 - 1) + 1.5 * ux * ux) * rho
        M = np.array([
            [cx(wn), (2 * cs2 / wn - 0.5 * (3 * cs2 - r * r) - 1.5 * uy * uy) * rho, 0.0],
            [cx(wn), 0.0, (2 * cs2 / wn - 0.5 * (3 * cs2 - s * s) - 1.5 * uz * uz) * rho],
            [cx(wb), (-2 * cs2 / wb + 0.5 * (3 * cs2 - r * r) + 1.5 * uy * uy) * rho,
             (-2 * cs2 / wb + 0.5 * (3 * cs2 - s * s) + 1.5 * uz * uz) * rho]])
        np.testing.assert_allclose(d, np.linalg.solve(M, R), rtol=1e-10, atol=1e-14)


def test_cubic_lattice_corrections_vanish(oracle_mod):
    """At r = s = 1 and cs2 = 1/3 the anisotropy factors (3 cs2 - c_i^2) vanish: the
    low-Mach corrections are identically zero (LOWMACH == NONE), and at zero velocity
    the aliasing part vanishes too (LOCAL == NONE).  The aliasing part of theta does
    not vanish at u != 0 (the paper's remark in Sec. 2.5 covers the anisotropy part)."""
    kw = dict(r=1.0, s=1.0, cs2=1 / 3, omega_nu=1.3, omega_xi=0.8)
    none = oracle_mod.Oracle(corr=oracle_mod.CORR_NONE, **kw)
    low = oracle_mod.Oracle(corr=oracle_mod.CORR_LOWMACH, **kw)
    loc = oracle_mod.Oracle(corr=oracle_mod.CORR_LOCAL, **kw)
    opp = [0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15, 26, 25, 24, 23, 22, 21, 20, 19]
    for f in synth.random_populations(4, seed=13):
        np.testing.assert_allclose(low.collide_node(f), none.collide_node(f), rtol=1e-14, atol=1e-16)
        fs = 0.5 * (f + f[opp])                       # zero momentum
        np.testing.assert_allclose(loc.collide_node(fs), none.collide_node(fs), rtol=1e-13, atol=1e-16)
        assert np.abs(loc.collide_node(f) - none.collide_node(f)).max() > 1e-9


def test_full_equals_local_without_density_gradient(oracle_mod):
    kw = dict(r=0.5, s=2.0, cs2=1 / 12, omega_nu=1.6, omega_xi=1.0)
    full = oracle_mod.Oracle(corr=oracle_mod.CORR_FULL, **kw)
    loc = oracle_mod.Oracle(corr=oracle_mod.CORR_LOCAL, **kw)
    for f in synth.random_populations(3, seed=17):
        np.testing.assert_allclose(full.collide_node(f, grad_rho=(0, 0, 0)), loc.collide_node(f), rtol=1e-15)
        assert np.abs(full.collide_node(f, grad_rho=(1e-2, 0, 0)) - loc.collide_node(f)).max() > 1e-8


def test_corrections_act_on_a_cuboid_lattice(oracle_mod):
    kw = dict(r=0.5, s=2.0, cs2=1 / 12, omega_nu=1.6, omega_xi=1.0)
    none = oracle_mod.Oracle(corr=oracle_mod.CORR_NONE, **kw)
    loc = oracle_mod.Oracle(corr=oracle_mod.CORR_LOCAL, **kw)
    f = synth.random_populations(1, seed=19)[0]
    assert np.abs(loc.collide_node(f) - none.collide_node(f)).max() > 1e-6


def _ce_moments(cs2, r, s, wn, wb, rho, u, gr, d):
    """Second-order non-equilibrium central moments predicted by the Chapman-Enskog
    analysis of Sec. 2.4-2.5 for prescribed diagonal strain rates d = (dxux, dyuy,
    dzuz), velocity u and density gradient gr: Eq. 33d-f with the error terms of
    Eq. 22a-f and the corrections fixed by Eq. 37, n_j^eq(1) = -(1 - w_j/2)(E_js + E_jg).
    Returns (n7, n8, n9, n7eq1, n8eq1, n9eq1)."""
    ux, uy, uz = u
    X, Y, Z = d
    dx_rux = rho * X + ux * gr[0]       # d(rho u_x)/dx
    dy_ruy = rho * Y + uy * gr[1]
    dz_ruz = rho * Z + uz * gr[2]
    a, b, c = 3 * cs2 - 1, 3 * cs2 - r * r, 3 * cs2 - s * s
    E7 = (a * dx_rux - b * dy_ruy) / wn + 3 * rho / wn * (ux * ux * X - uy * uy * Y)
    E8 = (a * dx_rux - c * dz_ruz) / wn + 3 * rho / wn * (ux * ux * X - uz * uz * Z)
    E9 = (a * dx_rux + b * dy_ruy + c * dz_ruz) / wb + 3 * rho / wb * (ux * ux * X + uy * uy * Y + uz * uz * Z)
    q7, q8, q9 = -(1 - wn / 2) * E7, -(1 - wn / 2) * E8, -(1 - wb / 2) * E9
    n7 = -2 * cs2 * rho / wn * (X - Y) + E7 + q7
    n8 = -2 * cs2 * rho / wn * (X - Z) + E8 + q8
    n9 = -2 * cs2 * rho / wb * (X + Y + Z) + E9 + q9
    return n7, n8, n9, q7, q8, q9


@pytest.mark.parametrize("r,s,cs2", [(0.5, 2.0, 1 / 12), (1.0, 0.5, 0.1), (0.406, 1.3, 0.04)])
def test_strain_rates_invert_the_chapman_enskog_moments(oracle_mod, r, s, cs2):
    """The local strain-rate formulas (Eq. 44-49, App. D; FULL with density gradients)
    recover the diagonal strain rates from the non-equilibrium moments that the
    Chapman-Enskog analysis (Eq. 22, 33, 37) predicts for them."""
    wn, wb = 1.45, 1.15
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=wn, omega_xi=wb, corr=oracle_mod.CORR_FULL)
    ex = o.moment_exponents()
    idx = {"%d%d%d" % tuple(ex[:, j]): j for j in range(27)}
    rng = np.random.default_rng(7)
    for _ in range(6):
        rho = 1 + 0.02 * rng.standard_normal()
        u = 0.06 * rng.standard_normal(3)
        gr = 0.01 * rng.standard_normal(3)
        d = 1e-3 * rng.standard_normal(3)
        n7, n8, n9, *_ = _ce_moments(cs2, r, s, wn, wb, rho, u, gr, d)
        # central moments with k200 - k020 = n7, k200 - k002 = n8, trace - 3 cs2 rho = n9
        k = np.zeros(27)
        k200 = cs2 * rho + (n9 + n7 + n8) / 3
        k[idx["200"]], k[idx["020"]], k[idx["002"]] = k200, k200 - n7, k200 - n8
        k[idx["000"]] = rho
        np.testing.assert_allclose(o.strain_rates(k, rho, u, gr, aliasing=True), d, rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("r,s,cs2", [(0.5, 2.0, 1 / 12), (1.0, 0.5, 0.1)])
def test_corrected_equilibria_cancel_the_truncation_errors(oracle_mod, r, s, cs2):
    """With the recovered strain rates, the correction of the combined equilibria built
    from the theta and lambda coefficients (Eq. 38-40; App. D) equals
    -(1 - omega/2)(E_s + E_g) of Eq. 37 with the error terms of Eq. 22."""
    wn, wb = 1.45, 1.15
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=wn, omega_xi=wb, corr=oracle_mod.CORR_FULL)
    ex = o.moment_exponents()
    idx = {"%d%d%d" % tuple(ex[:, j]): j for j in range(27)}
    rng = np.random.default_rng(9)
    for _ in range(6):
        rho = 1 + 0.02 * rng.standard_normal()
        u = 0.06 * rng.standard_normal(3)
        gr = 0.01 * rng.standard_normal(3)
        d = 1e-3 * rng.standard_normal(3)
        n7, n8, n9, q7, q8, q9 = _ce_moments(cs2, r, s, wn, wb, rho, u, gr, d)
        k = np.zeros(27)
        k200 = cs2 * rho + (n9 + n7 + n8) / 3
        k[idx["200"]], k[idx["020"]], k[idx["002"]] = k200, k200 - n7, k200 - n8
        k[idx["000"]] = rho
        kt = o.relax_central(k, rho, u, (0, 0, 0), gr)
        t7 = kt[idx["200"]] - kt[idx["020"]]
        t8 = kt[idx["200"]] - kt[idx["002"]]
        t9 = kt[idx["200"]] + kt[idx["020"]] + kt[idx["002"]] - 3 * cs2 * rho
        # k~ = k + w (k_eq - k)  ->  k_eq = (k~ - (1 - w) k) / w
        assert (t7 - (1 - wn) * n7) / wn == pytest.approx(q7, rel=1e-9, abs=1e-15)
        assert (t8 - (1 - wn) * n8) / wn == pytest.approx(q8, rel=1e-9, abs=1e-15)
        assert (t9 - (1 - wb) * n9) / wb == pytest.approx(q9, rel=1e-9, abs=1e-15)


def test_full_mode_density_gradient_is_exact_for_quadratics(oracle_mod):
    """FULL mode takes grad rho from second-order differences of the density field
    (central inside, one-sided next to a wall; spacings 1, r, s).  Second-order stencils
    are exact for a quadratic density, so every node of the lattice collision must equal
    the single-node collision given the analytic gradient (the lambda terms act through
    u . grad rho, so the velocity is non-zero)."""
    n, r, s = (6, 5, 7), 0.5, 1.3
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=0.06, omega_nu=1.6, omega_xi=1.2, corr=oracle_mod.CORR_FULL,
                          walls="xyz")
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    X, Y, Z = i * 1.0, j * r, k * s
    a, b, c, d, e, g = 2e-3, -1e-4, -3e-3, 2e-4, 1.5e-3, 1e-4
    rho = 1 + a * X + b * X ** 2 + c * Y + d * Y ** 2 + e * Z + g * Z ** 2
    rng = np.random.default_rng(31)
    u = 0.03 * rng.standard_normal((3,) + rho.shape)
    f = o.init(rho, u)
    ft = o.collide_all(f)
    changed = 0.0
    for (kk, jj, ii) in [(0, 0, 0), (n[2] - 1, n[1] - 1, n[0] - 1), (3, 2, 1), (1, 4, 5), (6, 0, 3), (2, 3, 0)]:
        grad = (a + 2 * b * X[kk, jj, ii], c + 2 * d * Y[kk, jj, ii], e + 2 * g * Z[kk, jj, ii])
        want = o.collide_node(f[:, kk, jj, ii], grad_rho=grad)
        np.testing.assert_allclose(ft[:, kk, jj, ii], want, rtol=1e-12, atol=1e-15)
        changed = max(changed, np.abs(want - o.collide_node(f[:, kk, jj, ii])).max())
    assert changed > 1e-9       # the gradient terms do act


def test_full_mode_density_gradient_wraps_on_periodic_axes(oracle_mod):
    """On periodic axes the central difference of rho = 1 + A sin(k x) is exactly
    A cos(k x) sin(k h) / h (wrap included); FULL-mode lattice collisions must equal the
    single-node collision given that gradient, at the first and last nodes as well."""
    n, r, s = (8, 6, 10), 0.5, 1.3
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=0.06, omega_nu=1.6, omega_xi=1.2, corr=oracle_mod.CORR_FULL)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    h = (1.0, r, s)
    kx, ky, kz = (2 * np.pi / (m * hh) for m, hh in zip(n, h))
    A = (2e-3, -1.5e-3, 1e-3)
    X, Y, Z = i * h[0], j * h[1], k * h[2]
    rho = 1 + A[0] * np.sin(kx * X) + A[1] * np.sin(ky * Y) + A[2] * np.sin(kz * Z)
    rng = np.random.default_rng(32)
    u = 0.03 * rng.standard_normal((3,) + rho.shape)
    f = o.init(rho, u)
    ft = o.collide_all(f)
    for (kk, jj, ii) in [(0, 0, 0), (n[2] - 1, n[1] - 1, n[0] - 1), (4, 2, 7), (9, 5, 0)]:
        grad = tuple(a_ * np.cos(kq * q[kk, jj, ii]) * np.sin(kq * hh) / hh
                     for a_, kq, q, hh in zip(A, (kx, ky, kz), (X, Y, Z), h))
        np.testing.assert_allclose(ft[:, kk, jj, ii], o.collide_node(f[:, kk, jj, ii], grad_rho=grad),
                                   rtol=1e-12, atol=1e-15)


def test_random_parameters_conservation_and_two_forms(oracle_mod):
    """Property test over random lattices and rates (both schemes, every correction mode):
    mass is conserved, momentum gains F, and the factored and definitional forms agree."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=60, deadline=None, derandomize=True)
    @hyp.given(r=st.floats(0.25, 2.0), s=st.floats(0.25, 2.0), frac=st.floats(0.15, 0.9),
               wn=st.floats(0.2, 1.95), wb=st.floats(0.2, 1.95), mode=st.sampled_from(MODES),
               model=st.sampled_from(["central", "raw"]), seed=st.integers(0, 2 ** 31 - 1))
    def check(r, s, frac, wn, wb, mode, model, seed):
        cs2 = frac * min(1.0, r * r, s * s)           # positive rest weights need cs2 < min(1, r^2, s^2)
        kw = dict(r=r, s=s, cs2=cs2, omega_nu=wn, omega_xi=wb, corr=getattr(oracle_mod, "CORR_" + mode), model=model)
        a = oracle_mod.Oracle(form=0, **kw)
        b = oracle_mod.Oracle(form=1, **kw)
        rng = np.random.default_rng(seed)
        u = 0.05 * rng.standard_normal(3) * np.array([1.0, r, s])
        f = a.equilibrium(1.0 + 0.02 * rng.standard_normal(), u)
        f = f * (1.0 + 0.01 * rng.standard_normal(27))
        F = 1e-4 * rng.standard_normal(3)
        g = 1e-2 * rng.standard_normal(3)
        fa, fb = a.collide_node(f, F, g), b.collide_node(f, F, g)
        np.testing.assert_allclose(fa, fb, rtol=1e-9, atol=1e-13 * np.abs(f).max())
        e = np.array([[1.0], [r], [s]]) * a.velocities()
        assert fa.sum() == pytest.approx(f.sum(), rel=1e-13)
        np.testing.assert_allclose(e @ fa, e @ f + F, rtol=0, atol=1e-13)
    check()
