"""Pins of the oracle's moment transforms (Sec. 3.1, Apps. A-C, E-G) against what
the paper prints and what the mathematics fixes.  CPU only."""
import os
from fractions import Fraction

import numpy as np
import pytest

from tests.analytic import raw_equilibria_eq10

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _names(o):
    e = o.moment_exponents()
    return ["%d%d%d" % tuple(e[:, j]) for j in range(27)]


def test_velocity_set_and_opposites(oracle_mod):
    e = oracle_mod.Oracle.velocities()
    # the 27 cubic velocities are exactly {-1,0,1}^3, each once (Eq. 1a-1c with r = s = 1)
    assert sorted(map(tuple, e.T.tolist())) == sorted(
        (a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
    assert tuple(e[:, 0]) == (0, 0, 0)
    # opposite pairs used by bounce-back: 1<->2, 3<->4, 5<->6 (Sec. 4 pairs 3/4, 8/9, 7/10, 17/16 ...)
    for a, b in [(1, 2), (3, 4), (5, 6), (8, 9), (7, 10), (17, 16), (15, 18), (24, 21), (23, 22),
                 (20, 25), (19, 26)]:
        assert np.all(e[:, a] == -e[:, b])


def test_scaling_matches_eq59(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "eq59_scaling.txt")) if l.strip() and l[0] != "#"]
    r, s = 0.37, 1.9
    want = np.array([r ** int(a) * s ** int(b) for a, b in rows])
    o = oracle_mod.Oracle(r=r, s=s, cs2=0.04)
    np.testing.assert_allclose(o.S(), want, rtol=1e-15)


def test_P_rows_match_appendix_A(oracle_mod):
    o = oracle_mod.Oracle()
    P, names = o.P(), _names(o)
    assert np.all(P[0] == 1.0)  # k'000 sums every population
    for line in open(os.path.join(GOLDEN, "appA_rows.txt")):
        if not line.strip() or line[0] == "#":
            continue
        tok = line.split()
        want = np.zeros(27)
        for t in tok[1:]:
            want[int(t[1:])] = 1.0 if t[0] == "+" else -1.0
        np.testing.assert_array_equal(P[names.index(tok[0][1:])], want, err_msg=tok[0])


def test_Pinv_rows_match_appendix_G_and_invert_P(oracle_mod):
    o = oracle_mod.Oracle()
    P, Pi, names = o.P(), o.Pinv(), _names(o)
    np.testing.assert_allclose(Pi @ P, np.eye(27), atol=1e-15)
    # P^-1 has dyadic-rational entries: every entry times 8 is an integer
    np.testing.assert_allclose(Pi * 8, np.round(Pi * 8), atol=1e-14)
    for line in open(os.path.join(GOLDEN, "appG_rows.txt")):
        if not line.strip() or line[0] == "#":
            continue
        tok = line.split()
        a, fac = int(tok[0][1:]), float(Fraction(tok[1]))
        want = np.zeros(27)
        for t in tok[2:]:
            want[names.index(t[1:])] = fac if t[0] == "+" else -fac
        np.testing.assert_allclose(Pi[a], want, atol=1e-15, err_msg=tok[0])


def test_Q_equals_SP_and_M_equals_FSP(oracle_mod):
    """Eq. 58: Q = S P, with Q the monomials of the cuboid velocities (Eq. 57);
    Eq. 3a: the central-moment matrix is F(u) Q."""
    r, s = 0.5, 2.0
    o = oracle_mod.Oracle(r=r, s=s, cs2=1 / 12)
    e = o.velocities().astype(float)
    ec = e * np.array([[1.0], [r], [s]])
    ex = o.moment_exponents()
    Q = np.array([[ec[0, a] ** ex[0, j] * ec[1, a] ** ex[1, j] * ec[2, a] ** ex[2, j] for a in range(27)]
                  for j in range(27)])
    np.testing.assert_allclose(np.diag(o.S()) @ o.P(), Q, rtol=1e-15, atol=1e-15)
    u = np.array([0.031, -0.017, 0.008])
    np.testing.assert_allclose(o.F(u) @ Q, o.M(u), rtol=1e-13, atol=1e-15)


def test_frame_transform_inverse_and_triangularity(oracle_mod):
    o = oracle_mod.Oracle()
    u = np.array([0.2, -0.15, 0.07])
    F, Fm = o.F(u), o.F(-u)
    np.testing.assert_allclose(F @ Fm, np.eye(27), atol=1e-15)   # F^-1 = F(-u) (App. E)
    ex = o.moment_exponents()
    # lower triangular in the product order: entry (i, j) is zero unless j <= i componentwise
    for i in range(27):
        for j in range(27):
            if np.any(ex[:, j] > ex[:, i]):
                assert F[i, j] == 0.0
    assert np.all(np.diag(F) == 1.0)


def test_raw_equilibria_match_eq10(oracle_mod):
    """F(-u) applied to the central equilibria of Eq. 9 gives the raw equilibria printed in Eq. 10."""
    o = oracle_mod.Oracle(cs2=0.07)
    rho, u = 1.013, np.array([0.04, -0.03, 0.025])
    m = o.F(-u) @ o.central_equilibrium(rho)
    want = raw_equilibria_eq10(rho, u, 0.07)
    for j, name in enumerate(_names(o)):
        assert m[j] == pytest.approx(want[name], rel=1e-14, abs=1e-17), name


def test_equilibrium_product_form(oracle_mod):
    """f^eq = Q^-1 m^eq equals rho * prod_i phi(e_i; c_i, u_i) with
    phi(0) = 1 - (cs2 + u^2)/c^2, phi(+-1) = ((cs2 + u^2)/c^2 +- u/c)/2: the 1-D
    three-velocity distribution with moments (1, u, cs2 + u^2) per axis."""
    r, s, cs2 = 0.5, 0.8, 0.06
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2)
    rho, u = 0.97, np.array([0.05, -0.02, 0.03])
    e = o.velocities()
    c = (1.0, r, s)

    def phi(v, ci, ui):
        t = (cs2 + ui * ui) / (ci * ci)
        return 1.0 - t if v == 0 else 0.5 * (t + v * ui / ci)

    want = np.array([rho * np.prod([phi(e[i, a], c[i], u[i]) for i in range(3)]) for a in range(27)])
    np.testing.assert_allclose(o.equilibrium(rho, u), want, rtol=1e-13)
    o1 = oracle_mod.Oracle(r=r, s=s, cs2=cs2, form=1)
    np.testing.assert_allclose(o1.equilibrium(rho, u), want, rtol=1e-12)


def test_table1_viscosity_relation(oracle_mod):
    """Eq. 53, nu = cs2 (1/omega_nu - 1/2), reproduces every row of Table 1."""
    for line in open(os.path.join(GOLDEN, "table1_duct.txt")):
        if not line.strip() or line[0] == "#":
            continue
        _, r, s, Fx, cs2, tau, nu = line.split()
        wn, _ = oracle_mod.omega_from_viscosity(float(nu), 0.01, float(cs2))
        assert 1.0 / wn == pytest.approx(float(tau), rel=1e-12)
