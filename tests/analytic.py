"""Closed-form solutions used as pins (not part of the method).

Each function cites the passage of arXiv:2107.14774 that states the solution.
"""
import numpy as np


def duct_series(y, z, a, b, F, rho, nu, nterms=201):
    """Fully developed flow in a rectangular duct |y| <= a, |z| <= b driven by a
    body force F along x: the separation-of-variables solution of
    nu (u_yy + u_zz) = -F / rho with u = 0 on the walls.  For a = b = L/2 it is
    the square-duct series of Eq. 70 (Sec. 5.1) with the exponent of (-1) read as
    (n-1)/2."""
    y = np.asarray(y, dtype=float)
    z = np.asarray(z, dtype=float)
    u = np.zeros(np.broadcast(y, z).shape)
    for n in range(1, 2 * nterms, 2):
        k = n * np.pi / (2 * a)
        # cosh ratio written with exponentials of non-positive arguments (no overflow)
        ratio = (np.exp(k * (np.abs(z) - b)) + np.exp(-k * (np.abs(z) + b))) / (1 + np.exp(-2 * k * b))
        u += (-1) ** ((n - 1) // 2) / n ** 3 * (1 - ratio) * np.cos(k * y)
    return 16 * a * a * F / (rho * nu * np.pi ** 3) * u


def raw_equilibria_eq10(rho, u, cs2):
    """Raw-moment equilibria k'^eq_mnp exactly as printed in Eq. 10 (Sec. 2.3),
    keyed by the exponent string 'mnp'."""
    ux, uy, uz = u
    c2, c4, c6 = cs2, cs2 * cs2, cs2 ** 3
    return {
        "000": rho, "100": rho * ux, "010": rho * uy, "001": rho * uz,
        "110": rho * ux * uy, "101": rho * ux * uz, "011": rho * uy * uz,
        "200": c2 * rho + rho * ux ** 2, "020": c2 * rho + rho * uy ** 2, "002": c2 * rho + rho * uz ** 2,
        "120": c2 * rho * ux + rho * ux * uy ** 2, "102": c2 * rho * ux + rho * ux * uz ** 2,
        "210": c2 * rho * uy + rho * ux ** 2 * uy, "012": c2 * rho * uy + rho * uy * uz ** 2,
        "201": c2 * rho * uz + rho * ux ** 2 * uz, "021": c2 * rho * uz + rho * uy ** 2 * uz,
        "111": rho * ux * uy * uz,
        "220": c4 * rho + rho * c2 * (ux ** 2 + uy ** 2) + rho * ux ** 2 * uy ** 2,
        "202": c4 * rho + rho * c2 * (ux ** 2 + uz ** 2) + rho * ux ** 2 * uz ** 2,
        "022": c4 * rho + rho * c2 * (uy ** 2 + uz ** 2) + rho * uy ** 2 * uz ** 2,
        "211": rho * (c2 + ux ** 2) * uy * uz, "121": rho * (c2 + uy ** 2) * ux * uz,
        "112": rho * (c2 + uz ** 2) * ux * uy,
        "122": c4 * rho * ux + rho * c2 * ux * (uy ** 2 + uz ** 2) + rho * ux * uy ** 2 * uz ** 2,
        "212": c4 * rho * uy + rho * c2 * uy * (ux ** 2 + uz ** 2) + rho * ux ** 2 * uy * uz ** 2,
        "221": c4 * rho * uz + rho * c2 * uz * (ux ** 2 + uy ** 2) + rho * ux ** 2 * uy ** 2 * uz,
        "222": c6 * rho + rho * c4 * (ux ** 2 + uy ** 2 + uz ** 2)
        + rho * c2 * (ux ** 2 * uy ** 2 + uy ** 2 * uz ** 2 + ux ** 2 * uz ** 2) + rho * ux ** 2 * uy ** 2 * uz ** 2,
    }


def lid_bounce_coefficients_eq69(r, s, cs2):
    """Wall terms of the momentum-augmented bounce-back printed in Eq. 69 (Sec. 4)
    for a lid moving with speed U along x: incoming direction -> (outgoing
    direction, coefficient c) with f_in(t+1) = f~_out(t) + c rho U.  The printed
    f_25 row names f~_24 as the outgoing population; direction 25 = (1,-r,-s) is
    the opposite of 20 = (-1,r,s), so f~_20 is used (reading)."""
    a = (cs2 - s * s) * cs2 / (2 * r * r * s * s)
    b = cs2 * cs2 / (4 * r * r * s * s)
    return {4: (3, 0.0), 16: (17, 0.0), 18: (15, 0.0), 9: (8, -a), 10: (7, +a),
            21: (24, +b), 22: (23, -b), 25: (20, +b), 26: (19, -b)}


def fit_decay_rate(times, amps):
    """Least-squares slope of -log(amplitude) against time."""
    t = np.asarray(times, dtype=float)
    la = np.log(np.abs(np.asarray(amps, dtype=float)))
    A = np.vstack([t, np.ones_like(t)]).T
    slope, _ = np.linalg.lstsq(A, la, rcond=None)[0]
    return -slope


def pulsatile_duct(y, z, t, a, Fm, omega, nu, rho=1.0, nterms=200):
    """Time-periodic flow in the square duct |y|, |z| <= a driven by F = Fm cos(omega t)
    along x (Sec. 5.2, its analytical solution): u = Re[U e^{i omega t}],
    U = Fm/(i omega rho) (1 - V), V = 2 sum_n (-1)^n / p_n [cosh(g_n y/a) cos(p_n z/a)
    + cosh(g_n z/a) cos(p_n y/a)] / cosh(g_n), p_n = (2n+1) pi / 2,
    g_n = sqrt(p_n^2 + i Wo^2), Wo = a sqrt(omega / nu).  Readings of the garbled print:
    the prefactor is Fm/(i omega) (the printed Fm/omega lacks the i that makes the
    core oscillate as (Fm/omega) sin(omega t)) and 1/p^n is 1/p_n."""
    y = np.asarray(y, dtype=float)
    z = np.asarray(z, dtype=float)
    wo2 = a * a * omega / nu
    V = np.zeros(np.broadcast(y, z).shape, dtype=complex)
    for n in range(nterms):
        p = (2 * n + 1) * np.pi / 2
        g = np.sqrt(p * p + 1j * wo2)
        # cosh(g q/a)/cosh(g) written with decaying exponentials (|q| <= a, Re g > 0)
        ch = lambda q: (np.exp(g * (np.abs(q) / a - 1)) + np.exp(-g * (np.abs(q) / a + 1))) / (1 + np.exp(-2 * g))
        V += 2 * (-1) ** n / p * (ch(y) * np.cos(p * z / a) + ch(z) * np.cos(p * y / a))
    U = Fm / (1j * omega * rho) * (1 - V)
    return np.real(U * np.exp(1j * omega * t))
