"""Differentiable FP64 reference of the cuboid D3Q27 central-moment scheme in plain
PyTorch CPU ops (test infrastructure only; see the package docstring).

A third implementation of the forward update, written from the paper in its
definitional form and vectorised over nodes, so that torch.autograd gives the
exact gradient of a flow objective for checking the hand-written adjoint:

  * central moments by their definition, k_mnp = sum_a f_a (e_ax-u_x)^m
    (e_ay-u_y)^n (e_az-u_z)^p with the cuboid velocities (Eq. 1a-1c, Eq. 3a) and
    rho u = sum f e + F/2 (Eq. 12);
  * relaxation of App. D: combined moments B, corrected second-order equilibria
    (Eq. 63 with the coefficients of Eq. 38-40), strain rates of Eq. 44-49,
    every rate other than omega_nu, omega_xi equal to 1, then B^-1;
  * post-collision populations by solving M(u) f~ = k~ (batched linear solve);
  * streaming f_a(x, t+1) = f~_a(x - e_a, t) with half-way bounce-back walls (Sec. 4).

Only the correction modes NONE, LOWMACH and LOCAL are provided (no density
gradients).  Everything is torch.float64 on the CPU.
"""
from __future__ import annotations

import itertools

import numpy as np
import torch

# cubic D3Q27 velocities in the paper's ordering (Eq. 1a-1c with r = s = 1)
EX = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1]
EY = [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1]
EZ = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1]
# the 27 exponent triples (any order works for the definitional form)
EXPONENTS = list(itertools.product(range(3), repeat=3))
IDX = {e: i for i, e in enumerate(EXPONENTS)}
OPP = [next(b for b in range(27) if (EX[b], EY[b], EZ[b]) == (-EX[a], -EY[a], -EZ[a])) for a in range(27)]


def _velocities(r, s):
    return torch.tensor([EX, [r * v for v in EY], [s * v for v in EZ]], dtype=torch.float64)


def central_matrix(u, r, s):
    """M[n, j, a] = (e_ax-u_x)^m (e_ay-u_y)^p (e_az-u_z)^q for exponents j = (m,p,q); u: [3, N]."""
    e = _velocities(r, s)
    d = e[:, :, None] - u[:, None, :]          # [3, 27, N]
    rows = []
    for (m, p, q) in EXPONENTS:
        rows.append(d[0] ** m * d[1] ** p * d[2] ** q)
    return torch.stack(rows, dim=0).permute(2, 0, 1)   # [N, 27 moments, 27 dirs]


def collide(f, F, r, s, cs2, omega_nu, omega_xi, corr="local"):
    """Post-collision populations for populations f [27, N] and force F [3, N]."""
    e = _velocities(r, s)
    rho = f.sum(0)
    u = (e @ f + 0.5 * F) / rho
    M = central_matrix(u, r, s)                                  # [N, 27, 27]
    k = torch.einsum("nja,an->jn", M, f)                          # central moments [27, N]
    K = lambda m, p, q: k[IDX[(m, p, q)]]
    wn, wb = omega_nu, omega_xi
    k2s = K(2, 0, 0) + K(0, 2, 0) + K(0, 0, 2)
    k2d1 = K(2, 0, 0) - K(0, 2, 0)
    k2d2 = K(2, 0, 0) - K(0, 0, 2)
    ux, uy, uz = u
    if corr == "none":
        eq2s, eq2d1, eq2d2 = 3 * cs2 * rho, torch.zeros_like(rho), torch.zeros_like(rho)
    else:
        al = 0.0 if corr == "lowmach" else 1.0
        cx, cy, cz = 3 * cs2 - 1.0, 3 * cs2 - r * r, 3 * cs2 - s * s
        # Eq. 47 / App. D coefficients and the right-hand sides (no density gradients)
        Csx = (-2 * cs2 / wn + 0.5 * cx + 1.5 * al * ux ** 2) * rho
        Cbx = (-2 * cs2 / wb + 0.5 * cx + 1.5 * al * ux ** 2) * rho
        Csy = (2 * cs2 / wn - 0.5 * cy - 1.5 * al * uy ** 2) * rho
        Cby = (-2 * cs2 / wb + 0.5 * cy + 1.5 * al * uy ** 2) * rho
        Csz = (2 * cs2 / wn - 0.5 * cz - 1.5 * al * uz ** 2) * rho
        Cbz = (-2 * cs2 / wb + 0.5 * cz + 1.5 * al * uz ** 2) * rho
        Rb, Rs1, Rs2 = k2s - 3 * cs2 * rho, k2d1, k2d2
        # the 3x3 system of Eq. 48 solved per node (library solve, not the Cramer form)
        zero = torch.zeros_like(rho)
        A = torch.stack([torch.stack([Csx, Csy, zero], -1), torch.stack([Csx, zero, Csz], -1),
                         torch.stack([Cbx, Cby, Cbz], -1)], -2)
        dux = torch.linalg.solve(A, torch.stack([Rs1, Rs2, Rb], -1).unsqueeze(-1)).squeeze(-1)
        dxux, dyuy, dzuz = dux[:, 0], dux[:, 1], dux[:, 2]
        tn, tb = 1 / wn - 0.5, 1 / wb - 0.5
        th = lambda c, uu, t: -rho * (3 * al * uu ** 2 + c) * t
        eq2s = 3 * cs2 * rho + th(cx, ux, tb) * dxux + th(cy, uy, tb) * dyuy + th(cz, uz, tb) * dzuz
        eq2d1 = th(cx, ux, tn) * dxux - th(cy, uy, tn) * dyuy
        eq2d2 = th(cx, ux, tn) * dxux - th(cz, uz, tn) * dzuz
    t2s = k2s + wb * (eq2s - k2s)
    t2d1 = k2d1 + wn * (eq2d1 - k2d1)
    t2d2 = k2d2 + wn * (eq2d2 - k2d2)
    kt = [None] * 27
    for (m, p, q) in EXPONENTS:
        order = m + p + q
        # equilibrium values (Eq. 9): rho, 0, cs2 rho, cs2^2 rho, cs2^3 rho
        ones = [m, p, q].count(1)
        twos = [m, p, q].count(2)
        eq = torch.zeros_like(rho) if ones else rho * cs2 ** twos
        kt[IDX[(m, p, q)]] = eq     # every other rate is 1: moment := equilibrium
    # first order: k~_100 = k + (0 - k) + (1 - 1/2) F = F/2
    kt[IDX[(1, 0, 0)]], kt[IDX[(0, 1, 0)]], kt[IDX[(0, 0, 1)]] = 0.5 * F[0], 0.5 * F[1], 0.5 * F[2]
    kt[IDX[(1, 1, 0)]] = (1 - wn) * K(1, 1, 0)
    kt[IDX[(1, 0, 1)]] = (1 - wn) * K(1, 0, 1)
    kt[IDX[(0, 1, 1)]] = (1 - wn) * K(0, 1, 1)
    kt[IDX[(2, 0, 0)]] = (t2s + t2d1 + t2d2) / 3
    kt[IDX[(0, 2, 0)]] = (t2s - 2 * t2d1 + t2d2) / 3
    kt[IDX[(0, 0, 2)]] = (t2s + t2d1 - 2 * t2d2) / 3
    kt = torch.stack(kt, 0)                                       # [27, N]
    ft = torch.linalg.solve(M, kt.T.unsqueeze(-1)).squeeze(-1)    # [N, 27]
    return ft.T


def stream_indices(nx, ny, nz, walls=""):
    """For every (direction a, node x): the flat index into [27 * N] of the
    post-collision value that streams into f_a(x) (Sec. 3.2 and half-way
    bounce-back of Sec. 4)."""
    N = nx * ny * nz
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = [x.ravel(), y.ravel(), z.ravel()]
    n = [nx, ny, nz]
    idx = np.empty((27, N), dtype=np.int64)
    for a in range(27):
        e = [EX[a], EY[a], EZ[a]]
        src = [c[i] - e[i] for i in range(3)]
        out = np.zeros(N, dtype=bool)
        for i in range(3):
            beyond = (src[i] < 0) | (src[i] >= n[i])
            if "xyz"[i] in walls:
                out |= beyond
            src[i] = np.mod(src[i], n[i])
        node = (src[2] * ny + src[1]) * nx + src[0]
        self_node = (c[2] * ny + c[1]) * nx + c[0]
        idx[a] = np.where(out, OPP[a] * N + self_node, a * N + node)
    return torch.from_numpy(idx)


def run(f0, force, r, s, cs2, omega_nu, omega_xi, steps, shape, walls="", corr="local"):
    """`steps` fused updates of f0 [27, N] with a per-node force [3, N]."""
    idx = stream_indices(*shape, walls=walls)
    f = f0
    for _ in range(steps):
        ft = collide(f, force, r, s, cs2, omega_nu, omega_xi, corr)
        f = ft.reshape(-1)[idx]
    return f


def mean_kinetic_energy(f, force, r, s):
    """J = (1/N) sum_x |j|^2 / (2 rho), j = sum f e + F/2."""
    e = _velocities(r, s)
    rho = f.sum(0)
    j = e @ f + 0.5 * force
    return (0.5 * (j * j).sum(0) / rho).mean()


def equilibrium(rho, u, r, s, cs2):
    """f^eq solving M(u) f = k^eq(rho) (Eq. 9): populations [27, N]."""
    M = central_matrix(u, r, s)
    keq = []
    for (m, p, q) in EXPONENTS:
        keq.append(torch.zeros_like(rho) if 1 in (m, p, q) else rho * cs2 ** [m, p, q].count(2))
    keq = torch.stack(keq, 0)
    return torch.linalg.solve(M, keq.T.unsqueeze(-1)).squeeze(-1).T
