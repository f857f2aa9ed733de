"""Seeded synthetic inputs shared by the oracle-side and CUDA-side tests and the bench.

This module holds NONE of the lattice Boltzmann arithmetic: it only produces
initial density/velocity fields and body-force fields (numpy, float64) with the
shapes and statistics of the paper's workloads.  Both the oracle and the CUDA
library are fed the identical arrays.

Coordinates are physical lattice units: node (i, j, k) sits at
x = i, y = j*r, z = k*s (Sec. 2.1: dx = 1, dy = r, dz = s).  Arrays are
``[nz][ny][nx]`` (density) and ``[3][nz][ny][nx]`` (velocity / force), x fastest.
"""
from __future__ import annotations

import numpy as np


def _coords(nx, ny, nz, r, s):
    z, y, x = np.meshgrid(np.arange(nz) * s, np.arange(ny) * r, np.arange(nx) * 1.0, indexing="ij")
    return x, y, z


def taylor_green_3d(nx, ny, nz, r, s, u0, modes=(1, 1, 1)):
    """3-D Taylor-Green field u = u0 (Ax cos kx x sin ky y sin kz z, Ay sin cos sin,
    Az sin sin cos), k = 2 pi modes / L_phys, amplitude vector A = (1, 1, -(kx+ky)/kz)
    so that A.k = 0 (divergence free).  Returns (rho, u, k)."""
    x, y, z = _coords(nx, ny, nz, r, s)
    L = np.array([nx * 1.0, ny * r, nz * s])
    k = 2 * np.pi * np.array(modes, dtype=float) / L
    A = np.array([1.0, 1.0, -(k[0] + k[1]) / k[2]])
    u = np.empty((3, nz, ny, nx))
    u[0] = A[0] * np.cos(k[0] * x) * np.sin(k[1] * y) * np.sin(k[2] * z)
    u[1] = A[1] * np.sin(k[0] * x) * np.cos(k[1] * y) * np.sin(k[2] * z)
    u[2] = A[2] * np.sin(k[0] * x) * np.sin(k[1] * y) * np.cos(k[2] * z)
    u *= u0
    return np.ones((nz, ny, nx)), u, k


def taylor_green_2d(nx, ny, nz, r, s, u0, plane="xy"):
    """Plane Taylor-Green vortex from the stream function psi = sin(k_a a) sin(k_b b)
    in the chosen plane ("xy", "xz" or "yz"); one wavelength per box side.
    Returns (rho, u, k_squared)."""
    x, y, z = _coords(nx, ny, nz, r, s)
    c = {"x": x, "y": y, "z": z}
    L = {"x": nx * 1.0, "y": ny * r, "z": nz * s}
    ia, ib = "xyz".index(plane[0]), "xyz".index(plane[1])
    a, b = plane[0], plane[1]
    ka, kb = 2 * np.pi / L[a], 2 * np.pi / L[b]
    u = np.zeros((3, nz, ny, nx))
    # u_a = d psi / d b, u_b = - d psi / d a, normalised to peak u0
    kk = max(ka, kb)
    u[ia] = u0 * (kb / kk) * np.sin(ka * c[a]) * np.cos(kb * c[b])
    u[ib] = -u0 * (ka / kk) * np.cos(ka * c[a]) * np.sin(kb * c[b])
    return np.ones((nz, ny, nx)), u, ka * ka + kb * kb


def shear_wave(nx, ny, nz, r, s, u0, flow_axis=0, grad_axis=2):
    """u_flow = u0 sin(k g) with g the coordinate along grad_axis; one wavelength."""
    x, y, z = _coords(nx, ny, nz, r, s)
    g = (x, y, z)[grad_axis]
    L = (nx * 1.0, ny * r, nz * s)[grad_axis]
    k = 2 * np.pi / L
    u = np.zeros((3, nz, ny, nx))
    u[flow_axis] = u0 * np.sin(k * g)
    return np.ones((nz, ny, nx)), u, k * k


def solenoidal_random(nx, ny, nz, r, s, k0, u_rms, seed):
    """Random divergence-free velocity with energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2),
    k in units of the fundamental mode of the physical box, random phases, projected
    with (I - k k^T/|k|^2) on the physical wavevectors, scaled to the given rms."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    L = np.array([nx * 1.0, ny * r, nz * s])
    kz = np.fft.fftfreq(nz, d=s) * 2 * np.pi
    ky = np.fft.fftfreq(ny, d=r) * 2 * np.pi
    kx = np.fft.fftfreq(nx, d=1.0) * 2 * np.pi
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    kmag = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    kfund = 2 * np.pi / L.max()
    kn = kmag / kfund
    amp = np.where(kmag > 0, kn ** 2 * np.exp(-(kn / k0) ** 2), 0.0)  # sqrt(E(k)/k^2) shape
    amp = amp / np.maximum(kn, 1e-30)
    uh = np.empty((3, nz, ny, nx), dtype=np.complex128)
    for c in range(3):
        phase = rng.uniform(0, 2 * np.pi, size=kmag.shape)
        mag = rng.standard_normal(size=kmag.shape)
        uh[c] = amp * mag * np.exp(1j * phase)
    kv = np.stack([KX, KY, KZ])
    k2 = np.where(kmag > 0, kmag ** 2, 1.0)
    kdotu = (kv * uh).sum(0)
    uh = uh - kv * kdotu / k2
    u = np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))
    # remove the mean and rescale to the requested rms of |u|
    u -= u.mean(axis=(1, 2, 3), keepdims=True)
    rms = np.sqrt((u ** 2).sum(0).mean())
    u *= u_rms / rms
    return np.ones((nz, ny, nx)), u


def force_field(nx, ny, nz, sigma, seed):
    """Per-node body force, i.i.d. N(0, sigma^2) per component."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    return sigma * rng.standard_normal((3, nz, ny, nx))


def random_direction(shape, norm, seed):
    """A seeded random direction with the given Euclidean norm."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    v = rng.standard_normal(shape)
    return v * (norm / np.linalg.norm(v))


def channel(nx, ny, nz, r, s, u_max, nu, amp, seed):
    """Wall-bounded channel (walls normal to y): laminar Poiseuille base flow with
    centre-line speed u_max plus a divergence-free perturbation (random solenoidal
    field damped by sin(pi y / h)) of relative amplitude amp.  The walls sit half a
    spacing outside the first and last node rows.  Returns (rho, u, Fx) with the
    driving force Fx = 8 nu u_max / h^2 of the base flow."""
    h = ny * r
    _, y, _ = _coords(nx, ny, nz, r, s)
    yw = y + 0.5 * r                     # distance from the lower wall
    u = np.zeros((3, nz, ny, nx))
    u[0] = 4 * u_max * yw * (h - yw) / h ** 2
    _, up = solenoidal_random(nx, ny, nz, r, s, 4.0, 1.0, seed)
    damp = np.sin(np.pi * yw / h)
    up *= damp
    up *= amp * u_max / np.sqrt((up ** 2).sum(0).mean())
    u += up
    return np.ones((nz, ny, nx)), u, 8 * nu * u_max / h ** 2


def random_populations(n, seed, scale=0.05):
    """Positive random population-like vectors for single-node checks: the
    27 weights of a random positive distribution (n x 27)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    return np.abs(1.0 + scale * rng.standard_normal((n, 27))) * rng.uniform(0.01, 0.1, size=(n, 27))
