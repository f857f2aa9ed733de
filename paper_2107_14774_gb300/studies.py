"""Parameter studies of the paper run through the library (no numerics of their own).

* Sec. 7: the largest lid velocity that a lid-driven cubic cavity tolerates for a given
  number of steps, for the central-moment (3DCCM) and the raw-moment (3DCRM) scheme, as a
  function of omega_nu (Fig. 8) and omega_xi (Fig. 9); the largest stable Reynolds number
  at a fixed lid velocity (Fig. 10).
* Sec. 6: the lid-driven shallow cavity (L/H = 4, W/H = 2, Re = U L / nu = 100) on the
  cubic lattice and on cuboid lattices with about 5-8 times fewer nodes: centreline
  velocity profiles, node counts and run times.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from .lattice import Lattice


def lid_cavity(nx, ny, nz, r, s, cs2, U, omega_nu, omega_xi=1.0, model="central", storage="f32", corr="local"):
    """Closed box (walls on every axis) with the wall at y = ny - 1/2 moving along x at U,
    at rest with unit density, on its own stream (lb_step then replays CUDA graphs)."""
    lat = Lattice(nx, ny, nz, r_y=r, r_z=s, nu=0.01, cs2=cs2, storage=storage, walls="xyz", lid_u=U,
                  model=model, corr=corr, stream=torch.cuda.Stream())
    lat.set_rates(omega_nu, omega_xi)
    dt = torch.float64 if storage == "f64" else torch.float32
    lat.init(torch.ones((nz, ny, nx), dtype=dt, device=lat.device),
             torch.zeros((3, nz, ny, nx), dtype=dt, device=lat.device))
    return lat


def survives(lat, steps, check_every=5000, lid_u=0.0, ramp_steps=0, ramp_every=100) -> bool:
    """Run up to `steps` steps, stopping at the first check that finds a non-positive or
    non-finite density.  With ramp_steps > 0 the lid starts at rest and its velocity rises
    linearly to lid_u over the first ramp_steps steps (updated every ramp_every steps)."""
    done = 0
    while done < steps:
        if ramp_steps and done < ramp_steps:
            lat.set_lid(lid_u * min(1.0, (done + ramp_every) / ramp_steps))
            k = min(ramp_every, steps - done)
        else:
            if ramp_steps:
                lat.set_lid(lid_u)
            k = min(check_every - done % check_every, steps - done)
        lat.step(k)
        done += k
        if done % check_every == 0 or done == steps:
            if not lat.is_stable():
                return False
    return True


def bisect(stable, lo, hi, tol):
    """Largest x in [lo, hi] with stable(x) True, assuming stable() is monotone; lo is
    taken as stable, hi is tested first."""
    if stable(hi):
        return hi
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return lo


def max_stable_lid_velocity(nx, ny, nz, r, s, cs2, omega_nu, omega_xi=1.0, model="central", steps=100_000,
                            u_hi=0.6, tol=0.005, storage="f32", corr="local", ramp_steps=0):
    """Sec. 7 stability test: the largest lid velocity U (to within tol) for which the
    cavity stays stable for `steps` steps (the lid started impulsively, or brought up to U
    linearly over ramp_steps steps)."""
    def stable(U):
        lat = lid_cavity(nx, ny, nz, r, s, cs2, U, omega_nu, omega_xi, model, storage, corr)
        try:
            return survives(lat, steps, lid_u=U, ramp_steps=ramp_steps)
        finally:
            lat.close()
    return bisect(stable, 0.0, u_hi, tol)


def max_stable_reynolds(nx, ny, nz, r, s, cs2, U, model="central", steps=100_000, re_lo=10.0, re_hi=1e5,
                        rel_tol=0.02, storage="f32"):
    """Sec. 7: the largest Re = U L / nu (L = nx, the cavity side in units of dx) that
    stays stable for `steps` steps at lid velocity U (bisection in log Re)."""
    L = float(nx)

    def stable(log_re):
        nu = U * L / np.exp(log_re)
        wn = 1.0 / (nu / cs2 + 0.5)
        lat = lid_cavity(nx, ny, nz, r, s, cs2, U, wn, 1.0, model, storage)
        try:
            return survives(lat, steps)
        finally:
            lat.close()
    return float(np.exp(bisect(stable, np.log(re_lo), np.log(re_hi), np.log1p(rel_tol))))


def shallow_cavity(nx, ny, nz, r, s, cs2, U, Re=100.0, transits=30.0, storage="f32"):
    """Sec. 6 shallow cavity on an nx x ny x nz lattice with spacings (1, r, s): L = nx,
    nu = U L / Re, run for `transits` lid transits (t U / L).  Returns the centreline
    profiles u(y) at x = L/2, z = W/2 and v(x) at y = H/2, z = W/2 (normalised by U, with
    coordinates normalised by H and L), the steps and the device time in seconds."""
    L = float(nx)
    nu = U * L / Re
    lat = Lattice(nx, ny, nz, r_y=r, r_z=s, nu=nu, cs2=cs2, storage=storage, walls="xyz", lid_u=U,
                  stream=torch.cuda.Stream())
    dt = torch.float64 if storage == "f64" else torch.float32
    lat.init(torch.ones((nz, ny, nx), dtype=dt, device=lat.device),
             torch.zeros((3, nz, ny, nx), dtype=dt, device=lat.device))
    steps = int(round(transits * L / U))
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(lat.stream)
    lat.step(steps)
    end.record(lat.stream)
    torch.cuda.synchronize()
    seconds = start.elapsed_time(end) / 1e3
    _, u = lat.moments()
    stable = lat.is_stable()
    lat.close()
    u = u.double().cpu().numpy() / U

    def mid(a, n):            # value at the centre plane of an axis of n nodes
        return 0.5 * (a.take(n // 2 - 1, axis=0) + a.take(n // 2, axis=0)) if n % 2 == 0 else a.take(n // 2, axis=0)
    ux_zy = mid(np.moveaxis(u[0], 2, 0), nx)          # [nz, ny] at x = L/2
    u_y = mid(ux_zy, nz)                               # [ny]
    uy_zx = mid(np.moveaxis(u[1], 1, 0), ny)          # [nz, nx] at y = H/2
    v_x = mid(uy_zx, nz)                               # [nx]
    return {"y": (np.arange(ny) + 0.5) / ny, "u": u_y, "x": (np.arange(nx) + 0.5) / nx, "v": v_x,
            "steps": steps, "seconds": seconds, "nodes": nx * ny * nz, "stable": stable}
