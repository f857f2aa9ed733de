"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  FP64 storage: <= 1e-12 relative; FP32: <= 1e-5 relative on rho and
u (relative error = ||a - b||_2 / ||b||_2)."""
import functools

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_pair(oracle_mod, n, r, s, nu, cs2=None, corr="local", walls="", force=(0.0, 0.0, 0.0), storage="f64",
              zeta=0.0, lid_u=0.0, force_field=None):
    from paper_2107_14774_gb300 import Lattice
    lat = Lattice(*n, r_y=r, r_z=s, nu=nu, zeta=zeta, cs2=cs2 or 0.0, storage=storage, corr=corr, walls=walls,
                  force=force, lid_u=lid_u)
    p = lat.params
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          corr=getattr(oracle_mod, "CORR_" + corr.upper()), walls=walls, force=force,
                          force_field=force_field, lid_u=lid_u)
    if force_field is not None:
        lat.set_force_field(torch.from_numpy(force_field).cuda())
    return lat, o


def run_both(lat, o, rho, u, steps):
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    lat.step(steps)
    f_gpu = lat.populations().cpu().numpy()
    rg, ug = (t.cpu().numpy() for t in lat.moments())
    f_ref = o.run(o.init(rho, u), steps)
    rr, ur = o.moments(f_ref)
    return f_gpu, f_ref, rg, ug, rr, ur


@pytest.mark.parametrize("corr", ["none", "lowmach", "local", "full"])
@pytest.mark.parametrize("n,r,s,walls", [
    ((37, 12, 9), 0.5, 2.0, ""),          # ragged x (not a multiple of the 32-wide block)
    ((20, 12, 9), 1.0, 0.5, "y"),         # channel walls
    ((16, 10, 12), 0.5, 1.0, "yz"),       # duct walls
    ((9, 7, 6), 0.406, 1.3, "xyz"),       # closed box, corners and edges
    ((1, 24, 16), 0.25, 1.0, "y"),        # degenerate x axis
])
def test_fp64_parity_small(oracle_mod, corr, n, r, s, walls):
    rho, u = synth.solenoidal_random(*n, r, s, 2.0, 0.03, seed=11)
    rho = rho + 0.002 * np.cos(2 * np.pi * np.arange(n[0]) / max(n[0], 2))[None, None, :]
    F = (2e-5, -1e-5, 5e-6)
    lat, o = make_pair(oracle_mod, n, r, s, 0.02, corr=corr, walls=walls, force=F, zeta=0.01)
    f_gpu, f_ref, rg, ug, rr, ur = run_both(lat, o, rho, u, 6)
    assert rel(f_gpu, f_ref) < TOL64
    assert rel(rg, rr) < TOL64 and rel(ug, ur) < TOL64
    # density as its deviation from 1, and the worst node of the velocity field
    assert rel(rg - 1, rr - 1) < rho_dev_tol(rr, TOL64, 8)
    assert np.abs(ug - ur).max() / np.abs(ur).max() < TOL64
    lat.close()


def rho_dev_tol(rr, tol, real_size):
    """Bound on rel(rho - 1, rho_ref - 1): the parity tolerance plus the rounding of the
    output format itself (rho is returned in the compute type, whose half ulp at 1 is
    2^-24 in FP32: an absolute error no computation can remove from rho - 1)."""
    half_ulp = 2.0 ** -53 if real_size == 8 else 2.0 ** -24
    return tol + half_ulp * np.linalg.norm(rr) / np.linalg.norm(rr - 1)


@pytest.mark.parametrize("kernel", ["one", "auto", "onepass"])
@pytest.mark.parametrize("storage", ["f32", "f32s", "bf16s"])
@pytest.mark.parametrize("n,r,s,walls", [
    ((37, 12, 9), 0.5, 2.0, ""),          # periodic, ragged x (one node per thread)
    ((38, 12, 9), 0.5, 2.0, ""),          # periodic, even x (two nodes per thread)
    ((128, 12, 9), 0.5, 1.0, ""),         # periodic, rows of 2 x 64 nodes (single pass)
    ((20, 12, 9), 1.0, 0.5, "y"),         # channel walls (one-sided stencils)
    ((16, 10, 12), 0.5, 1.0, "yz"),       # duct walls
    ((16, 2, 7), 0.5, 1.0, "y"),          # two nodes across the channel: first-order stencil
    ((9, 7, 6), 0.406, 1.3, "xyz"),       # closed box
])
def test_fp32_full_corrections_parity(oracle_mod, kernel, storage, n, r, s, walls):
    """FULL corrections (lambda and e-terms of App. D with the density gradient of the
    current density, Sec. 2.5) at the production precision: FP32 arithmetic with plain
    and shifted FP32 storage against the FP64 oracle after 6 steps, u within 1e-5
    (relative L2 and worst node) and rho - 1 within 1e-5 plus the FP32 rounding of rho.
    The density carries 2 % waves so that FULL differs from LOCAL by far more than the
    tolerance (checked on the oracle side).  Both the one-node kernel (with its density
    pre-pass) and the automatic choice (two nodes per thread where x allows it) are run;
    BF16 storage is held to the reduced-precision bound of the short-run test (6e-3) in L2
    and to 4 x 2^-8 at the worst node (8 significant bits per stored deviation)."""
    rho, u = synth.solenoidal_random(*n, r, s, 2.0, 0.03, seed=11)
    rho = (rho + 0.02 * np.cos(2 * np.pi * np.arange(n[0]) / n[0])[None, None, :]
           + 0.02 * np.sin(2 * np.pi * np.arange(n[2]) / n[2])[:, None, None])
    F = (2e-5, -1e-5, 5e-6)
    from paper_2107_14774_gb300 import Lattice
    lat = Lattice(*n, r_y=r, r_z=s, nu=0.02, zeta=0.01, storage=storage, corr="full", walls=walls, force=F,
                  kernel=kernel)
    p = lat.params
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          corr=oracle_mod.CORR_FULL, walls=walls, force=F)
    if kernel == "onepass" and n[0] % 64 == 0 and not walls:
        want = "k_step_full<"
    elif kernel != "one" and n[0] % 2 == 0 and "x" not in walls:
        want = "k_step_pair<"
    else:
        want = "k_step<"
    assert lat.step_kernel.startswith(want), lat.step_kernel
    _, _, rg, ug, rr, ur = run_both(lat, o, rho, u, 6)
    p = lat.params
    lat.close()
    o_local = oracle_mod.Oracle(*n, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                                corr=oracle_mod.CORR_LOCAL, walls=walls, force=F)
    _, ul = o_local.moments(o_local.run(o_local.init(rho, u), 6))
    tol = TOL32 if storage != "bf16s" else 6e-3
    assert rel(ul, ur) > 10 * TOL32
    assert rel(ug, ur) < tol
    assert np.abs(ug - ur).max() / np.abs(ur).max() < (tol if storage != "bf16s" else 4 * 2.0 ** -8)
    assert rel(rg - 1, rr - 1) < rho_dev_tol(rr, tol if storage != "bf16s" else 20 * tol, 4)


def test_fp64_parity_force_field(oracle_mod):
    n, r, s = (24, 16, 8), 1.0, 0.5
    ff = synth.force_field(*n, 1e-5, seed=44)
    rho, u = synth.solenoidal_random(*n, r, s, 4.0, 0.01, seed=4)
    lat, o = make_pair(oracle_mod, n, r, s, 0.01, force_field=ff)
    f_gpu, f_ref, *_ = run_both(lat, o, rho, u, 5)
    assert rel(f_gpu, f_ref) < TOL64
    lat.close()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-6), ("f32s", 1e-6)])
def test_reduce_matches_oracle_moments(oracle_mod, storage, tol):
    """lb_reduce (FP64 sums of rho and rho u = sum f e + F/2, Eq. 12) against the sums of
    the oracle's moments of the populations the GPU holds, with y and z walls, a uniform
    force and a per-node force field: FP64 within 1e-12; FP32 within 1e-6 (lb_reduce forms
    each node's moments in FP32 before the FP64 sum).  Momentum is compared relative to
    the total |rho u| of the flow."""
    n, r, s = (22, 18, 10), 0.5, 2.0
    ff = synth.force_field(*n, 1e-5, seed=45)
    F = (2e-5, -1e-5, 4e-6)
    rho, u = synth.solenoidal_random(*n, r, s, 3.0, 0.02, seed=21)
    rho = rho + 0.003 * np.sin(2 * np.pi * np.arange(n[1]) / n[1])[None, :, None]
    lat, o = make_pair(oracle_mod, n, r, s, 0.02, walls="yz", force=F, storage=storage, force_field=ff)
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    scale = np.sqrt((u ** 2).sum(0)).sum()
    for steps in (0, 4):
        lat.step(steps)
        got = lat.reduce()
        rr, ur = o.moments(lat.populations().double().cpu().numpy())
        want = np.array([rr.sum(), *(rr[None] * ur).reshape(3, -1).sum(1)])
        assert abs(got[0] / want[0] - 1) < tol
        assert np.abs(got[1:] - want[1:]).max() < tol * scale
    lat.close()


def test_taylor_green_32x32x16_fp64_full_run(oracle_mod):
    """32x32x16, r=1, s=0.5, nu=0.01, u0=0.02, FP64, 100 steps: fields within 1e-12 of the
    oracle; mass conserved to 1e-13 and total momentum zero."""
    n, r, s = (32, 32, 16), 1.0, 0.5
    rho, u, _ = synth.taylor_green_3d(*n, r, s, 0.02)
    lat, o = make_pair(oracle_mod, n, r, s, 0.01)
    m0 = lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).reduce()
    lat.step(100)
    m1 = lat.reduce()
    rg, ug = (t.cpu().numpy() for t in lat.moments())
    rr, ur = o.moments(o.run(o.init(rho, u), 100))
    assert rel(rg, rr) < TOL64 and rel(ug, ur) < TOL64
    assert rel(rg - 1, rr - 1) < rho_dev_tol(rr, TOL64, 8)
    assert np.abs(ug - ur).max() / np.abs(ur).max() < TOL64
    assert abs(m1[0] / m0[0] - 1) < 1e-13
    assert np.abs(m1[1:]).max() < 1e-12
    lat.close()


@pytest.mark.parametrize("storage,steps,tol", [("f64", 1000, TOL64), ("f32s", 300, TOL32), ("f32", 300, 1e-4)])
def test_duct_16x64x128_parity(oracle_mod, storage, steps, tol):
    """The 16x64x128 duct from rest: r=0.5, s=2, walls y/z, periodic x,
    F=(1e-6,0,0), starting from rest.  The flow is invariant along x (periodic x,
    uniform force and initial state), so the GPU field must be identical in every
    x-column and the oracle runs the 1x64x128 cross-section.
    FP64 is compared after 1000 steps: earlier the velocity is so small (1e-5..1e-4)
    that the FP64 rounding of O(0.1) populations, in the oracle as on the GPU, already
    amounts to ~1e-12 of it.  FP32 is compared after 300 steps: storing h in FP32 adds
    ~6e-8 |h| of rounding per step while the force adds only ~1e-6 per step, so the
    FP32 error grows with the run (1.3e-5 after 1000 steps with shifted storage).
    Plain FP32 storage (f = w + h rounded) loses more low bits of h: bound 1e-4."""
    n, r, s, cs2 = (16, 64, 128), 0.5, 2.0, 1 / 12
    from paper_2107_14774_gb300 import Lattice
    lat = Lattice(*n, r_y=r, r_z=s, nu=cs2 / 2, cs2=cs2, storage=storage, walls="yz", force=(1e-6, 0.0, 0.0))
    lat.init(torch.ones(n[::-1], dtype=torch.float64).cuda(), torch.zeros((3,) + n[::-1], dtype=torch.float64).cuda())
    lat.step(steps)
    rg, ug = (t.cpu().numpy().astype(np.float64) for t in lat.moments())
    p = lat.params
    lat.close()
    assert np.array_equal(ug, np.broadcast_to(ug[..., :1], ug.shape))   # x-invariant, bit for bit
    o = oracle_mod.Oracle(1, n[1], n[2], r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          walls="yz", force=(1e-6, 0.0, 0.0))
    rr, ur = o.moments(o.run(o.init(np.ones((n[2], n[1], 1)), np.zeros((3, n[2], n[1], 1))), steps))
    e_rho, e_u = rel(rg[..., :1], rr), rel(ug[..., :1], ur)
    print(f"duct {storage}: rel err rho {e_rho:.2e}  u {e_u:.2e}")
    assert e_rho < tol and e_u < tol


def test_duct_16x64x128_disturbed_fp64(oracle_mod):
    """The 16x64x128 duct with a seeded solenoidal disturbance added to the initial
    state, so that every velocity component and every wall link carries signal."""
    n, r, s, cs2 = (16, 64, 128), 0.5, 2.0, 1 / 12
    rho, up = synth.solenoidal_random(*n, r, s, 3.0, 0.01, seed=2)
    lat, o = make_pair(oracle_mod, n, r, s, cs2 / 2, cs2=cs2, walls="yz", force=(1e-6, 0.0, 0.0))
    f_gpu, f_ref, rg, ug, rr, ur = run_both(lat, o, rho, up, 150)
    assert rel(f_gpu, f_ref) < TOL64 and rel(ug, ur) < TOL64
    lat.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_duct_16x64x128_converges_to_series(storage):
    """Full config-2 run (20k steps) on the GPU against the rectangular-duct series (Eq. 70
    generalised), 2a = ny r = 32, 2b = nz s = 256."""
    from paper_2107_14774_gb300 import Lattice
    from tests.analytic import duct_series
    n, r, s, cs2 = (16, 64, 128), 0.5, 2.0, 1 / 12
    nu, Fx = cs2 / 2, 1e-6
    lat = Lattice(*n, r_y=r, r_z=s, nu=nu, cs2=cs2, storage=storage, walls="yz", force=(Fx, 0, 0))
    lat.init(torch.ones(n[::-1]).cuda(), torch.zeros((3,) + n[::-1]).cuda()).step(20000)
    _, u = lat.moments()
    ux = u[0].mean(dim=2).cpu().numpy().astype(np.float64)    # average over x: [nz, ny]
    a, b = n[1] * r / 2, n[2] * s / 2
    Z, Y = np.meshgrid((np.arange(n[2]) + 0.5) * s - b, (np.arange(n[1]) + 0.5) * r - a, indexing="ij")
    ua = duct_series(Y, Z, a, b, Fx, 1.0, nu)
    assert rel(ux, ua) < 0.01
    lat.close()


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f32s", 1e-5), ("f16s", 1e-3), ("bf16s", 6e-3)])
def test_reduced_precision_storage_short_run(oracle_mod, storage, tol):
    """Shifted FP16/BF16 storage against the FP64 oracle after a few steps: the stored
    deviations carry 11 (FP16) / 8 (BF16) significant bits."""
    n, r, s = (40, 24, 24), 0.5, 0.5
    rho, u = synth.solenoidal_random(*n, r, s, 4.0, 0.03, seed=3)
    lat, o = make_pair(oracle_mod, n, r, s, 0.005, storage=storage)
    f_gpu, f_ref, rg, ug, rr, ur = run_both(lat, o, rho, u, 10)
    assert rel(ug, ur) < tol
    assert rel(rg - 1, rr - 1) < 20 * tol
    lat.close()


@pytest.mark.parametrize("storage", ["f32", "f32s"])
def test_fp32_velocity_amplitude_tracks_fp64(storage):
    """FP32 arithmetic against the FP64 path on a decaying solenoidal flow (128x64x64,
    r = s = 0.5, cs2 = 1/12, nu = 0.005) after 500 steps from the same FP32-rounded
    initial field: the velocity error's component along the flow itself (the amplitude
    error beta = <du.u>/<u.u>) stays below 5e-6.  Rest weights whose per-axis sums miss 1
    in FP32 (2/3 + 2 (1/6) rounds to 1 + 2^-25) scale the momentum by 1 + 6e-8 at every
    collision: beta = 3.4e-5 after these 500 steps."""
    from paper_2107_14774_gb300 import Lattice
    n, r, s = (128, 64, 64), 0.5, 0.5
    rho, u = synth.solenoidal_random(*n, r, s, 4.0, 0.03, seed=3)
    u32 = torch.from_numpy(u.astype(np.float32)).cuda()
    out = {}
    for st in ("f64", storage):
        lat = Lattice(*n, r_y=r, r_z=s, nu=0.005, cs2=1 / 12, storage=st)
        lat.init(torch.ones(n[::-1], dtype=lat.dtype).cuda(), u32.to(lat.dtype)).step(500)
        out[st] = lat.moments()[1].double()
        lat.close()
    ref = out["f64"]
    du = out[storage] - ref
    beta = float((du * ref).sum() / (ref * ref).sum())
    err = float(torch.linalg.vector_norm(du) / torch.linalg.vector_norm(ref))
    print(storage, "beta", beta, "u_rel_l2", err)
    assert abs(beta) < 5e-6
    assert err < 1e-4


STORED_DTYPE = {"f32": torch.float32, "f32s": torch.float32, "f16s": torch.float16, "bf16s": torch.bfloat16}


@functools.lru_cache(maxsize=1)
def decaying_512x256x256_inputs():
    rho, u = synth.solenoidal_random(512, 256, 256, 0.5, 0.5, 4.0, 0.03, seed=3)
    return rho.astype(np.float32), u.astype(np.float32)


@functools.lru_cache(maxsize=1)
def channel_768x192x384_inputs():
    rho, u, Fx = synth.channel(768, 192, 384, 0.25, 1.0, 0.02, 0.005, 0.05, seed=5)
    return rho.astype(np.float32), u.astype(np.float32), Fx


def sampled_step_errors(lat, o, n, pts, storage, F=(0.0, 0.0, 0.0), wall_y=False):
    """One fused step of `lat` (already initialised) checked at sampled nodes against the
    oracle's collision of the same stored pre-collision values, pulled from the GPU's
    own state by the streaming rule (f_a(x) = S_a(x - e_a), periodic wrap; S_opp(a)(x)
    across a y wall).  Returns the worst error over the sampled nodes and their 27
    populations:
      f32 / f32s: |got - want| beyond the half ulp the FP32 store of the value itself
                  may round off and beyond 16 FP32 ulps of the rest weight (the absolute
                  rounding of the O(w) terms of the arithmetic, such as phi = w + dphi:
                  it dominates at slow nodes, next to a wall), relative to the node's
                  largest deviation |f~ - w|;
      f16s / bf16s: |got - round(want)| in units of the storage ulp, with round() the
                  oracle's storage emulation (round to nearest even), beyond 16 FP32 ulps
                  of the rest weight."""
    e = o.velocities()
    opp = [int(np.flatnonzero((e == -e[:, [a]]).all(axis=0))[0]) for a in range(27)]
    w = o.equilibrium(1.0, [0, 0, 0])
    # FP16 stores h * 2^(10 - ilogb w_a) per direction
    scale = 2.0 ** (10 - (np.frexp(w)[1] - 1))
    dt = STORED_DTYPE[storage]
    S0 = lat.get_state().view(dt).reshape((27,) + n[::-1])
    blocks = {}
    for (i, j, k) in pts:      # the 3x3x3 neighbourhood of each sampled node in the stored state
        ks = [(k + d) % n[2] for d in (-1, 0, 1)]
        js = [(j + d) % n[1] for d in (-1, 0, 1)]
        is_ = [(i + d) % n[0] for d in (-1, 0, 1)]
        blocks[(i, j, k)] = S0[:, ks][:, :, js][:, :, :, is_].double().cpu().numpy()
    del S0
    lat.step(1)
    S1 = lat.get_state().view(dt).reshape((27,) + n[::-1])
    worst = 0.0
    for (i, j, k) in pts:
        blk = blocks[(i, j, k)]
        raw = np.empty(27)
        for a in range(27):
            if wall_y and not 0 <= j - e[1, a] < n[1]:
                raw[a] = blk[opp[a], 1, 1, 1]
            else:
                raw[a] = blk[a, 1 - e[2, a], 1 - e[1, a], 1 - e[0, a]]
        # stored value -> pre-collision deviation h = f - w
        h = raw - w if storage == "f32" else (raw / scale if storage == "f16s" else raw)
        ft = o.collide_node(w + h, F)
        got = S1[:, k, j, i].double().cpu().numpy()
        if storage in ("f32", "f32s"):
            want = ft if storage == "f32" else ft - w
            dev = np.abs(ft - w).max()
            d = np.maximum(np.abs(got - want) - 2.0 ** -24 * np.abs(want) - 2.0 ** -20 * w, 0.0)
            worst = max(worst, float(d.max() / dev))
        else:
            q = o.quantize(ft.reshape(27, 1, 1, 1)).ravel() - w
            gh = got / scale if storage == "f16s" else got
            want = torch.from_numpy(q * (scale if storage == "f16s" else 1.0)).to(dt).double().numpy()
            want = want / scale if storage == "f16s" else want
            mant = 10 if storage == "f16s" else 7
            sp = 2.0 ** (np.frexp(np.where(want == 0, 1e-300, want))[1] - 1 - mant)
            if storage == "f16s":   # subnormal range of the scaled binary16 value
                sp = np.maximum(sp, 2.0 ** -24 / scale)
            dd = np.abs(gh - want) / sp
            floor = 2.0 ** -20 * w / sp
            worst = max(worst, float(np.max(dd - np.minimum(dd, floor))))
    return worst


@pytest.mark.parametrize("storage", ["f32", "f32s", "f16s", "bf16s"])
def test_full_size_decaying_512x256x256_sampled_nodes(oracle_mod, storage):
    """Decaying anisotropic flow 512x256x256 (r = s = 0.5, cs2 = 1/12, nu = 0.005), in the
    launch configuration the bench times, one fused step from the seeded solenoidal field:
    sampled nodes (all 27 populations) against the oracle's collision of the GPU's own stored
    pre-collision values.  FP32 storage: within 1e-5 of the node's largest deviation
    |f~ - w| (beyond the half ulp of the FP32 store and 16 FP32 ulps of w); FP16/BF16: the
    oracle's output rounded
    by its storage emulation, within one storage ulp.  Mass is conserved to 1e-6."""
    from paper_2107_14774_gb300 import Lattice
    n, r, s, cs2, nu = (512, 256, 256), 0.5, 0.5, 1 / 12, 0.005
    rho, u = decaying_512x256x256_inputs()
    lat = Lattice(*n, r_y=r, r_z=s, nu=nu, cs2=cs2, storage=storage)
    assert "k_step_pair" in lat.step_kernel
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    lat.step(2)
    m0 = lat.reduce()
    p = lat.params
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          storage_emulation=storage if storage in ("f16s", "bf16s") else None)
    rng = np.random.default_rng(0)
    pts = [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1), (31, 32, 255)] + [
        tuple(int(rng.integers(0, m)) for m in n) for _ in range(12)]
    worst = sampled_step_errors(lat, o, n, pts, storage)
    m1 = lat.reduce()
    lat.close()
    print(storage, "worst", worst)
    assert worst < (1e-5 if storage in ("f32", "f32s") else 1.0 + 1e-9)
    assert abs(m1[0] / m0[0] - 1) < 1e-6


@pytest.mark.parametrize("storage", ["f32", "bf16s"])
def test_lattice_beyond_32bit_offsets_sampled_nodes(oracle_mod, storage):
    """A 1024x512x328 lattice holds 27 N = 4.64e9 > 2^32 populations per buffer, so the
    two-node kernel (32-bit element offsets) gives way to the one-node kernel with 64-bit
    offsets.  One fused step from a smooth field (three Fourier modes, built on the
    device), checked at sampled nodes against the oracle's collision of the GPU's own
    stored values: the last node and the highest plane included, whose populations sit
    beyond element 2^32 of the buffer.  Mass (FP64 sum over every node) is conserved to
    1e-6."""
    from paper_2107_14774_gb300 import Lattice
    n, r, s, cs2, nu = (1024, 512, 328), 0.5, 1.0, 1 / 12, 0.01
    assert 27 * n[0] * n[1] * n[2] > 2 ** 32
    lat = Lattice(*n, r_y=r, r_z=s, nu=nu, cs2=cs2, storage=storage)
    assert lat.step_kernel.startswith("k_step<"), lat.step_kernel
    ax = [torch.arange(m, device="cuda", dtype=torch.float32) * (2 * np.pi / m) for m in n]
    X, Y, Z = ax[0][None, None, :], ax[1][None, :, None], ax[2][:, None, None]
    rho = 1.0 + 1e-3 * torch.cos(X + Z) * torch.ones_like(Y)
    u = torch.stack([0.02 * torch.sin(X) * torch.cos(Y) * torch.cos(Z),
                     -0.01 * torch.cos(X) * torch.sin(Y) * torch.cos(Z),
                     0.005 * torch.sin(2 * Z) * torch.cos(X) * torch.ones_like(Y)])
    lat.init(rho, u)
    del rho, u, X, Y, Z
    lat.step(1)
    m0 = lat.reduce()
    p = lat.params
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          storage_emulation="bf16s" if storage == "bf16s" else None)
    rng = np.random.default_rng(9)
    pts = [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1), (511, 255, n[2] - 1), (n[0] - 1, 0, n[2] - 2)] + [
        tuple(int(rng.integers(0, m)) for m in n) for _ in range(8)]
    worst = sampled_step_errors(lat, o, n, pts, storage)
    m1 = lat.reduce()
    lat.close()
    print(storage, "worst", worst)
    assert worst < (1e-5 if storage == "f32" else 1.0 + 1e-9)
    assert abs(m1[0] / m0[0] - 1) < 1e-6


def test_state_checkpoint_resume_is_bit_exact():
    from paper_2107_14774_gb300 import Lattice
    n = (24, 16, 8)
    rho, u = synth.solenoidal_random(*n, 1.0, 0.5, 3.0, 0.02, seed=9)
    for storage in ["f32", "bf16s", "f16s"]:
        a = Lattice(*n, r_y=1.0, r_z=0.5, nu=0.01, storage=storage, walls="z")
        b = Lattice(*n, r_y=1.0, r_z=0.5, nu=0.01, storage=storage, walls="z")
        a.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).step(7)
        st = a.get_state().cpu()
        a.step(5)
        b.set_state(st.cuda(), 7).step(5)
        assert torch.equal(a.get_state(), b.get_state())
        assert b.time_step == 12
        a.close()
        b.close()


def test_host_and_device_pointers_agree():
    from paper_2107_14774_gb300 import Lattice
    n = (16, 8, 8)
    rho, u = synth.solenoidal_random(*n, 0.5, 0.5, 3.0, 0.02, seed=1)
    a = Lattice(*n, r_y=0.5, r_z=0.5, nu=0.01)
    b = Lattice(*n, r_y=0.5, r_z=0.5, nu=0.01)
    a.init(torch.from_numpy(rho).float().cuda(), torch.from_numpy(u).float().cuda()).step(3)
    b.init(torch.from_numpy(rho).float(), torch.from_numpy(u).float().pin_memory()).step(3)
    ra, ua = a.moments()
    rb = torch.empty(n[::-1]).pin_memory()
    ub = torch.empty((3,) + n[::-1])
    b.moments(rb, ub)
    assert torch.equal(ra.cpu(), rb) and torch.equal(ua.cpu(), ub)
    a.close()
    b.close()


def test_set_populations_roundtrip(oracle_mod):
    from paper_2107_14774_gb300 import Lattice
    n = (12, 10, 8)
    rho, u = synth.solenoidal_random(*n, 0.5, 1.0, 3.0, 0.02, seed=5)
    lat, o = make_pair(oracle_mod, n, 0.5, 1.0, 0.02, walls="xz")
    f0 = o.init(rho, u)
    lat.set_populations(torch.from_numpy(f0).cuda())
    np.testing.assert_array_equal(lat.populations().cpu().numpy(), f0)
    lat.step(4)
    assert rel(lat.populations().cpu().numpy(), o.run(f0, 4)) < TOL64
    lat.close()


def test_moving_lid_parity(oracle_mod):
    """Lid-driven box (walls on every axis, lid at the top y wall), FP64, 30 steps."""
    n, r, s = (10, 12, 8), 0.5, 0.75
    rho, u = np.ones(n[::-1]), np.zeros((3,) + n[::-1])
    lat, o = make_pair(oracle_mod, n, r, s, 0.02, cs2=0.04, walls="xyz", lid_u=0.05)
    f_gpu, f_ref, *_ = run_both(lat, o, rho, u, 30)
    assert rel(f_gpu, f_ref) < TOL64
    lat.close()


@pytest.mark.parametrize("own_stream", [False, True])
def test_lid_velocity_changed_between_steps(oracle_mod, own_stream):
    """lb_set_lid between lb_step calls (a lid ramp): the step from t to t + 1 uses the lid
    set before the call that runs it, as in the oracle with its lid changed between the
    same steps (Eq. 69).  On a stream of its own the 70-step segment replays CUDA graphs."""
    from paper_2107_14774_gb300 import Lattice
    n, r, s = (10, 12, 8), 0.5, 0.75
    rho, u = np.ones(n[::-1]), np.zeros((3,) + n[::-1])
    lat = Lattice(*n, r_y=r, r_z=s, nu=0.02, cs2=0.04, storage="f64", walls="xyz", lid_u=0.03,
                  stream=torch.cuda.Stream() if own_stream else None)
    p = lat.params
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          corr=oracle_mod.CORR_LOCAL, walls="xyz", lid_u=0.03)
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    f = o.init(rho, u)
    for lid, steps in ((0.03, 5), (0.06, 3), (0.08, 70 if own_stream else 9), (0.0, 4), (0.05, 1)):
        lat.set_lid(lid).step(steps)
        o.p.lid_u = lid
        f = o.run(f, steps)
        assert rel(lat.populations().cpu().numpy(), f) < TOL64
    lat.close()


def test_lid_requires_y_walls():
    """lb_set_lid refuses a moving lid without walls normal to y and a non-finite value;
    a lid at rest is accepted on any lattice."""
    from paper_2107_14774_gb300 import Lattice, LBError
    lat = Lattice(8, 8, 8, nu=0.02, walls="z")
    lat.set_lid(0.0)
    with pytest.raises(LBError, match="walls normal to y"):
        lat.set_lid(0.1)
    lat.close()
    lat = Lattice(8, 8, 8, nu=0.02, walls="y")
    with pytest.raises(LBError, match="non-finite"):
        lat.set_lid(float("nan"))
    lat.set_lid(0.1)
    lat.close()


def test_unstable_state_is_reported():
    """A NaN planted in the initial density is reported by lb_reduce as LB_EUNSTABLE."""
    from paper_2107_14774_gb300 import Lattice, LBError
    n = (8, 8, 8)
    rho = np.ones(n[::-1])
    rho[3, 4, 5] = np.nan
    lat = Lattice(*n, nu=0.02)
    lat.init(torch.from_numpy(rho).cuda(), torch.zeros((3,) + n[::-1]).cuda()).step(2)
    with pytest.raises(LBError, match="EUNSTABLE"):
        lat.reduce()
    sums = lat.reduce(allow_unstable=True)
    assert np.isnan(sums[0])
    lat.close()


@pytest.mark.parametrize("walls", ["y", "z", "yz", ""])
@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f32s", 1e-5), ("f16s", 1e-3), ("bf16s", 6e-3)])
def test_kernel_variants_agree(oracle_mod, storage, tol, walls):
    """The row-staged kernel, the two-nodes-per-thread kernel (packed FP32x2 arithmetic;
    the automatic choice) and the one-node kernel agree with the oracle and with each
    other (channel walls, force field)."""
    from paper_2107_14774_gb300 import Lattice
    n, r, s = (64, 20, 12), 0.5, 1.0
    rho, u = synth.solenoidal_random(*n, r, s, 3.0, 0.03, seed=21)
    ff = synth.force_field(*n, 1e-5, seed=22)
    out = {}
    for kern in ("auto", "pair", "one", "staged", "march"):
        lat = Lattice(*n, r_y=r, r_z=s, nu=0.01, storage=storage, walls=walls, force=(1e-6, 0, 0), kernel=kern)
        lat.set_force_field(torch.from_numpy(ff).cuda())
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).step(8)
        out[kern] = lat.moments()[1].cpu().numpy()
        p = lat.params
        lat.close()
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          walls=walls, force=(1e-6, 0, 0), force_field=ff)
    _, ur = o.moments(o.run(o.init(rho, u), 8))
    for kern in out:
        assert rel(out[kern], ur) < tol, kern
    for kern in ("auto", "pair", "staged", "march"):
        assert rel(out[kern], out["one"]) < tol, kern


@pytest.mark.parametrize("n", [(128, 16, 40), (64, 12, 17), (192, 1, 20), (64, 2, 1), (64, 9, 33)])
@pytest.mark.parametrize("storage", ["f32", "f32s", "f16s", "bf16s"])
def test_full_single_pass_matches_two_pass_bit_for_bit(storage, n):
    """FULL corrections: the single-pass kernel (densities of the next plane and of the
    tile's halo computed into a shared-memory ring while marching along z) stores the same
    state as the density pre-pass plus two-node step, bit for bit, after several steps:
    tiles cut short in y (12 and 9 rows against 8 per tile) and in z (17, 33 and 40 planes
    against 16), a lattice one row and one two rows high, a single plane, a force field
    and density waves along every axis."""
    from paper_2107_14774_gb300 import Lattice
    rho, u = synth.solenoidal_random(*n, 0.5, 1.0, 2.0, 0.03, seed=41)
    rho = (rho + 0.02 * np.cos(2 * np.pi * np.arange(n[0]) / n[0])[None, None, :]
           + 0.01 * np.sin(2 * np.pi * np.arange(n[1]) / n[1])[None, :, None]
           + 0.02 * np.sin(2 * np.pi * np.arange(n[2]) / n[2])[:, None, None])
    ff = synth.force_field(*n, 1e-5, seed=42)
    states = {}
    for kern in ("onepass", "auto"):
        lat = Lattice(*n, r_y=0.5, r_z=1.0, nu=0.02, zeta=0.01, storage=storage, corr="full", kernel=kern,
                      force=(2e-5, -1e-5, 5e-6))
        assert lat.step_kernel.startswith("k_step_full<" if kern == "onepass" else "k_step_pair<"), lat.step_kernel
        lat.set_force_field(torch.from_numpy(ff).cuda())
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).step(5)
        states[kern] = lat.get_state().cpu()
        lat.close()
    assert torch.equal(states["onepass"], states["auto"])


@pytest.mark.parametrize("n", [(160, 6, 13), (66, 5, 9), (64, 4, 8)])
@pytest.mark.parametrize("walls", ["", "y", "z", "yz"])
@pytest.mark.parametrize("storage,rounding", [("bf16s", "nearest"), ("f16s", "nearest"), ("bf16s", "stochastic"),
                                              ("f16s", "stochastic")])
def test_march_kernel_matches_pair_bit_for_bit(storage, rounding, walls, n):
    """The z-marching kernel (sources of the next plane staged in shared memory) computes
    what the two-node kernel computes from the same words: the stored state is equal bit
    for bit after several steps, on rows that end inside a warp (80 and 33 node pairs: a
    segment whose only lane is both first and last), rows of exactly one segment, partial
    blocks in y, plane counts that are not a multiple of the marching depth, walls,
    stochastic rounding and a per-node force field."""
    from paper_2107_14774_gb300 import Lattice
    rho, u = synth.solenoidal_random(*n, 0.5, 1.0, 2.0, 0.03, seed=31)
    ff = synth.force_field(*n, 1e-5, seed=32)
    states = {}
    for kern in ("pair", "march"):
        lat = Lattice(*n, r_y=0.5, r_z=1.0, nu=0.01, storage=storage, walls=walls, kernel=kern, rounding=rounding,
                      rounding_seed=3)
        lat.set_force_field(torch.from_numpy(ff).cuda())
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).step(5)
        assert lat.step_kernel.startswith("k_step_march<" if kern == "march" else "k_step_pair<"), lat.step_kernel
        states[kern] = lat.get_state().cpu()
        lat.close()
    assert torch.equal(states["march"], states["pair"])


@pytest.mark.parametrize("kern", ["auto", "one", "staged"])
@pytest.mark.parametrize("storage", ["bf16s", "f16s"])
def test_stochastic_rounding_is_unbiased_and_keeps_lanes(oracle_mod, storage, kern):
    """Stochastic rounding of the 16-bit stores.  From rest (h = 0, exact in every
    format) a body force that varies along x only drives one collision.  The raw stored
    deviations (lb_get_state: after a step the state holds each node's post-collision
    values g = f~ - w, FP16 scaled by 2^(10 - ilogb(w)) per direction) averaged over the
    64 x 64 nodes of each x-column equal the oracle's post-collision deviations to well
    below one storage ulp (unbiased draws, correct lane order of the packed pairs),
    while every column shows the spread of the draws."""
    from paper_2107_14774_gb300 import Lattice
    n, r, s, nu = (64, 64, 64), 0.5, 1.0, 0.02
    x = np.arange(n[0])
    ff = np.zeros((3,) + n[::-1])
    ff[0] += (1e-3 * np.sin(2 * np.pi * x / n[0]))[None, None, :]
    ff[1] += (5e-4 * np.cos(2 * np.pi * x / n[0]))[None, None, :]
    ff[2] += (3e-4 * np.sin(4 * np.pi * x / n[0]))[None, None, :]
    lat = Lattice(*n, r_y=r, r_z=s, nu=nu, storage=storage, kernel=kern, rounding="stochastic", rounding_seed=7)
    lat.set_force_field(torch.from_numpy(ff).cuda())
    lat.init(torch.ones(n[::-1]).cuda(), torch.zeros((3,) + n[::-1]).cuda()).step(1)
    raw = lat.get_state().view(torch.bfloat16 if storage == "bf16s" else torch.float16)
    g = raw.double().cpu().numpy().reshape((27,) + n[::-1])
    p = lat.params
    lat.close()
    o = oracle_mod.Oracle(n[0], 1, 1, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          force_field=ff[:, :1, :1, :].copy())
    w = o.equilibrium(1.0, [0, 0, 0])
    ft = o.collide_all(o.init(np.ones((1, 1, n[0])), np.zeros((3, 1, 1, n[0]))))[:, 0, 0, :]   # [27, nx]
    want = ft - w[:, None]
    if storage == "f16s":
        scale = 2.0 ** (10 - (np.frexp(w)[1] - 1))
        g = g / scale[:, None, None, None]
    mean = g.mean(axis=(1, 2))
    spread = g.std(axis=(1, 2))
    bits = 8 if storage == "bf16s" else 11
    ulp = np.abs(want) * 2.0 ** (1 - bits)     # storage ulp of the deviation, per value
    moving = ulp > 1e-12
    assert np.all(np.abs(mean - want)[moving] < 0.05 * ulp[moving] + 1e-12)
    assert np.median(spread[moving] / ulp[moving]) > 0.1


def _storage_spacing(g, w, storage):
    """Spacing of the stored format around each deviation g (in units of g): bfloat16
    2^(e-7); binary16 of g * 2^(10 - ilogb w) is 2^(max(e, -14) - 10), divided back."""
    if storage == "bf16s":
        e = np.frexp(np.where(g == 0, 1e-300, g))[1] - 1
        return 2.0 ** (e - 7)
    sc = (2.0 ** (10 - (np.frexp(w)[1] - 1)))[:, None, None, None]
    e = np.maximum(np.frexp(np.where(g == 0, 1e-300, g * sc))[1] - 1, -14)
    return 2.0 ** (e - 10) / sc


def _snap(x, w, storage):
    """Round values that lie within FP64 rounding of the stored format back onto it (the
    oracle keeps f = w + g in FP64, so f - w can differ from g in the last FP64 bit)."""
    if storage == "bf16s":
        return torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16).double().numpy()
    sc = (2.0 ** (10 - (np.frexp(w)[1] - 1)))[:, None, None, None]
    return (x * sc).astype(np.float16).astype(np.float64) / sc


def _decode_state(lat, w, storage, shape):
    raw = lat.get_state().view(torch.bfloat16 if storage == "bf16s" else torch.float16)
    g = raw.double().cpu().numpy().reshape((27,) + shape)
    if storage == "f16s":
        g = g / (2.0 ** (10 - (np.frexp(w)[1] - 1)))[:, None, None, None]
    return g


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("steps", [1, 10])
def test_reduced_storage_step_matches_emulated_oracle(oracle_mod, storage, steps):
    """One step of the 16-bit path against one step of the oracle's storage emulation (the
    same rounding of the stored deviations, in FP64 from the IEEE definition) from the
    same stored state, the GPU's own after steps - 1 steps: streaming the stored values
    gives the pre-collision populations (pull layout), the oracle collides and rounds
    them.  Nearly every stored value is then bit-identical and none differs by more than
    one storage ulp plus 16 FP32 ulps of the rest weight (the FP32 arithmetic can move a
    value across a rounding boundary, and dominates for deviations far below w).  The
    initial state is checked the same way against the emulated initialisation."""
    n, r, s = (40, 24, 24), 0.5, 0.5
    rho, u = synth.solenoidal_random(*n, r, s, 4.0, 0.03, seed=3)
    from paper_2107_14774_gb300 import Lattice
    lat = Lattice(*n, r_y=r, r_z=s, nu=0.005, storage=storage)
    p = lat.params
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          storage_emulation=storage)
    w = o.equilibrium(1.0, [0, 0, 0])
    wb = w[:, None, None, None]
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    checks = []
    g0 = _decode_state(lat, w, storage, n[::-1])
    checks.append(("init", _snap(o.stream(wb + g0) - wb, w, storage), _snap(o.init(rho, u) - wb, w, storage)))
    lat.step(steps - 1)
    g_prev = _decode_state(lat, w, storage, n[::-1])
    lat.step(1)
    g = _decode_state(lat, w, storage, n[::-1])
    lat.close()
    want = _snap(o.quantize(o.collide_all(o.stream(wb + g_prev))) - wb, w, storage)
    checks.append(("step", g, want))
    for name, got, ref in checks:
        sp = _storage_spacing(ref, w, storage)
        d = np.abs(got - ref) / sp
        floor = (2.0 ** -20 * wb) / sp
        same = float(np.mean(got == ref))
        print(storage, steps, name, "identical %.6f" % same, "max ulps %.3f" % float(np.max(d - np.minimum(d, floor))))
        assert same > 0.995, name
        assert np.all(d <= 1.0 + floor), name


@pytest.mark.parametrize("storage,walls,lid", [("f32", "", 0.0), ("f32", "xyz", 0.03), ("bf16s", "y", 0.0),
                                               ("f64", "yz", 0.0)])
def test_graph_replay_is_bit_identical(storage, walls, lid):
    """lb_step(n) on a non-default stream replays captured CUDA graphs of 64 steps; the
    result equals n single-step calls bit for bit, across both buffer parities and after
    a force change (which forces a new capture)."""
    from paper_2107_14774_gb300 import Lattice
    n = (24, 16, 12)
    rho, u = synth.solenoidal_random(*n, 0.5, 1.0, 2.0, 0.02, seed=31)
    out = []
    for mode in ("single", "batched"):
        stream = torch.cuda.Stream()
        lat = Lattice(*n, r_y=0.5, r_z=1.0, nu=0.02, storage=storage, walls=walls, lid_u=lid,
                      force=(1e-5, 0.0, 0.0), stream=stream)
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        for steps, F in ((201, (1e-5, 0.0, 0.0)), (130, (-2e-5, 1e-6, 0.0)), (65, (-2e-5, 1e-6, 0.0))):
            lat.set_force(F)
            if mode == "single":
                for _ in range(steps):
                    lat.step(1)
            else:
                lat.step(steps)
        assert lat.time_step == 396
        out.append(lat.populations().cpu().numpy())
        lat.close()
    assert np.array_equal(out[0], out[1])



@pytest.mark.parametrize("storage", ["f32", "f32s", "bf16s"])
def test_full_size_channel_768x192x384_sampled_nodes(oracle_mod, storage):
    """Channel 768x192x384 (r = 0.25, s = 1, cs2 = 1/48, nu = 0.005, walls normal
    to y, Poiseuille base flow plus a 5 % perturbation, uniform force), in the launch
    configuration the bench times, one fused step: for sampled nodes, wall rows included,
    the stored post-collision values against the oracle's collision of the same stored
    pre-collision values.  FP32: within 1e-5 of the node's largest deviation |f~ - w|
    (beyond the half ulp of the FP32 store and 16 FP32 ulps of w); BF16: the oracle's output rounded by its
    storage emulation, within one storage ulp (plus 16 FP32 ulps of w)."""
    from paper_2107_14774_gb300 import Lattice
    n, r, s, cs2, nu = (768, 192, 384), 0.25, 1.0, 1 / 48, 0.005
    rho, u, Fx = channel_768x192x384_inputs()
    lat = Lattice(*n, r_y=r, r_z=s, nu=nu, cs2=cs2, storage=storage, walls="y", force=(Fx, 0.0, 0.0))
    assert "k_step_pair" in lat.step_kernel
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    p = lat.params
    o = oracle_mod.Oracle(r=r, s=s, cs2=cs2, omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          storage_emulation="bf16s" if storage == "bf16s" else None)
    rng = np.random.default_rng(5)
    pts = [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1), (100, 0, 17), (5, n[1] - 1, 300)] + [
        tuple(int(rng.integers(0, m)) for m in n) for _ in range(10)]
    worst = sampled_step_errors(lat, o, n, pts, storage, F=(Fx, 0.0, 0.0), wall_y=True)
    lat.close()
    print(storage, "worst", worst)
    assert worst < (1e-5 if storage in ("f32", "f32s") else 1.0 + 1e-9)
