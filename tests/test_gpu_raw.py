"""The raw-moment scheme (3DCRM, Sec. 7) on the GPU against the oracle's raw-moment
collision (FP64 <= 1e-12; FP32 <= 1e-5 on rho and u) in every kernel that runs it."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _pair(oracle_mod, n, r, s, nu, storage="f64", walls="", force=(0.0, 0.0, 0.0), lid_u=0.0, cs2=0.0,
          kernel="auto", **kw):
    from paper_2107_14774_gb300 import Lattice
    lat = Lattice(*n, r_y=r, r_z=s, nu=nu, cs2=cs2, storage=storage, walls=walls, force=force, lid_u=lid_u,
                  model="raw", kernel=kernel, **kw)
    p = lat.params
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          walls=walls, force=force, lid_u=lid_u, model="raw")
    return lat, o


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,r,s,walls,lid", [
    ((37, 12, 9), 0.5, 2.0, "", 0.0),
    ((20, 12, 9), 1.0, 0.5, "y", 0.0),
    ((16, 10, 12), 0.5, 1.0, "yz", 0.0),
    ((9, 7, 6), 0.406, 1.3, "xyz", 0.04),
])
def test_raw_model_fp64_parity(oracle_mod, n, r, s, walls, lid):
    rho, u = synth.solenoidal_random(*n, r, s, 2.0, 0.03, seed=12)
    F = (2e-5, -1e-5, 5e-6)
    lat, o = _pair(oracle_mod, n, r, s, 0.02, walls=walls, force=F, lid_u=lid)
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).step(6)
    fg = lat.populations().cpu().numpy()
    assert "RAW" in lat.step_kernel
    fr = o.run(o.init(rho, u), 6)
    assert _rel(fg, fr) < 1e-12
    lat.close()


@pytest.mark.parametrize("kernel", ["auto", "one", "pair"])
@pytest.mark.parametrize("storage", ["f32", "f32s"])
def test_raw_model_fp32_kernels(oracle_mod, kernel, storage):
    n, r, s = (32, 24, 16), 0.5, 0.75
    rho, u = synth.solenoidal_random(*n, r, s, 3.0, 0.03, seed=13)
    lat, o = _pair(oracle_mod, n, r, s, 0.01, storage=storage, walls="y", force=(1e-5, 0.0, 2e-6),
                   kernel=kernel)
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).step(8)
    rg, ug = (t.cpu().numpy() for t in lat.moments())
    name = lat.step_kernel
    assert "RAW" in name and ("k_step<" in name) == (kernel == "one")
    rr, ur = o.moments(o.run(o.init(rho, u), 8))
    assert _rel(ug, ur) < 1e-5 and _rel(rg, rr) < 1e-5
    lat.close()


def test_raw_and_central_differ_on_the_gpu():
    """The model switch acts: the same state stepped by both schemes differs, and at rest
    (no force) both keep it."""
    from paper_2107_14774_gb300 import Lattice
    n = (16, 16, 16)
    rho, u = synth.solenoidal_random(*n, 0.5, 1.0, 2.0, 0.05, seed=14)
    out = {}
    for model in ("central", "raw"):
        lat = Lattice(*n, r_y=0.5, r_z=1.0, nu=0.01, storage="f64", model=model)
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).step(5)
        out[model] = lat.populations().cpu().numpy()
        lat.close()
    assert _rel(out["raw"], out["central"]) > 1e-9


def test_raw_model_rejects_other_modes():
    from paper_2107_14774_gb300 import Lattice, LBError
    with pytest.raises(LBError):
        Lattice(8, 8, 8, nu=0.01, corr="full", model="raw")
