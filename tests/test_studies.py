"""The study drivers of Secs. 6-7: bisection logic on the CPU, one small run of each
driver on the GPU."""
import math

import numpy as np
import pytest


def test_bisect_finds_monotone_threshold():
    from paper_2107_14774_gb300.studies import bisect
    calls = []

    def stable(x):
        calls.append(x)
        return x <= 0.137

    x = bisect(stable, 0.0, 0.4, 0.005)
    assert 0.137 - 0.005 <= x <= 0.137 and len(calls) <= 8
    assert bisect(lambda v: True, 0.0, 0.4, 0.005) == 0.4
    assert bisect(lambda v: False, 0.0, 0.4, 0.005) < 0.005


class _Recorder:
    """Stands in for a Lattice: records lid changes and step counts; never unstable."""

    def __init__(self):
        self.log, self.t = [], 0

    def set_lid(self, u):
        self.log.append(("lid", self.t, u))
        return self

    def step(self, k):
        self.t += k
        self.log.append(("step", k))
        return self

    def is_stable(self):
        self.log.append(("check", self.t))
        return True


def test_survives_ramps_the_lid_then_holds_it():
    """With a ramp the lid rises linearly to U in equal increments over ramp_steps steps and
    then stays at U; the stability checks fall on multiples of check_every and at the end."""
    from paper_2107_14774_gb300.studies import survives
    lat = _Recorder()
    assert survives(lat, 1250, check_every=500, lid_u=0.2, ramp_steps=400, ramp_every=100)
    lids = [(t, u) for kind, t, u in (e for e in lat.log if e[0] == "lid")]
    assert [t for t, _ in lids[:4]] == [0, 100, 200, 300]
    assert np.allclose([u for _, u in lids[:4]], [0.05, 0.1, 0.15, 0.2])
    assert all(u == 0.2 for _, u in lids[4:])
    assert lat.t == 1250
    assert [e[1] for e in lat.log if e[0] == "check"] == [500, 1000, 1250]
    plain = _Recorder()
    assert survives(plain, 1250, check_every=500)
    assert not any(e[0] == "lid" for e in plain.log)
    assert [e[1] for e in plain.log if e[0] == "step"] == [500, 500, 250]


@pytest.mark.gpu
def test_stability_driver_small():
    """A tiny cavity: a lid at rest-like speed survives, the bisected threshold lies inside
    the bracket, and the raw scheme's threshold is no higher than the central one's at a
    low viscosity (Sec. 7)."""
    from paper_2107_14774_gb300 import studies
    lat = studies.lid_cavity(12, 16, 12, 0.75, 1.0, 0.08, 0.01, 1.5)
    assert studies.survives(lat, 500, 250)
    lat.close()
    u_c = studies.max_stable_lid_velocity(12, 16, 12, 0.75, 1.0, 0.08, 1.97, steps=3000, u_hi=0.5, tol=0.02)
    u_r = studies.max_stable_lid_velocity(12, 16, 12, 0.75, 1.0, 0.08, 1.97, model="raw", steps=3000, u_hi=0.5,
                                          tol=0.02)
    print("U_max central %.3f raw %.3f" % (u_c, u_r))
    assert 0.0 < u_c <= 0.5 and 0.0 < u_r <= 0.5


@pytest.mark.gpu
def test_shallow_cavity_driver_small():
    from paper_2107_14774_gb300 import studies
    c = studies.shallow_cavity(32, 8, 16, 1.0, 1.0, 1 / 3, 0.05, Re=20.0, transits=3.0)
    assert c["stable"] and c["steps"] == round(3.0 * 32 / 0.05)
    assert c["u"].shape == (8,) and c["v"].shape == (32,)
    assert c["u"][-1] > 0.0 > c["u"].min()          # dragged along under the lid, return flow below


@pytest.mark.gpu
@pytest.mark.parametrize("model", ["central", "raw"])
def test_study_cavity_matches_oracle(oracle_mod, model):
    """The configuration the Sec. 7 studies run (closed box, lid, rates set directly with
    omega_xi = 0.5, own stream, graph replay), FP64 storage, 150 steps: within 1e-12 of
    the oracle."""
    from paper_2107_14774_gb300 import studies
    n, r, s, cs2, U = (12, 16, 12), 0.75, 1.0, 0.08, 0.05
    lat = studies.lid_cavity(*n, r, s, cs2, U, 1.9, 0.5, model=model, storage="f64")
    lat.step(150)
    fg = lat.populations().cpu().numpy()
    lat.close()
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=cs2, omega_nu=1.9, omega_xi=0.5, walls="xyz", lid_u=U, model=model)
    f = o.run(o.init(np.ones(n[::-1]), np.zeros((3,) + n[::-1])), 150)
    assert np.linalg.norm(fg - f) / np.linalg.norm(f) < 1e-12
