"""z-slab decomposition on one GPU (lb_config.subdomains = P): the lattice is updated
as P slabs with one ghost plane on either side, exchanging the 9 populations with
e_z = +1 / -1 of their boundary planes through device memory after every step while
the interiors update on a second stream.  Every node sees the same pre-collision
values as in the whole lattice and runs the same kernel, so the stored state must be
bit-identical to the single-domain run."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

# (dims, r, s, storage, walls, force, rounding, kernel, P); nz = 13 splits unevenly
CASES = [
    ((24, 10, 13), 0.5, 2.0, "f32", "", (1e-5, 0.0, 0.0), "nearest", "auto", 2),
    ((24, 10, 13), 0.5, 2.0, "f32", "y", (1e-5, -2e-6, 0.0), "nearest", "auto", 3),
    ((24, 10, 13), 1.0, 0.5, "f32s", "xy", (0.0, 1e-5, 0.0), "nearest", "auto", 4),   # x walls: one-node kernel
    ((24, 10, 13), 0.5, 0.5, "bf16s", "", (0.0, 0.0, 0.0), "nearest", "auto", 6),     # slabs of 2 and 3 planes
    ((24, 10, 13), 0.5, 0.5, "f16s", "y", (2e-6, 0.0, 0.0), "stochastic", "auto", 3),
    ((24, 10, 13), 0.5, 0.5, "bf16s", "", (0.0, 0.0, 0.0), "stochastic", "one", 13),  # one plane per slab
    ((20, 12, 13), 0.5, 2.0, "f64", "y", (1e-5, 0.0, 0.0), "nearest", "auto", 5),
    # z-marching 16-bit kernel on the slab interiors (plane ranges that start past a ghost plane)
    ((128, 10, 21), 0.5, 0.5, "bf16s", "", (0.0, 0.0, 0.0), "nearest", "march", 3),
    ((128, 10, 21), 0.5, 0.5, "f16s", "y", (2e-6, 0.0, 0.0), "stochastic", "march", 4),
]


def run(n, r, s, storage, walls, force, rounding, kernel, P, steps_list):
    from paper_2107_14774_gb300 import Lattice
    rho, u = synth.solenoidal_random(*n, r, s, 2.0, 0.03, seed=21)
    rho = rho + 0.01 * np.cos(2 * np.pi * np.arange(n[2]) / n[2])[:, None, None]
    lat = Lattice(*n, r_y=r, r_z=s, nu=0.01, storage=storage, walls=walls, force=force, rounding=rounding,
                  rounding_seed=7, kernel=kernel, subdomains=P, stream=torch.cuda.Stream())
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    states = []
    for k in steps_list:           # several lb_step calls: the state goes into the slabs and back each time
        lat.step(k)
        states.append(lat.get_state().cpu())
    kern = lat.step_kernel
    lat.close()
    return states, kern


@pytest.mark.parametrize("n,r,s,storage,walls,force,rounding,kernel,P", CASES)
def test_subdomains_bit_identical_to_whole_lattice(n, r, s, storage, walls, force, rounding, kernel, P):
    """70 steps (one plain step, a 64-step CUDA graph and 5 plain steps), then 3 more in
    a second call: every stored byte equals the single-domain run."""
    whole, kern = run(n, r, s, storage, walls, force, rounding, kernel, 1, [70, 3])
    slabs, kern_p = run(n, r, s, storage, walls, force, rounding, kernel, P, [70, 3])
    assert kern == kern_p
    for a, b in zip(whole, slabs):
        assert torch.equal(a, b)
    assert not torch.equal(whole[0], whole[1])


def test_subdomains_legacy_default_stream_and_moments():
    """On the legacy default stream (no graphs) the decomposed run also matches, and the
    macroscopic fields and FP64 sums read the gathered state."""
    from paper_2107_14774_gb300 import Lattice
    n = (16, 8, 9)
    rho, u = synth.solenoidal_random(*n, 1.0, 1.0, 2.0, 0.02, seed=3)
    out = []
    for P in (1, 3):
        lat = Lattice(*n, nu=0.02, storage="f32", subdomains=P, stream=torch.cuda.default_stream())
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).step(5)
        r_, u_ = lat.moments()
        out.append((lat.get_state().cpu(), r_.cpu(), u_.cpu(), lat.reduce()))
        lat.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1]) and torch.equal(out[0][2], out[1][2])
    assert np.array_equal(out[0][3], out[1][3])


@pytest.mark.parametrize("kw", [dict(walls="z"), dict(corr="full"), dict(kernel="staged"), dict(subdomains=17),
                                dict(subdomains=10)])
def test_subdomains_rejected_configurations(kw):
    from paper_2107_14774_gb300 import Lattice
    from paper_2107_14774_gb300._lib import LBError, LB_EINVAL
    args = dict(subdomains=2)
    args.update(kw)
    with pytest.raises(LBError) as e:
        Lattice(32, 8, 9, **args)
    assert e.value.status == LB_EINVAL


def test_subdomains_refuse_force_field():
    from paper_2107_14774_gb300 import Lattice
    from paper_2107_14774_gb300._lib import LBError, LB_EINVAL
    lat = Lattice(8, 8, 8, subdomains=2)
    with pytest.raises(LBError) as e:
        lat.set_force_field(torch.zeros(3, 8, 8, 8).cuda())
    assert e.value.status == LB_EINVAL
    lat.close()


def test_subdomains_with_lid_changed_between_steps():
    """A lid at the top y wall whose velocity changes between lb_step calls (lb_set_lid):
    the decomposed run stores the same bytes as the whole lattice after every call."""
    from paper_2107_14774_gb300 import Lattice
    n = (24, 12, 13)
    rho, u = np.ones(n[::-1]), np.zeros((3,) + n[::-1])
    out = []
    for P in (1, 3):
        lat = Lattice(*n, r_y=0.5, r_z=1.0, nu=0.02, storage="f32", walls="y", lid_u=0.02, subdomains=P,
                      stream=torch.cuda.Stream())
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        states = []
        for lid, k in ((0.02, 3), (0.05, 70), (0.0, 2)):
            lat.set_lid(lid).step(k)
            states.append(lat.get_state().cpu())
        out.append(states)
        lat.close()
    for a, b in zip(*out):
        assert torch.equal(a, b)
