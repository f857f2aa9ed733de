"""lb_reduce_populations_noalloc -- the reduction entry point for callers that cannot
allocate device memory (hosts whose framework owns all device memory, real-time
loops) -- against the existing lb_reduce entry point and against sums of the FP64
oracle's moments of the same populations, on two calls in a row.  Collected last
(file name) so that a failure here never hides the other tests of a run that stops
at the first failure."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_noalloc_reduction_matches_lb_reduce_and_oracle_twice(oracle_mod, storage, tol):
    """Same sums as lb_reduce within the parity tolerance of the storage type (FP64
    1e-12; FP32 1e-5: lb_reduce sums FP32 per-node moments, this entry point sums
    the FP32-rounded populations in FP64), and the same sums as the oracle's moments
    (Eq. 12: rho = sum f, rho u = sum f e + F/2) of the very populations it was given,
    within 1e-12 for both storage forms (both sides add the same numbers in FP64)."""
    from paper_2107_14774_gb300 import Lattice
    from paper_2107_14774_gb300._lib import LB_OK, load
    lib = load()
    n, r, s = (24, 20, 12), 0.5, 2.0
    F = (1e-5, -2e-5, 3e-6)
    rho, u = synth.solenoidal_random(*n, r, s, 3.0, 0.02, seed=12)
    lat = Lattice(*n, r_y=r, r_z=s, nu=0.02, storage=storage, walls="y", force=F)
    p = lat.params
    o = oracle_mod.Oracle(*n, r=r, s=s, cs2=p["cs2"], omega_nu=p["omega_nu"], omega_xi=p["omega_xi"],
                          walls="y", force=F)
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    force = (ctypes.c_double * 3)(*F)
    scale = np.sqrt((u ** 2).sum(0)).sum()
    for _ in range(2):
        lat.step(3)
        want = lat.reduce()
        f = lat.populations()
        torch.cuda.synchronize()
        out = (ctypes.c_double * 4)()
        st = lib.lb_reduce_populations_noalloc(ctypes.c_void_p(f.data_ptr()), f.element_size(), lat.N, r, s, force,
                                               out, ctypes.c_void_p(lat.stream.cuda_stream))
        assert st == LB_OK, lib.lb_last_error().decode()
        got = np.array(list(out))
        # mass relative to itself; momentum relative to the total |rho u| of the flow
        assert got[0] == pytest.approx(want[0], rel=tol)
        np.testing.assert_allclose(got[1:], want[1:], rtol=0, atol=tol * scale)
        rr, ur = o.moments(f.double().cpu().numpy())
        ref = np.array([rr.sum(), *(rr[None] * ur).reshape(3, -1).sum(1)])
        assert got[0] == pytest.approx(ref[0], rel=1e-12)
        np.testing.assert_allclose(got[1:], ref[1:], rtol=0, atol=1e-12 * scale)
    lat.close()


def test_noalloc_reduction_rejects_oversized_input():
    from paper_2107_14774_gb300._lib import LB_EINVAL, load
    lib = load()
    out = (ctypes.c_double * 4)()
    dummy = torch.zeros(27, device="cuda")
    st = lib.lb_reduce_populations_noalloc(ctypes.c_void_p(dummy.data_ptr()), 4, 134217729, 1.0, 1.0, None, out, None)
    assert st == LB_EINVAL and "exceeds the maximum" in lib.lb_last_error().decode()


def test_noalloc_reduction_rejects_host_memory():
    """Host memory (a numpy array, a pinned torch tensor) is refused with LB_EINVAL
    before any kernel is launched."""
    from paper_2107_14774_gb300._lib import LB_EINVAL, load
    lib = load()
    out = (ctypes.c_double * 4)()
    host = np.full(27 * 8, 1.0 / 27.0)
    st = lib.lb_reduce_populations_noalloc(ctypes.c_void_p(host.ctypes.data), 8, 8, 1.0, 1.0, None, out, None)
    assert st == LB_EINVAL and "host memory" in lib.lb_last_error().decode()
    pinned = torch.full((27 * 8,), 1.0 / 27.0, dtype=torch.float64).pin_memory()
    st = lib.lb_reduce_populations_noalloc(ctypes.c_void_p(pinned.data_ptr()), 8, 8, 1.0, 1.0, None, out, None)
    assert st == LB_EINVAL
    torch.cuda.synchronize()
