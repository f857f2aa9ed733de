"""Failure detection on the GPU without a fault: the bounded mbarrier wait of the
row-staged kernel gives up on a phase that nothing completes and reports it, and the
context stays usable afterwards."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports():
    from paper_2107_14774_gb300 import Lattice
    from paper_2107_14774_gb300._lib import check, load
    lib = load()
    out = (ctypes.c_int * 2)(-1, -1)
    check(lib.lb_selftest_bounded_wait(out))
    assert out[0] == 1, "the wait on a phase nobody completes must time out"
    assert out[1] == 1, "the wait must succeed once the phase completes"
    lat = Lattice(16, 8, 8, nu=0.02, kernel="staged")
    lat.init(torch.ones(8, 8, 16).cuda(), torch.zeros(3, 8, 8, 16).cuda()).step(3)
    assert np.allclose(lat.reduce()[0], 16 * 8 * 8)     # no error word set by the staged kernel
    lat.close()
