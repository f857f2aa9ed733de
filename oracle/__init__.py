"""FP64 CPU oracle of the cuboid D3Q27 central-moment LB scheme (arXiv:2107.14774).

TEST INFRASTRUCTURE ONLY: this package is the slow, obviously-correct reference
against which the CUDA path is checked.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with ``paper_2107_14774_gb300`` and is never imported by it.

The numerics live in ``lbref.c`` (plain C, FP64, no FMA contraction); this module
only compiles it and marshals numpy arrays.  Parameter names follow the paper:
``r``/``s`` are the grid aspect ratios (Sec. 2.1), ``cs2`` the squared sound
speed, ``omega_nu``/``omega_xi`` the shear/bulk relaxation rates (App. D).
"""
from .lbref import (  # noqa: F401
    CORR_FULL,
    CORR_LOCAL,
    CORR_LOWMACH,
    CORR_NONE,
    Oracle,
    build,
    omega_from_viscosity,
)
