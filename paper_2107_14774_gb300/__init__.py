"""GB300-native fused collide-and-stream update of the cuboid-lattice D3Q27
central-moment lattice Boltzmann method (3DCCM-LBM, arXiv:2107.14774).

The numerics run in hand-written sm_103a CUDA kernels behind the C ABI of
``include/lbcuboid.h`` (``liblbcuboid.so``); this package only marshals
arguments (ctypes) and uses PyTorch for device memory and streams.
"""
from ._lib import (  # noqa: F401
    LB_BF16_SHIFTED, LB_CORR_FULL, LB_CORR_LOCAL, LB_CORR_LOWMACH, LB_CORR_NONE, LB_F16_SHIFTED, LB_F32,
    LB_F32_SHIFTED, LB_F64, LB_WALL_X, LB_WALL_Y, LB_WALL_Z, LBError, lb_config,
)
from .lattice import Lattice, STORAGE, CORR  # noqa: F401
from .autograd import KineticEnergyRollout, kinetic_energy_rollout  # noqa: F401
