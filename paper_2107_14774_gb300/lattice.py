"""Python binding of one lattice context (argument marshalling only).

``Lattice`` owns an ``lb_ctx`` of liblbcuboid.  Inputs and outputs are torch
tensors; CUDA tensors are passed as device pointers, CPU tensors as host pointers
(the library stages those through its stream).  All numerics run in the CUDA
kernels behind the C ABI.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, lb_config, load

STORAGE = {"f64": _lib.LB_F64, "f32": _lib.LB_F32, "f32s": _lib.LB_F32_SHIFTED,
           "f16s": _lib.LB_F16_SHIFTED, "bf16s": _lib.LB_BF16_SHIFTED}
CORR = {"none": _lib.LB_CORR_NONE, "lowmach": _lib.LB_CORR_LOWMACH, "local": _lib.LB_CORR_LOCAL,
        "full": _lib.LB_CORR_FULL}
STORAGE_BYTES = {"f64": 8, "f32": 4, "f32s": 4, "f16s": 2, "bf16s": 2}


def _ptr(t) -> int:
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous()
        return t.data_ptr()
    assert isinstance(t, np.ndarray) and t.flags.c_contiguous
    return t.ctypes.data


class Lattice:
    """A cuboid D3Q27 lattice of nx x ny x nz nodes (x fastest).

    storage: "f64", "f32", "f32s" (shifted FP32), "f16s", "bf16s" (shifted FP16 /
    BF16, FP32 arithmetic).  corr: "none", "lowmach", "local", "full".
    walls: any of "x", "y", "z" (half-way bounce-back walls normal to that axis).
    kernel: "auto" (two-node kernel where possible), "one" (one node per thread), "pair" (two
    nodes per thread), "staged" (rows staged in shared memory by bulk copies), "march" (two
    nodes per thread marching along z, the next plane's sources staged in shared memory) or
    "onepass" (FULL corrections without the density pre-pass).
    rounding: "nearest" or "stochastic" (FP16/BF16 storage only).
    model: "central" (3DCCM) or "raw" (3DCRM: raw moments relaxed with the same corrected
    equilibria; LOCAL corrections only).
    subdomains: P > 1 steps the lattice as P z-slabs exchanging one-plane halos through
    device memory (bit-identical to one domain; z periodic, no FULL, no force field).
    """

    def __init__(self, nx, ny, nz, r_y=1.0, r_z=1.0, nu=0.01, zeta=0.0, cs2=0.0, storage="f32",
                 corr="local", walls="", force=(0.0, 0.0, 0.0), lid_u=0.0, stream=None, device=None,
                 kernel="auto", rounding="nearest", rounding_seed=0, model="central", subdomains=1):
        self.lib = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = s
        cfg = lb_config()
        self.lib.lb_config_default(ctypes.byref(cfg), nx, ny, nz, r_y, r_z, nu)
        cfg.zeta, cfg.cs2 = zeta, cs2
        cfg.storage, cfg.corr = STORAGE[storage], CORR[corr]
        cfg.wall_mask = sum(m for c, m in zip("xyz", (1, 2, 4)) if c in walls)
        cfg.force = (ctypes.c_double * 3)(*force)
        cfg.lid_u = lid_u
        cfg.stream = s.cuda_stream
        cfg.kernel = {"auto": 0, "one": 1, "pair": 2, "staged": 3, "march": 4, "onepass": 5}[kernel]
        cfg.rounding = {"nearest": 0, "stochastic": 1}[rounding]
        cfg.rounding_seed = rounding_seed
        cfg.model = {"central": 0, "raw": 1}[model]
        cfg.subdomains = int(subdomains)
        self.cfg = cfg
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.storage = storage
        self.dtype = torch.float64 if storage == "f64" else torch.float32
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.lb_create_ex(ctypes.byref(cfg), ctypes.byref(ctx)))
        self.ctx = ctx

    # ------------------------------------------------------------------ basics
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def params(self):
        out = (ctypes.c_double * 3)()
        check(self.lib.lb_get_params(self.ctx, out))
        return {"omega_nu": out[0], "omega_xi": out[1], "cs2": out[2]}

    @property
    def step_kernel(self) -> str:
        """lb_step_kernel: the step kernel lb_step launches for this lattice."""
        return self.lib.lb_step_kernel(self.ctx).decode()

    @property
    def time_step(self) -> int:
        return self.lib.lb_time_step(self.ctx)

    def _after_caller(self):
        """Order the context's stream after the caller's current stream (inputs written
        there, output buffers allocated there)."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _before_caller(self):
        """Order the caller's current stream after the context's stream (device outputs)."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def _real(self, x, shape):
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(x)
        x = x.to(dtype=self.dtype).reshape(shape).contiguous()
        if x.is_cuda and x.device != self.device:
            x = x.to(self.device)
        return x

    # ---------------------------------------------------------------- C ABI
    def init(self, rho, u):
        """lb_init: f := f^eq(rho, u) at every node."""
        rho = self._real(rho, self.shape)
        u = self._real(u, (3,) + self.shape)
        self._after_caller()
        check(self.lib.lb_init(self.ctx, _ptr(rho), _ptr(u)))
        self._keep = (rho, u)  # keep inputs alive until the stream has consumed them
        return self

    def set_force_field(self, force):
        """lb_set_force_field: per-node body force [3][nz][ny][nx] (None removes it)."""
        if force is None:
            check(self.lib.lb_set_force_field(self.ctx, None))
            return
        force = self._real(force, (3,) + self.shape)
        self._after_caller()
        check(self.lib.lb_set_force_field(self.ctx, _ptr(force)))
        self._keep_force = force

    def step(self, n: int = 1):
        """lb_step: enqueue n fused collide-and-stream steps."""
        check(self.lib.lb_step(self.ctx, int(n)))
        return self

    def moments(self, rho=None, u=None):
        """lb_moments: density [nz,ny,nx] and velocity [3,nz,ny,nx]."""
        if rho is None:
            rho = torch.empty(self.shape, dtype=self.dtype, device=self.device)
        if u is None:
            u = torch.empty((3,) + self.shape, dtype=self.dtype, device=self.device)
        self._after_caller()
        check(self.lib.lb_moments(self.ctx, _ptr(rho), _ptr(u)))
        self._before_caller()
        return rho, u

    def reduce(self, allow_unstable: bool = False) -> np.ndarray:
        """lb_reduce: FP64 (sum rho, sum rho u)."""
        out = (ctypes.c_double * 4)()
        st = self.lib.lb_reduce(self.ctx, out)
        if st != _lib.LB_OK and not (allow_unstable and st == _lib.LB_EUNSTABLE):
            check(st)
        return np.array(list(out))

    def is_stable(self) -> bool:
        """lb_reduce's status: False once a density is non-positive or not finite."""
        out = (ctypes.c_double * 4)()
        st = self.lib.lb_reduce(self.ctx, out)
        if st == _lib.LB_EUNSTABLE:
            return False
        check(st)
        return bool(np.all(np.isfinite(np.array(list(out)))))

    def populations(self, out=None):
        """lb_get_populations: pre-collision f [27,nz,ny,nx]."""
        if out is None:
            out = torch.empty((27,) + self.shape, dtype=self.dtype, device=self.device)
        self._after_caller()
        check(self.lib.lb_get_populations(self.ctx, _ptr(out)))
        self._before_caller()
        return out

    def set_populations(self, f):
        f = self._real(f, (27,) + self.shape)
        self._after_caller()
        check(self.lib.lb_set_populations(self.ctx, _ptr(f)))
        return self

    def state_bytes(self) -> int:
        return self.lib.lb_state_bytes(self.ctx)

    def get_state(self, out=None):
        """lb_get_state: raw stored state (bit-exact checkpoint)."""
        if out is None:
            out = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        self._after_caller()
        check(self.lib.lb_get_state(self.ctx, _ptr(out)))
        self._before_caller()
        return out

    def set_state(self, state, time_step: int = 0):
        self._after_caller()
        check(self.lib.lb_set_state(self.ctx, _ptr(state), int(time_step)))
        return self

    # ------------------------------------------------------------ adjoint
    def set_force(self, force):
        """lb_set_force: uniform body force for the following steps."""
        check(self.lib.lb_set_force(self.ctx, (ctypes.c_double * 3)(*[float(v) for v in force])))
        return self

    def set_rates(self, omega_nu: float, omega_xi: float):
        """lb_set_rates: relaxation rates directly (0 < omega < 2)."""
        check(self.lib.lb_set_rates(self.ctx, float(omega_nu), float(omega_xi)))
        return self

    def set_lid(self, lid_u: float):
        """lb_set_lid: lid velocity (x velocity of the wall at the top in y) for the following steps."""
        check(self.lib.lb_set_lid(self.ctx, float(lid_u)))
        return self

    def objective_ke(self) -> float:
        """lb_objective_ke: mean kinetic energy of the current state (FP64 sum)."""
        out = ctypes.c_double()
        check(self.lib.lb_objective_ke(self.ctx, ctypes.byref(out)))
        return out.value

    def adjoint_ke(self, T: int, K: int, dJdF=None):
        """lb_adjoint_ke: run T steps and the discrete adjoint of the mean kinetic
        energy; returns (J, dJ/dF [3,nz,ny,nx], (dJ/domega_nu, dJ/domega_xi))."""
        if dJdF is None:
            dJdF = torch.empty((3,) + self.shape, dtype=self.dtype, device=self.device)
        dw = (ctypes.c_double * 2)()
        J = ctypes.c_double()
        self._after_caller()
        check(self.lib.lb_adjoint_ke(self.ctx, int(T), int(K), _ptr(dJdF), dw, ctypes.byref(J)))
        self._before_caller()
        return J.value, dJdF, (dw[0], dw[1])

    def collide_vjp(self, f, F, lam):
        """lb_collide_vjp: per-node VJP of the collision for n nodes ([27,n], [3,n], [27,n])."""
        n = f.shape[1]
        f, F, lam = (x.to(self.device, self.dtype).contiguous() for x in (f, F, lam))
        fb = torch.empty_like(f)
        Fb = torch.empty_like(F)
        wb = (ctypes.c_double * 2)()
        self._after_caller()
        check(self.lib.lb_collide_vjp(self.ctx, n, _ptr(f), _ptr(F), _ptr(lam), _ptr(fb), _ptr(Fb), wb))
        self._before_caller()
        return fb, Fb, (wb[0], wb[1])
