"""ctypes marshalling for the FP64 C oracle ``lbref.c`` (test infrastructure only).

Arrays follow the layout ``[27][nz][ny][nx]`` (x fastest) for populations,
``[nz][ny][nx]`` for the density and ``[3][nz][ny][nx]`` for velocity/force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

CORR_NONE, CORR_LOWMACH, CORR_LOCAL, CORR_FULL = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbref.c")
_LIB = os.path.join(_HERE, "liblbref.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``lbref.c`` into ``liblbref.so`` (gcc, OpenMP, no FP contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                   "-Wall", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_mask", ctypes.c_uint),
        ("r", ctypes.c_double), ("s", ctypes.c_double), ("cs2", ctypes.c_double),
        ("omega_nu", ctypes.c_double), ("omega_xi", ctypes.c_double),
        ("corr", ctypes.c_int), ("form", ctypes.c_int),
        ("force", ctypes.c_double * 3),
        ("force_field", ctypes.c_void_p),
        ("lid_u", ctypes.c_double),
        ("model", ctypes.c_int),
        ("storage_emulation", ctypes.c_int),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_Params)
        d = ctypes.c_void_p
        for name, args in [
            ("or_collide_all", [P, d, d]), ("or_stream", [P, d, d]), ("or_step", [P, d, d]),
            ("or_run", [P, d, ctypes.c_int]), ("or_init", [P, d, d, d]),
            ("or_moments", [P, d, d, d]), ("or_collide_node", [P, d, d, d, d]),
            ("or_equilibrium", [P, ctypes.c_double, d, d]),
            ("or_num_threads", [ctypes.c_int]), ("or_quantize", [P, d]),
        ]:
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        for name in ("or_round_binary16", "or_round_bfloat16"):
            fn = getattr(_lib, name)
            fn.argtypes = [ctypes.c_double]
            fn.restype = ctypes.c_double
        _lib.or_relax_central.argtypes = [P, d, ctypes.c_double, d, d, d, d]
        _lib.or_relax_central.restype = None
        _lib.or_strain_rates.argtypes = [P, d, ctypes.c_double, d, d, ctypes.c_int, d]
        _lib.or_strain_rates.restype = None
        for name, args in [("or_matrix_P", [d]), ("or_matrix_Pinv", [d]),
                           ("or_matrix_S", [ctypes.c_double, ctypes.c_double, d]),
                           ("or_matrix_F", [d, d]),
                           ("or_matrix_M", [ctypes.c_double, ctypes.c_double, d, d]),
                           ("or_velocities", [d, d, d]), ("or_moment_exponents", [d, d, d]),
                           ("or_central_equilibrium", [ctypes.c_double, ctypes.c_double, d]),
                           ("or_raw_equilibrium", [ctypes.c_double, ctypes.c_double, d, d])]:
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = None
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags.c_contiguous
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def omega_from_viscosity(nu: float, xi: float, cs2: float) -> tuple[float, float]:
    """Relaxation rates from the transport coefficients (Eq. 53):
    nu = cs2 (1/omega_nu - 1/2),  xi = (2 cs2 / 3)(1/omega_xi - 1/2)."""
    return 1.0 / (nu / cs2 + 0.5), 1.0 / (1.5 * xi / cs2 + 0.5)


class Oracle:
    """FP64 oracle for one lattice configuration.

    ``corr``: CORR_NONE / CORR_LOWMACH / CORR_LOCAL / CORR_FULL.  ``form``: 0
    factored (P, S, F(u) of Sec. 3.1), 1 definitional (Eq. 3a with an LU solve).
    ``walls``: string with any of "x", "y", "z" naming the non-periodic axes.
    ``model``: "central" (3DCCM, the collision in central moments) or "raw" (3DCRM: the
    same corrected equilibria relaxed in raw moments, Sec. 7).
    ``storage_emulation``: None, "f16s" or "bf16s": round the stored deviations from the
    rest weights after every collision and after ``init`` (binary16 scaled by
    2^(10 - ilogb w_a), or bfloat16; round to nearest, ties to even).
    """

    def __init__(self, nx=1, ny=1, nz=1, r=1.0, s=1.0, cs2=None, omega_nu=1.0, omega_xi=1.0,
                 corr=CORR_LOCAL, form=0, walls="", force=(0.0, 0.0, 0.0), force_field=None,
                 lid_u=0.0, threads=0, storage_emulation=None, model="central"):
        self.lib = _load()
        if cs2 is None:
            cs2 = min(1.0, r * r, s * s) / 3.0
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self._ff = None if force_field is None else _f64(force_field).reshape(3, self.N)
        p = _Params()
        p.nx, p.ny, p.nz = nx, ny, nz
        p.wall_mask = sum(1 << i for i, c in enumerate("xyz") if c in walls)
        p.r, p.s, p.cs2 = r, s, cs2
        p.omega_nu, p.omega_xi = omega_nu, omega_xi
        p.corr, p.form = corr, form
        p.force = (ctypes.c_double * 3)(*force)
        p.force_field = None if self._ff is None else _ptr(self._ff)
        p.lid_u = lid_u
        p.storage_emulation = {None: 0, "f16s": 1, "bf16s": 2}[storage_emulation]
        p.model = {"central": 0, "raw": 1}[model]
        self.p = p
        self.pp = ctypes.byref(p)
        if threads:
            self.lib.or_num_threads(threads)

    @property
    def threads(self) -> int:
        return self.lib.or_num_threads(0)

    def set_force(self, force):
        """Uniform body force for the following steps (a time-dependent forcing)."""
        self.p.force = (ctypes.c_double * 3)(*[float(v) for v in force])

    # ---- single node -------------------------------------------------------
    def collide_node(self, f, F=(0.0, 0.0, 0.0), grad_rho=(0.0, 0.0, 0.0)) -> np.ndarray:
        f, F, g = _f64(f), _f64(F), _f64(grad_rho)
        out = np.empty(27)
        if self.lib.or_collide_node(self.pp, _ptr(f), _ptr(F), _ptr(g), _ptr(out)):
            raise FloatingPointError("singular system in the oracle collision")
        return out

    def equilibrium(self, rho, u) -> np.ndarray:
        u = _f64(u)
        out = np.empty(27)
        self.lib.or_equilibrium(self.pp, float(rho), _ptr(u), _ptr(out))
        return out

    def relax_central(self, k, rho, u, F=(0, 0, 0), grad_rho=(0, 0, 0)) -> np.ndarray:
        k, u, F, g = _f64(k), _f64(u), _f64(F), _f64(grad_rho)
        out = np.empty(27)
        self.lib.or_relax_central(self.pp, _ptr(k), float(rho), _ptr(u), _ptr(F), _ptr(g), _ptr(out))
        return out

    def strain_rates(self, k, rho, u, grad_rho=(0, 0, 0), aliasing=True) -> np.ndarray:
        k, u, g = _f64(k), _f64(u), _f64(grad_rho)
        out = np.empty(3)
        self.lib.or_strain_rates(self.pp, _ptr(k), float(rho), _ptr(u), _ptr(g), int(aliasing), _ptr(out))
        return out

    # ---- whole lattice -----------------------------------------------------
    def init(self, rho, u) -> np.ndarray:
        rho = _f64(rho).reshape(self.N)
        u = _f64(u).reshape(3, self.N)
        f = np.empty((27, self.N))
        if self.lib.or_init(self.pp, _ptr(rho), _ptr(u), _ptr(f)):
            raise FloatingPointError("oracle init failed")
        return f.reshape((27,) + self.shape)

    def collide_all(self, f) -> np.ndarray:
        f = _f64(f)
        out = np.empty_like(f)
        if self.lib.or_collide_all(self.pp, _ptr(f), _ptr(out)):
            raise FloatingPointError("oracle collision failed")
        return out

    def stream(self, ft) -> np.ndarray:
        ft = _f64(ft)
        out = np.empty_like(ft)
        self.lib.or_stream(self.pp, _ptr(ft), _ptr(out))
        return out

    def step(self, f) -> np.ndarray:
        f = _f64(f)
        out = np.empty_like(f)
        if self.lib.or_step(self.pp, _ptr(f), _ptr(out)):
            raise FloatingPointError("oracle step failed")
        return out

    def run(self, f, steps: int) -> np.ndarray:
        f = _f64(f).copy()
        if self.lib.or_run(self.pp, _ptr(f), int(steps)):
            raise FloatingPointError("oracle run failed")
        return f

    def quantize(self, f) -> np.ndarray:
        """The rounding of the storage emulation applied to populations f (a copy)."""
        f = _f64(f).copy()
        if self.lib.or_quantize(self.pp, _ptr(f)):
            raise ValueError("bad storage emulation mode")
        return f

    def moments(self, f):
        f = _f64(f)
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        self.lib.or_moments(self.pp, _ptr(f), _ptr(rho), _ptr(u))
        return rho, u

    # ---- matrices (Sec. 3.1) -----------------------------------------------
    def P(self) -> np.ndarray:
        out = np.empty((27, 27)); self.lib.or_matrix_P(_ptr(out)); return out

    def Pinv(self) -> np.ndarray:
        out = np.empty((27, 27)); self.lib.or_matrix_Pinv(_ptr(out)); return out

    def S(self) -> np.ndarray:
        out = np.empty(27); self.lib.or_matrix_S(self.p.r, self.p.s, _ptr(out)); return out

    def F(self, u) -> np.ndarray:
        u = _f64(u); out = np.empty((27, 27)); self.lib.or_matrix_F(_ptr(u), _ptr(out)); return out

    def M(self, u) -> np.ndarray:
        u = _f64(u); out = np.empty((27, 27))
        self.lib.or_matrix_M(self.p.r, self.p.s, _ptr(u), _ptr(out)); return out

    def central_equilibrium(self, rho) -> np.ndarray:
        out = np.empty(27); self.lib.or_central_equilibrium(self.p.cs2, float(rho), _ptr(out)); return out

    def raw_equilibrium(self, rho, u) -> np.ndarray:
        u = _f64(u); out = np.empty(27)
        self.lib.or_raw_equilibrium(self.p.cs2, float(rho), _ptr(u), _ptr(out)); return out

    @staticmethod
    def round_binary16(x: float) -> float:
        return _load().or_round_binary16(float(x))

    @staticmethod
    def round_bfloat16(x: float) -> float:
        return _load().or_round_bfloat16(float(x))

    @staticmethod
    def velocities() -> np.ndarray:
        lib = _load()
        e = np.empty((3, 27), dtype=np.int32)
        lib.or_velocities(_ptr(e[0]), _ptr(e[1]), _ptr(e[2]))
        return e

    @staticmethod
    def moment_exponents() -> np.ndarray:
        lib = _load()
        e = np.empty((3, 27), dtype=np.int32)
        lib.or_moment_exponents(_ptr(e[0]), _ptr(e[1]), _ptr(e[2]))
        return e
