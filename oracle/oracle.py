"""ctypes wrapper of the C oracle (fdlbm_oracle.c).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays crossing this
interface are float64, C-contiguous, row-major [ny][nx] (fields) or
[16][ny][nx] (populations / moment sets), as in the GPU library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdlbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_ZERO_GRADIENT, BC_EQUILIBRIUM, BC_NEQ_WALL = 0, 1, 2, 3
LIM_MC, LIM_LW, LIM_UPWIND = 0, 1, 2

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, strict IEEE: no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.or_create.restype = ctypes.c_void_p
        lib.or_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, _D, ctypes.c_int, _I, _D]
        lib.or_destroy.argtypes = [ctypes.c_void_p]
        lib.or_init.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
        lib.or_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.or_get_state.argtypes = [ctypes.c_void_p, _D]
        lib.or_set_state.argtypes = [ctypes.c_void_p, _D]
        lib.or_moments.argtypes = [ctypes.c_void_p, _D, _D, _D, _D, _D]
        lib.or_moments_central.argtypes = [ctypes.c_void_p, _D]
        lib.or_totals.argtypes = [ctypes.c_void_p, _D]
        lib.or_matrices.argtypes = [_D, _D, _D, _D, _D]
        lib.or_matrices.restype = ctypes.c_int
        lib.or_central_matrix.argtypes = [ctypes.c_double, ctypes.c_double, _D]
        lib.or_feq_hat.argtypes = [ctypes.c_double] * 5 + [_D]
        lib.or_feq.argtypes = [ctypes.c_double] * 5 + [_D]
        lib.or_feq.restype = ctypes.c_int
        lib.or_psi.argtypes = [ctypes.c_double]
        lib.or_psi.restype = ctypes.c_double
        lib.or_collision.argtypes = [_D, _D, ctypes.c_double, _D, _D]
        lib.or_update_patch.argtypes = [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, _D, ctypes.c_int, _D]
        lib.or_update_patch.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def set_threads(n: int) -> None:
    load().or_set_threads(int(n))


def max_threads() -> int:
    return int(load().or_max_threads())


def matrices():
    """Return (M, Minv, vx, vy, eta) as built by the oracle."""
    M = np.zeros((16, 16)); Mi = np.zeros((16, 16))
    vx = np.zeros(16); vy = np.zeros(16); eta = np.zeros(16)
    if load().or_matrices(_p(M), _p(Mi), _p(vx), _p(vy), _p(eta)) != 0:
        raise RuntimeError("oracle: M is singular")
    return M, Mi, vx, vy, eta


def central_matrix(ux: float, uy: float) -> np.ndarray:
    Ms = np.zeros((16, 16))
    load().or_central_matrix(float(ux), float(uy), _p(Ms))
    return Ms


def feq_hat(rho, ux, uy, T, b) -> np.ndarray:
    out = np.zeros(16)
    load().or_feq_hat(float(rho), float(ux), float(uy), float(T), float(b), _p(out))
    return out


def feq(rho, ux, uy, T, b) -> np.ndarray:
    out = np.zeros(16)
    if load().or_feq(float(rho), float(ux), float(uy), float(T), float(b), _p(out)) != 0:
        raise RuntimeError("oracle: M is singular")
    return out


def collision(f, s, gamma, grad=(0.0, 0.0, 0.0, 0.0)) -> np.ndarray:
    """C = M^-1 S_hat (f_hat - f_hat^eq) of one cell (with the energy-flux correction)."""
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    g = np.ascontiguousarray(np.asarray(grad, dtype=np.float64))
    out = np.zeros(16)
    load().or_collision(_p(f), _p(s), float(gamma), _p(g), _p(out))
    return out


def update_patch(patch, dx, dt, gamma, s, limiter=LIM_MC, dy=None) -> np.ndarray:
    """Time-(n+1) populations of the centre of a [16][5][5] neighbourhood at time n."""
    patch = np.ascontiguousarray(np.asarray(patch, dtype=np.float64))
    assert patch.shape == (16, 5, 5)
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    out = np.zeros(16)
    rc = load().or_update_patch(_p(patch), float(dx), float(dx if dy is None else dy), float(dt),
                                float(gamma), _p(s), int(limiter), _p(out))
    if rc != 0:
        raise ValueError("oracle: invalid parameters")
    return out


def psi(theta: float) -> float:
    return float(load().or_psi(float(theta)))


class Oracle:
    """One FDLBM problem on the host.

    bc: sequence of 4 (kind, rho, ux, uy, T) tuples for x-low, x-high, y-low, y-high.
    s:  16 relaxation rates (s_1..s_16; s_1..s_4 unused).
    """

    def __init__(self, nx, ny, dx, dt, gamma, s, limiter=LIM_MC, bc=None, dy=None):
        lib = load()
        self.nx, self.ny = int(nx), int(ny)
        self.dx = float(dx); self.dy = float(dx if dy is None else dy); self.dt = float(dt)
        self.gamma = float(gamma); self.b = 2.0 / (self.gamma - 1.0)
        s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
        assert s.shape == (16,)
        if bc is None:
            bc = [(BC_PERIODIC, 0, 0, 0, 0)] * 4
        kinds = (ctypes.c_int * 4)(*[int(e[0]) for e in bc])
        states = np.ascontiguousarray(np.array([e[1:5] for e in bc], dtype=np.float64).reshape(16))
        self._h = lib.or_create(self.nx, self.ny, self.dx, self.dy, self.dt, self.gamma, _p(s),
                                int(limiter), kinds, _p(states))
        if not self._h:
            raise ValueError("oracle: invalid parameters")
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.or_destroy(self._h)
            self._h = None

    __del__ = close

    def _field(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if a.shape != (self.ny, self.nx):
            a = np.ascontiguousarray(np.broadcast_to(a, (self.ny, self.nx)))
        return a

    def init(self, rho, ux, uy, T):
        r, x, y, t = (self._field(a) for a in (rho, ux, uy, T))
        self._lib.or_init(self._h, _p(r), _p(x), _p(y), _p(t))

    def step(self, n: int = 1):
        self._lib.or_step(self._h, int(n))

    def get_state(self) -> np.ndarray:
        out = np.zeros((16, self.ny, self.nx))
        self._lib.or_get_state(self._h, _p(out))
        return out

    def set_state(self, f: np.ndarray):
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
        assert f.shape == (16, self.ny, self.nx)
        self._lib.or_set_state(self._h, _p(f))

    def moments(self, delta: bool = False):
        shape = (self.ny, self.nx)
        rho, ux, uy, T = (np.zeros(shape) for _ in range(4))
        d = np.zeros((16,) + shape) if delta else None
        self._lib.or_moments(self._h, _p(rho), _p(ux), _p(uy), _p(T), _p(d))
        return (rho, ux, uy, T, d) if delta else (rho, ux, uy, T)

    def moments_central(self) -> np.ndarray:
        out = np.zeros((16, self.ny, self.nx))
        self._lib.or_moments_central(self._h, _p(out))
        return out

    def totals(self) -> np.ndarray:
        out = np.zeros(4)
        self._lib.or_totals(self._h, _p(out))
        return out
