"""Thin ctypes binding of liblbm.so (include/lbm.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels.  Device
memory comes from PyTorch's caching allocator (passed through the allocator
callbacks of lbm_create_ex) and work is enqueued on the current PyTorch CUDA
stream.  There is no CPU fallback: `load()` raises if the library was not built.

    lbm_create(...) / lbm_create_ex(...) -> handle     (raise LbmError on failure)
    lbm_init, lbm_step, lbm_moments, lbm_moments_central, lbm_totals,
    lbm_get_state, lbm_set_state, lbm_step_count, lbm_footprint, lbm_destroy

`Solver` wraps one context with numpy arrays in and out.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CFL, LBM_ERR_STABILITY = 0, -1, -2, -3
LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_NONFINITE, LBM_ERR_STATE, LBM_ERR_TIMEOUT = -4, -5, -6, -7, -8
LBM_LIMITER_MC, LBM_LIMITER_LW, LBM_LIMITER_UPWIND = 0, 1, 2
LBM_BC_PERIODIC, LBM_BC_ZERO_GRADIENT, LBM_BC_EQUILIBRIUM, LBM_BC_NEQ_WALL = 0, 1, 2, 3
LBM_FP64, LBM_FP32_DEV = 0, 1

EXPORTS = ["lbm_create", "lbm_create_ex", "lbm_init", "lbm_step", "lbm_moments", "lbm_moments_central",
           "lbm_totals", "lbm_get_state", "lbm_get_state_rows", "lbm_set_state", "lbm_step_count", "lbm_step_kernel",
           "lbm_footprint", "lbm_profile_begin", "lbm_profile_end", "lbm_peak_fp64", "lbm_totals_noalloc",
           "lbm_autotune", "lbm_batch_create", "lbm_batch_step", "lbm_batch_destroy", "lbm_wait_selftest",
           "lbm_last_error", "lbm_destroy"]


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


class EdgeBC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rho", ctypes.c_double), ("u", ctypes.c_double),
                ("v", ctypes.c_double), ("T", ctypes.c_double)]


class BC(ctypes.Structure):
    _fields_ = [("xlo", EdgeBC), ("xhi", EdgeBC), ("ylo", EdgeBC), ("yhi", EdgeBC)]


_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC), ("free", _FREE), ("user", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rho0", ctypes.c_double), ("T0", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("allocator", ctypes.POINTER(Allocator)),
                ("device", ctypes.c_int), ("step_kernel", ctypes.c_int), ("dy", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load liblbm.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"liblbm.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        lib.lbm_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, _D, ctypes.c_int, ctypes.POINTER(BC), ctypes.POINTER(vp)]
        lib.lbm_create_ex.argtypes = lib.lbm_create.argtypes[:-1] + [ctypes.POINTER(Options), ctypes.POINTER(vp)]
        lib.lbm_init.argtypes = [vp, _D, _D, _D, _D]
        lib.lbm_step.argtypes = [vp, ctypes.c_int]
        lib.lbm_moments.argtypes = [vp, _D, _D, _D, _D, _D]
        lib.lbm_moments_central.argtypes = [vp, _D]
        lib.lbm_totals.argtypes = [vp, _D]
        lib.lbm_get_state.argtypes = [vp, _D]
        lib.lbm_set_state.argtypes = [vp, _D]
        lib.lbm_get_state_rows.argtypes = [vp, ctypes.c_int, ctypes.c_int, _D]
        lib.lbm_profile_begin.argtypes = [vp, ctypes.c_int]
        lib.lbm_profile_end.argtypes = [vp, _D]
        lib.lbm_peak_fp64.argtypes = [ctypes.c_int, _D]
        lib.lbm_wait_selftest.argtypes = [ctypes.c_int, _D]
        lib.lbm_wait_selftest.restype = ctypes.c_int
        lib.lbm_totals_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_void_p, _D]
        lib.lbm_totals_noalloc.restype = ctypes.c_int
        lib.lbm_autotune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.lbm_autotune.restype = ctypes.c_int
        lib.lbm_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
        lib.lbm_batch_create.restype = ctypes.c_int
        lib.lbm_batch_step.argtypes = [vp, ctypes.c_int]
        lib.lbm_batch_step.restype = ctypes.c_int
        lib.lbm_batch_destroy.argtypes = [vp]
        lib.lbm_batch_destroy.restype = None
        lib.lbm_step_count.argtypes = [vp]
        lib.lbm_step_count.restype = ctypes.c_longlong
        lib.lbm_step_kernel.argtypes = [vp]
        lib.lbm_step_kernel.restype = ctypes.c_int
        lib.lbm_footprint.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.lbm_footprint.restype = ctypes.c_size_t
        lib.lbm_last_error.argtypes = [vp]
        lib.lbm_last_error.restype = ctypes.c_char_p
        lib.lbm_destroy.argtypes = [vp]
        lib.lbm_destroy.restype = None
        for name in ("lbm_create", "lbm_create_ex", "lbm_init", "lbm_step", "lbm_moments",
                     "lbm_moments_central", "lbm_totals", "lbm_get_state", "lbm_set_state",
                     "lbm_get_state_rows", "lbm_profile_begin", "lbm_profile_end", "lbm_peak_fp64"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _check(rc: int, handle=None):
    if rc != LBM_OK:
        msg = load().lbm_last_error(handle)
        raise LbmError(rc, msg.decode() if msg else "")
    return rc


def make_bc(edges) -> BC:
    """edges: 4 x (kind, rho, u, v, T) for x-lo, x-hi, y-lo, y-hi."""
    bc = BC()
    for name, e in zip(("xlo", "xhi", "ylo", "yhi"), edges):
        setattr(bc, name, EdgeBC(int(e[0]), float(e[1]), float(e[2]), float(e[3]), float(e[4])))
    return bc


# --------------------------------------------------------------------------- C-ABI names
def lbm_create(nx, ny, dx, dt, gamma, Pr, s, limiter, bc):
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    h = ctypes.c_void_p()
    b = bc if isinstance(bc, BC) else make_bc(bc)
    _check(load().lbm_create(int(nx), int(ny), float(dx), float(dt), float(gamma), float(Pr), _p(s),
                             int(limiter), ctypes.byref(b), ctypes.byref(h)))
    return h


def lbm_create_ex(nx, ny, dx, dt, gamma, Pr, s, limiter, bc, options: Options):
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    h = ctypes.c_void_p()
    b = bc if isinstance(bc, BC) else make_bc(bc)
    _check(load().lbm_create_ex(int(nx), int(ny), float(dx), float(dt), float(gamma), float(Pr), _p(s),
                                int(limiter), ctypes.byref(b), ctypes.byref(options), ctypes.byref(h)))
    return h


def lbm_init(h, rho, u, v, T):
    _check(load().lbm_init(h, _p(rho), _p(u), _p(v), _p(T)), h)


def lbm_step(h, n):
    _check(load().lbm_step(h, int(n)), h)


def lbm_moments(h, rho=None, u=None, v=None, T=None, delta=None):
    return load().lbm_moments(h, _p(rho), _p(u), _p(v), _p(T), _p(delta))


def lbm_moments_central(h, delta_star):
    _check(load().lbm_moments_central(h, _p(delta_star)), h)


def lbm_totals(h, out):
    _check(load().lbm_totals(h, _p(out)), h)


def lbm_get_state(h, f):
    _check(load().lbm_get_state(h, _p(f)), h)


def lbm_get_state_rows(h, row0, rows, f):
    _check(load().lbm_get_state_rows(h, int(row0), int(rows), _p(f)), h)


def lbm_set_state(h, f):
    _check(load().lbm_set_state(h, _p(f)), h)


def lbm_profile_begin(h, max_steps):
    _check(load().lbm_profile_begin(h, int(max_steps)), h)


def lbm_profile_end(h):
    out = np.zeros(4)
    _check(load().lbm_profile_end(h, _p(out)), h)
    return out


def lbm_peak_fp64(device=0) -> float:
    out = np.zeros(1)
    _check(load().lbm_peak_fp64(int(device), _p(out)))
    return float(out[0])


def lbm_wait_selftest(device=0):
    """Failure-path check of the kernels' bounded waits: (status, kernel ms); the expected
    status is LBM_ERR_TIMEOUT."""
    out = np.zeros(1)
    rc = load().lbm_wait_selftest(int(device), _p(out))
    return int(rc), float(out[0])


def lbm_totals_noalloc(f_device_ptr, nx, ny, dx, dy=None, stream=None):
    """Totals of a dense [16][ny][nx] float64 device field (times dx dy), without device allocation."""
    out = np.zeros(4)
    _check(load().lbm_totals_noalloc(ctypes.c_void_p(int(f_device_ptr)), int(nx), int(ny), float(dx),
                                     float(dx if dy is None else dy), ctypes.c_void_p(int(stream or 0)),
                                     _p(out)))
    return out


def lbm_autotune(h, reps=5) -> int:
    choice = ctypes.c_int(0)
    _check(load().lbm_autotune(h, int(reps), ctypes.byref(choice)), h)
    return choice.value


def lbm_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[ctypes.c_void_p(int(h.value if hasattr(h, "value") else h))
                                              for h in handles])
    out = ctypes.c_void_p()
    _check(load().lbm_batch_create(arr, len(handles), ctypes.byref(out)))
    return out


def lbm_batch_step(b, n):
    rc = load().lbm_batch_step(b, int(n))
    if rc != LBM_OK:
        raise LbmError(rc, "lbm_batch_step failed")


def lbm_batch_destroy(b):
    load().lbm_batch_destroy(b)


class Batch:
    """Several Solvers stepped together (one batched launch pair per precision/limiter group)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.b = lbm_batch_create([s.h for s in self.solvers])

    def step(self, n=1):
        lbm_batch_step(self.b, n)

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_step_count(h) -> int:
    return int(load().lbm_step_count(h))


def lbm_step_kernel(h) -> int:
    return int(load().lbm_step_kernel(h))


def lbm_footprint(nx, ny, precision=LBM_FP64) -> int:
    return int(load().lbm_footprint(int(nx), int(ny), int(precision)))


def lbm_destroy(h):
    load().lbm_destroy(h)


# --------------------------------------------------------------------------- convenience
class Solver:
    """One FDLBM problem resident on the GPU.

    Memory comes from torch's caching allocator and work runs on `stream`
    (default: torch's current stream of `device`)."""

    def __init__(self, nx, ny, dx, dt, gamma, Pr, s, limiter=LBM_LIMITER_MC, bc=None,
                 precision=LBM_FP64, rho0=1.0, T0=1.0, device=0, stream=None, use_torch_allocator=True,
                 step_kernel=0, dy=None):
        import torch
        self.nx, self.ny = int(nx), int(ny)
        self.precision = precision
        self.device = int(device)
        torch.cuda.init()
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self._stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._keep = []
        opts = Options(int(precision), float(rho0), float(T0), ctypes.c_void_p(handle), None, self.device,
                       int(step_kernel), float(dy) if dy is not None else 0.0)
        if use_torch_allocator:
            dev = self.device

            def _alloc(nbytes, st, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(st or 0))
                except Exception:
                    return None

            def _free(ptr, nbytes, st, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            a = Allocator(_ALLOC(_alloc), _FREE(_free), None)
            self._keep += [a]
            opts.allocator = ctypes.pointer(a)
        self._keep.append(opts)
        if bc is None:
            bc = [(LBM_BC_PERIODIC, 0, 0, 0, 0)] * 4
        with torch.cuda.device(self.device):
            self.h = lbm_create_ex(nx, ny, dx, dt, gamma, Pr, s, limiter, bc, opts)

    @classmethod
    def from_problem(cls, p, precision=LBM_FP64, **kw):
        kw.setdefault("dy", p.dy)
        return cls(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter, p.bc, precision=precision, **kw)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _field(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if a.shape != (self.ny, self.nx):
            a = np.ascontiguousarray(np.broadcast_to(a, (self.ny, self.nx)))
        return a

    def init(self, rho, u, v, T):
        lbm_init(self.h, *(self._field(a) for a in (rho, u, v, T)))

    def step(self, n=1):
        lbm_step(self.h, n)

    def moments(self, delta=False, check=True):
        shape = (self.ny, self.nx)
        rho, u, v, T = (np.empty(shape) for _ in range(4))
        d = np.empty((16,) + shape) if delta else None
        rc = lbm_moments(self.h, rho, u, v, T, d)
        if check:
            _check(rc, self.h)
        return (rho, u, v, T, d) if delta else (rho, u, v, T)

    def moments_central(self):
        out = np.empty((16, self.ny, self.nx))
        lbm_moments_central(self.h, out)
        return out

    def totals(self):
        out = np.empty(4)
        lbm_totals(self.h, out)
        return out

    def get_state(self):
        out = np.empty((16, self.ny, self.nx))
        lbm_get_state(self.h, out)
        return out

    def get_state_rows(self, row0, rows):
        out = np.empty((16, int(rows), self.nx))
        lbm_get_state_rows(self.h, row0, rows, out)
        return out

    def set_state(self, f):
        lbm_set_state(self.h, np.ascontiguousarray(np.asarray(f, dtype=np.float64)))

    def autotune(self, reps=5):
        return lbm_autotune(self.h, reps)

    @property
    def step_count(self):
        return lbm_step_count(self.h)

    @property
    def step_kernel(self):
        """lbm_options.step_kernel code of the fused-step kernel in use (1 .. 9)."""
        return lbm_step_kernel(self.h)
