"""ctypes binding of libvlasov.so (include/vlasov.h), argument marshalling only.

Every function keeps the C name. Device memory and streams come from PyTorch:
``Sim`` asks the library for its workspace size, allocates that many bytes as
a CUDA tensor and passes the raw pointer. All compute runs in the CUDA
library; if the library is missing this module raises on load.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvlasov.so")

VP_OK, VP_ERR_ARG, VP_ERR_CUDA, VP_ERR_WORKSPACE, VP_ERR_NONFINITE, VP_ERR_TIMEOUT, \
    VP_ERR_STATE, VP_ERR_UNSUPPORTED = range(8)
VP_BASIS_TENT, VP_BASIS_CUBIC_BSPLINE = 0, 1
VP_PUSH_LEAPFROG_KDK, VP_PUSH_EXACT_ROTATION, VP_PUSH_FEL_DKD = 0, 1, 2
VP_POT_FREE, VP_POT_PENDULUM, VP_POT_HARMONIC = 0, 1, 2
VP_FP32, VP_FP64 = 0, 1
VP_PROJ_GALERKIN, VP_PROJ_LUMPED = 0, 1
VP_KERNEL_AUTO, VP_KERNEL_TILED, VP_KERNEL_SCATTER, VP_KERNEL_FUSED = 0, 1, 2, 3


class vp_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("np", C.c_int32), ("x0", C.c_double), ("x1", C.c_double),
                ("p0", C.c_double), ("p1", C.c_double)]


class vp_pusher(C.Structure):
    _fields_ = [("kind", C.c_int32), ("potential", C.c_int32), ("v_sign", C.c_double),
                ("omega", C.c_double), ("dt", C.c_double), ("a0_re", C.c_double),
                ("a0_im", C.c_double)]


class vp_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("projection", C.c_int32), ("kernel", C.c_int32),
                ("tile_x", C.c_int32), ("tile_p", C.c_int32), ("history_cap", C.c_int32),
                ("stream", C.c_void_p)]


class vp_moments_t(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "sum_w", "mass", "mean_x", "mean_p", "var_x", "var_p", "cov_xp", "energy", "trapped",
        "entropy", "neg_mass", "b_re", "b_im", "max_abs_w", "lost_mass", "a_re", "a_im", "tau")] + \
        [("step", C.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None

# (name, restype, argtypes) for every function of include/vlasov.h
_SIGNATURES = [
    ("vp_workspace_size", C.c_int, [C.POINTER(vp_grid), C.c_int32, C.POINTER(vp_pusher),
                                    C.POINTER(vp_opts), C.POINTER(C.c_size_t)]),
    ("vp_create", C.c_int, [C.POINTER(vp_grid), C.c_int32, C.POINTER(vp_pusher), C.POINTER(vp_opts),
                            C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]),
    ("vp_set_f", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_set_f_device", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_step", C.c_int, [C.c_void_p, C.c_int32]),
    ("vp_step_profiled", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.c_int32]),
    ("vp_get_f", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_get_f_device", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_moments", C.c_int, [C.c_void_p, C.POINTER(vp_moments_t)]),
    ("vp_field_history", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_size_t,
                                   C.POINTER(C.c_size_t)]),
    ("vp_sync", C.c_int, [C.c_void_p]),
    ("vp_set_stream", C.c_int, [C.c_void_p, C.c_void_p]),
    ("vp_state_device", C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    ("vp_destroy", None, [C.c_void_p]),
    ("vp_last_error", C.c_char_p, [C.c_void_p]),
    ("vp_status_string", C.c_char_p, [C.c_int]),
]


def lib():
    """Load libvlasov.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class VlasovError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{lib().vp_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _check(status, sim=None):
    if status != VP_OK:
        msg = lib().vp_last_error(sim).decode() if sim else ""
        raise VlasovError(status, msg)


def make_grid(g) -> vp_grid:
    return vp_grid(int(g.nx), int(g.np), float(g.x0), float(g.x1), float(g.p0), float(g.p1))


def make_pusher(p) -> vp_pusher:
    return vp_pusher(int(p.kind), int(p.potential), float(p.v_sign), float(p.omega), float(p.dt),
                     float(p.a0_re), float(p.a0_im))


def vp_workspace_size(grid, basis, pusher, opts) -> int:
    n = C.c_size_t()
    _check(lib().vp_workspace_size(C.byref(grid), int(basis), C.byref(pusher), C.byref(opts),
                                   C.byref(n)))
    return n.value


class Sim:
    """One simulation: workspace tensor from torch, all calls through the C ABI."""

    def __init__(self, grid, basis, pusher, precision=VP_FP32, projection=VP_PROJ_GALERKIN,
                 kernel=VP_KERNEL_AUTO, tile_x=0, tile_p=0, history_cap=0, device="cuda",
                 stream=None):
        import torch
        self.grid_c = make_grid(grid)
        self.pusher_c = make_pusher(pusher)
        self.nx, self.np = int(grid.nx), int(grid.np)
        self.precision = precision
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.opts = vp_opts(precision, projection, kernel, tile_x, tile_p, history_cap,
                            C.c_void_p(stream.cuda_stream))
        self.bytes = vp_workspace_size(self.grid_c, basis, self.pusher_c, self.opts)
        self.workspace = torch.empty(self.bytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        h = C.c_void_p()
        _check(lib().vp_create(C.byref(self.grid_c), int(basis), C.byref(self.pusher_c),
                               C.byref(self.opts), C.c_void_p(aligned), self.bytes, C.byref(h)))
        self.h = h

    @property
    def n(self):
        return self.nx * self.np

    def set_f(self, f):
        """f: numpy array [np][nx] (float32/float64) or a CUDA torch tensor."""
        if isinstance(f, np.ndarray):
            a = np.ascontiguousarray(f.reshape(self.np, self.nx))
            dt = VP_FP64 if a.dtype == np.float64 else VP_FP32
            if a.dtype not in (np.float32, np.float64):
                a = a.astype(np.float64)
                dt = VP_FP64
            _check(lib().vp_set_f(self.h, a.ctypes.data_as(C.c_void_p), dt, a.size), self.h)
        else:
            t = f.contiguous()
            import torch
            dt = VP_FP64 if t.dtype == torch.float64 else VP_FP32
            _check(lib().vp_set_f_device(self.h, C.c_void_p(t.data_ptr()), dt, t.numel()), self.h)
            self._keep = t

    def set_f_host_ptr(self, ptr: int, dtype: int):
        _check(lib().vp_set_f(self.h, C.c_void_p(ptr), dtype, self.n), self.h)

    def step(self, n=1):
        _check(lib().vp_step(self.h, int(n)), self.h)

    def step_profiled(self, n=1):
        """Advance n steps; returns summed device ms per phase (deposit, x solve, p solve, field)."""
        ms = (C.c_double * 4)()
        _check(lib().vp_step_profiled(self.h, int(n), ms, 4), self.h)
        return list(ms)

    def get_f(self, dtype=np.float64):
        out = np.empty((self.np, self.nx), dtype=dtype)
        dt = VP_FP64 if out.dtype == np.float64 else VP_FP32
        _check(lib().vp_get_f(self.h, out.ctypes.data_as(C.c_void_p), dt, out.size), self.h)
        return out

    def get_f_host_ptr(self, ptr: int, dtype: int):
        _check(lib().vp_get_f(self.h, C.c_void_p(ptr), dtype, self.n), self.h)

    def get_f_device(self, out):
        import torch
        dt = VP_FP64 if out.dtype == torch.float64 else VP_FP32
        _check(lib().vp_get_f_device(self.h, C.c_void_p(out.data_ptr()), dt, out.numel()), self.h)
        return out

    def moments(self) -> dict:
        m = vp_moments_t()
        _check(lib().vp_moments(self.h, C.byref(m)), self.h)
        return m.as_dict()

    def field_history(self, max_entries=1 << 20):
        buf = np.zeros(2 * max_entries, dtype=np.float64)
        cnt = C.c_size_t()
        _check(lib().vp_field_history(self.h, buf.ctypes.data_as(C.POINTER(C.c_double)),
                                      max_entries, C.byref(cnt)), self.h)
        return buf[: 2 * cnt.value].reshape(-1, 2)

    def sync(self):
        _check(lib().vp_sync(self.h), self.h)

    def state_ptr(self) -> int:
        p = C.c_void_p()
        _check(lib().vp_state_device(self.h, C.byref(p)), self.h)
        return p.value

    def close(self):
        if getattr(self, "h", None):
            lib().vp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
