"""Python handle on the FP64 CPU oracle (vp_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline use it. The library never imports it. It shares no code with the CUDA
path; it is built from its own C source with gcc.

Every function takes plain float64 numpy arrays laid out [np][nx] (x fastest),
the grid convention of Sec. IV (periodic coordinate, open momentum with both
end nodes on the grid).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KDK, ROTATION, FEL, FEL_RK4 = 0, 1, 2, 3
FREE, PENDULUM, HARMONIC = 0, 1, 2
TENT, CUBIC, SEPTIC = 0, 1, 2
GALERKIN, LUMPED = 0, 1

MOMENT_NAMES = ["sum_w", "mass", "mean_x", "mean_p", "var_x", "var_p", "cov_xp",
                "energy", "trapped", "entropy", "neg_mass", "b_re", "b_im", "max_abs_w"]


class OrGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("np", C.c_int), ("x0", C.c_double), ("x1", C.c_double),
                ("p0", C.c_double), ("p1", C.c_double)]


class OrPusher(C.Structure):
    _fields_ = [("kind", C.c_int), ("potential", C.c_int), ("v_sign", C.c_double),
                ("omega", C.c_double), ("dt", C.c_double), ("delta", C.c_double),
                ("sigma2", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (serial FP64, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-pthread",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            L.or_step.argtypes = [C.POINTER(OrGrid), C.c_int, C.c_int, C.POINTER(OrPusher),
                                  dp, dp, dp, dp]
            L.or_step.restype = C.c_int
            L.or_step_par.argtypes = [C.POINTER(OrGrid), C.c_int, C.c_int, C.POINTER(OrPusher),
                                      dp, dp, dp, dp, C.c_int]
            L.or_step_par.restype = C.c_int
            L.or_run.argtypes = [C.POINTER(OrGrid), C.c_int, C.c_int, C.POINTER(OrPusher),
                                 dp, dp, C.c_long, dp, dp]
            L.or_run.restype = C.c_int
            L.or_push_many.argtypes = [C.POINTER(OrPusher), C.c_double, C.c_double, C.c_long,
                                       dp, dp, dp, dp]
            L.or_push_many.restype = None
            L.or_mass_solve.argtypes = [C.POINTER(OrGrid), dp]
            L.or_mass_solve.restype = None
            L.or_moments.argtypes = [C.POINTER(OrGrid), C.POINTER(OrPusher), dp, dp, dp]
            L.or_moments.restype = None
            L.or_bunching.argtypes = [C.POINTER(OrGrid), dp, dp, dp]
            L.or_bunching.restype = None
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _grid(g) -> OrGrid:
    return OrGrid(int(g.nx), int(g.np), float(g.x0), float(g.x1), float(g.p0), float(g.p1))


def _pusher(pu) -> OrPusher:
    return OrPusher(int(pu.kind), int(pu.potential), float(pu.v_sign), float(pu.omega),
                    float(pu.dt), float(getattr(pu, "delta", 0.0)), float(getattr(pu, "sigma2", 0.0)))


def _arr(w, g) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(g.np, g.nx)).copy()
    return a


class State:
    """Oracle state: weights, FEL field [A_re, A_im, b_re, b_im], lost weight."""

    def __init__(self, grid, pusher, basis, projection, w0):
        self.grid, self.pusher = grid, pusher
        self.basis, self.projection = int(basis), int(projection)
        self.w = _arr(w0, grid)
        self.fel = np.zeros(4, dtype=np.float64)
        self.lost = np.zeros(1, dtype=np.float64)
        self.step_count = 0
        if pusher.kind in (FEL, FEL_RK4):
            self.fel[0], self.fel[1] = pusher.a0_re, pusher.a0_im
            br, bi = bunching(grid, self.w)
            self.fel[2], self.fel[3] = br, bi

    def run(self, nsteps: int, history: bool = False):
        g, pu = _grid(self.grid), _pusher(self.pusher)
        hist = np.zeros(2 * max(nsteps, 1), dtype=np.float64) if history else None
        rc = lib().or_run(C.byref(g), self.basis, self.projection, C.byref(pu),
                          _dp(self.fel), _dp(self.w), int(nsteps), _dp(self.lost),
                          _dp(hist) if hist is not None else None)
        if rc:
            raise RuntimeError(f"or_run failed with code {rc}")
        self.step_count += nsteps
        if history:
            return hist.reshape(-1, 2)[:nsteps]
        return None

    def moments(self) -> dict:
        return moments(self.grid, self.pusher, self.w, self.fel[:2])


def step(grid, basis, projection, pusher, w, fel=None):
    """One step; returns (w_out, fel_out, lost)."""
    g, pu = _grid(grid), _pusher(pusher)
    w_in = _arr(w, grid)
    w_out = np.empty_like(w_in)
    f = np.zeros(4) if fel is None else np.array(fel, dtype=np.float64).copy()
    lost = np.zeros(1)
    rc = lib().or_step(C.byref(g), int(basis), int(projection), C.byref(pu), _dp(f), _dp(w_in),
                       _dp(w_out), _dp(lost))
    if rc:
        raise RuntimeError(f"or_step failed with code {rc}")
    return w_out, f, float(lost[0])


def step_par(grid, basis, projection, pusher, w, fel=None, threads=None):
    """One step on `threads` host threads (default: all cores), bitwise equal to step()."""
    g, pu = _grid(grid), _pusher(pusher)
    w_in = _arr(w, grid)
    w_out = np.empty_like(w_in)
    f = np.zeros(4) if fel is None else np.array(fel, dtype=np.float64).copy()
    lost = np.zeros(1)
    nt = threads or os.cpu_count() or 1
    rc = lib().or_step_par(C.byref(g), int(basis), int(projection), C.byref(pu), _dp(f), _dp(w_in),
                           _dp(w_out), _dp(lost), int(nt))
    if rc:
        raise RuntimeError(f"or_step_par failed with code {rc}")
    return w_out, f, float(lost[0])


def push(pusher, x, p, a=(0.0, 0.0)):
    """Push arrays of points one step; returns (x', p')."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64).ravel())
    xo, po = np.empty_like(x), np.empty_like(p)
    pu = _pusher(pusher)
    lib().or_push_many(C.byref(pu), float(a[0]), float(a[1]), x.size, _dp(x), _dp(p), _dp(xo),
                       _dp(po))
    return xo, po


def mass_solve(grid, r):
    """Apply Lambda^{-1} (tent basis, Kronecker cyclic-x / open-p) to r."""
    g = _grid(grid)
    a = _arr(r, grid)
    lib().or_mass_solve(C.byref(g), _dp(a))
    return a


def bunching(grid, w):
    g = _grid(grid)
    a = _arr(w, grid)
    br, bi = C.c_double(), C.c_double()
    lib().or_bunching(C.byref(g), _dp(a), C.byref(br), C.byref(bi))
    return br.value, bi.value


def moments(grid, pusher, w, a=None) -> dict:
    g, pu = _grid(grid), _pusher(pusher)
    ww = _arr(w, grid)
    out = np.zeros(len(MOMENT_NAMES))
    aa = None if a is None else np.array(a[:2], dtype=np.float64)
    lib().or_moments(C.byref(g), C.byref(pu), _dp(ww), _dp(aa) if aa is not None else None,
                     _dp(out))
    return dict(zip(MOMENT_NAMES, out.tolist()))
