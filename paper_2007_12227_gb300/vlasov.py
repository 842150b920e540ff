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
    VP_ERR_STATE, VP_ERR_UNSUPPORTED, VP_ERR_CANCELLED = range(9)
VP_BASIS_TENT, VP_BASIS_CUBIC_BSPLINE, VP_BASIS_SEPTIC_BSPLINE = 0, 1, 2
VP_PUSH_LEAPFROG_KDK, VP_PUSH_EXACT_ROTATION, VP_PUSH_FEL_DKD, VP_PUSH_FEL_RK4 = 0, 1, 2, 3
VP_POT_FREE, VP_POT_PENDULUM, VP_POT_HARMONIC = 0, 1, 2
VP_FP32, VP_FP64 = 0, 1
VP_PROJ_GALERKIN, VP_PROJ_LUMPED = 0, 1
VP_KERNEL_AUTO, VP_KERNEL_TILED, VP_KERNEL_SCATTER, VP_KERNEL_FUSED, VP_KERNEL_FUSED_XPASS = 0, 1, 2, 3, 4


class vp_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("np", C.c_int32), ("x0", C.c_double), ("x1", C.c_double),
                ("p0", C.c_double), ("p1", C.c_double)]


class vp_pusher(C.Structure):
    _fields_ = [("kind", C.c_int32), ("potential", C.c_int32), ("v_sign", C.c_double),
                ("omega", C.c_double), ("dt", C.c_double), ("a0_re", C.c_double),
                ("a0_im", C.c_double), ("delta", C.c_double), ("sigma2", C.c_double)]


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


class vp_server_opts(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("slice_steps", C.c_int32), ("max_active", C.c_int32),
                ("stream", C.c_void_p)]


class vp_request(C.Structure):
    _fields_ = [("id", C.c_uint64), ("grid", vp_grid), ("basis", C.c_int32), ("pusher", vp_pusher),
                ("precision", C.c_int32), ("projection", C.c_int32), ("steps", C.c_int32),
                ("keep_f", C.c_int32), ("f0", C.c_void_p), ("f0_dtype", C.c_int32)]


class vp_result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int32), ("batched", C.c_int32),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_finish", C.c_double),
                ("moments", vp_moments_t)]


class vp_plan_info(C.Structure):
    _fields_ = [(n, C.c_int32) for n in (
        "kernel", "tile_x", "tile_p", "ntiles_x", "ntiles_p", "threads", "full_row", "state_is_s",
        "launches_per_step", "pad")] + [("workspace_bytes", C.c_int64), ("smem_bytes", C.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "pad"}


class vp_tune_config(C.Structure):
    _fields_ = [("grid", vp_grid), ("basis", C.c_int32), ("pad", C.c_int32), ("pusher", vp_pusher)]


class vp_tune_opts(C.Structure):
    _fields_ = [("min_steps", C.c_int32), ("batched", C.c_int32), ("use_cache", C.c_int32),
                ("pad", C.c_int32), ("min_ms", C.c_double)]


class vp_tune_result(C.Structure):
    _fields_ = [("tile_x", C.c_int32), ("tile_p", C.c_int32), ("kernel", C.c_int32),
                ("candidates", C.c_int32), ("from_cache", C.c_int32), ("pad", C.c_int32),
                ("ms_per_step", C.c_double), ("default_ms_per_step", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "pad"}


_lib = None

# (name, restype, argtypes) for every function of include/vlasov.h
_SIGNATURES = [
    ("vp_workspace_size", C.c_int, [C.POINTER(vp_grid), C.c_int32, C.POINTER(vp_pusher),
                                    C.POINTER(vp_opts), C.POINTER(C.c_size_t)]),
    ("vp_create", C.c_int, [C.POINTER(vp_grid), C.c_int32, C.POINTER(vp_pusher), C.POINTER(vp_opts),
                            C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]),
    ("vp_set_f", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_set_f_device", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_set_f_async", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_step", C.c_int, [C.c_void_p, C.c_int32]),
    ("vp_step_profiled", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.c_int32]),
    ("vp_get_f", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_get_f_device", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_get_f_async", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_moments", C.c_int, [C.c_void_p, C.POINTER(vp_moments_t)]),
    ("vp_field_history", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_size_t,
                                   C.POINTER(C.c_size_t)]),
    ("vp_sync", C.c_int, [C.c_void_p]),
    ("vp_set_stream", C.c_int, [C.c_void_p, C.c_void_p]),
    ("vp_state_device", C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    ("vp_batch_workspace_size", C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_size_t)]),
    ("vp_batch_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.c_void_p,
                                  C.c_size_t, C.POINTER(C.c_void_p)]),
    ("vp_batch_step", C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    ("vp_batch_step_each", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_int32]),
    ("vp_batch_sync", C.c_int, [C.c_void_p]),
    ("vp_batch_destroy", None, [C.c_void_p]),
    ("vp_batch_last_error", C.c_char_p, [C.c_void_p]),
    ("vp_server_create", C.c_int, [C.POINTER(vp_server_opts), C.c_void_p, C.c_size_t,
                                   C.POINTER(C.c_void_p)]),
    ("vp_server_submit", C.c_int, [C.c_void_p, C.POINTER(vp_request)]),
    ("vp_server_run", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("vp_server_poll", C.c_int, [C.c_void_p, C.POINTER(vp_result), C.c_int32, C.POINTER(C.c_int32)]),
    ("vp_server_cancel", C.c_int, [C.c_void_p, C.c_uint64]),
    ("vp_server_take_f", C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int32, C.c_size_t]),
    ("vp_server_clock", C.c_double, []),
    ("vp_server_destroy", None, [C.c_void_p]),
    ("vp_server_last_error", C.c_char_p, [C.c_void_p]),
    ("vp_moments_static", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(vp_grid), C.POINTER(vp_pusher),
                                    C.c_double, C.POINTER(C.c_double), C.POINTER(vp_moments_t),
                                    C.c_void_p]),
    ("vp_plan", C.c_int, [C.c_void_p, C.POINTER(vp_plan_info)]),
    ("vp_autotune_workspace_size", C.c_int, [C.POINTER(vp_tune_config), C.c_int32, C.POINTER(vp_opts),
                                             C.POINTER(vp_tune_opts), C.POINTER(C.c_size_t)]),
    ("vp_autotune", C.c_int, [C.POINTER(vp_tune_config), C.c_int32, C.POINTER(vp_opts),
                              C.POINTER(vp_tune_opts), C.c_void_p, C.c_size_t,
                              C.POINTER(vp_tune_result)]),
    ("vp_autotune_clear_cache", None, []),
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
                     float(p.a0_re), float(p.a0_im), float(getattr(p, "delta", 0.0)),
                     float(getattr(p, "sigma2", 0.0)))


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
            # the library reads t on the sim's stream: whatever wrote it on torch's stream finishes first
            torch.cuda.current_stream(t.device).synchronize()
            _check(lib().vp_set_f_device(self.h, C.c_void_p(t.data_ptr()), dt, t.numel()), self.h)
            self._keep = t

    def set_f_host_ptr(self, ptr: int, dtype: int):
        _check(lib().vp_set_f(self.h, C.c_void_p(ptr), dtype, self.n), self.h)

    def set_f_async_ptr(self, ptr: int, dtype: int):
        """vp_set_f_async: returns at once; keep the host buffer unchanged until sync()."""
        _check(lib().vp_set_f_async(self.h, C.c_void_p(ptr), dtype, self.n), self.h)

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

    def get_f_async_ptr(self, ptr: int, dtype: int):
        """vp_get_f_async: returns at once; the host buffer holds the weights after sync()."""
        _check(lib().vp_get_f_async(self.h, C.c_void_p(ptr), dtype, self.n), self.h)

    def get_f_device(self, out):
        import torch
        dt = VP_FP64 if out.dtype == torch.float64 else VP_FP32
        _check(lib().vp_get_f_device(self.h, C.c_void_p(out.data_ptr()), dt, out.numel()), self.h)
        return out

    def plan(self) -> dict:
        """What the planner chose (kernel, tile shape, threads, launches per step, bytes)."""
        pi = vp_plan_info()
        _check(lib().vp_plan(self.h, C.byref(pi)), self.h)
        return pi.as_dict()

    def kernel(self) -> int:
        return self.plan()["kernel"]

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


class Batch:
    """Several Sim objects advanced together by the batched one-pass kernel."""

    def __init__(self, sims, stream=None, device="cuda"):
        import torch
        self.sims = list(sims)
        if stream is None:
            stream = self.sims[0].stream
        self.stream = stream
        arr = (C.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        self._arr = arr
        n = C.c_size_t()
        _check(lib().vp_batch_workspace_size(arr, len(self.sims), C.byref(n)))
        self.workspace = torch.empty(n.value + 256, dtype=torch.uint8, device=device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        h = C.c_void_p()
        st = lib().vp_batch_create(arr, len(self.sims), C.c_void_p(stream.cuda_stream),
                                   C.c_void_p(aligned), n.value, C.byref(h))
        if st != VP_OK:
            raise VlasovError(st, "vp_batch_create")
        self.h = h

    def step(self, n=1, use_graph=True):
        st = lib().vp_batch_step(self.h, int(n), 1 if use_graph else 0)
        if st != VP_OK:
            raise VlasovError(st, lib().vp_batch_last_error(self.h).decode())

    def step_each(self, n, max_steps, use_graph=True):
        """n steps; simulation k takes min(n, max_steps[k]) of them."""
        arr = (C.c_int32 * len(self.sims))(*[int(v) for v in max_steps])
        st = lib().vp_batch_step_each(self.h, int(n), arr, 1 if use_graph else 0)
        if st != VP_OK:
            raise VlasovError(st, lib().vp_batch_last_error(self.h).decode())

    def sync(self):
        st = lib().vp_batch_sync(self.h)
        if st != VP_OK:
            raise VlasovError(st, lib().vp_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().vp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over a torch-allocated device arena."""

    def __init__(self, arena_bytes, budget_bytes=0, slice_steps=0, max_active=0, stream=None,
                 device="cuda"):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.arena = torch.empty(arena_bytes + 256, dtype=torch.uint8, device=device)
        aligned = (self.arena.data_ptr() + 255) // 256 * 256
        self.opts = vp_server_opts(int(budget_bytes), int(slice_steps), int(max_active),
                                   C.c_void_p(stream.cuda_stream))
        h = C.c_void_p()
        st = lib().vp_server_create(C.byref(self.opts), C.c_void_p(aligned), int(arena_bytes), C.byref(h))
        if st != VP_OK:
            raise VlasovError(st, "vp_server_create")
        self.h = h
        self._hold = {}

    def _err(self, st):
        if st != VP_OK:
            raise VlasovError(st, lib().vp_server_last_error(self.h).decode())

    def submit(self, rid, grid, basis, pusher, f0, steps, precision=VP_FP32,
               projection=VP_PROJ_GALERKIN, keep_f=False):
        a = np.ascontiguousarray(f0.reshape(grid.np, grid.nx))
        dt = VP_FP64 if a.dtype == np.float64 else VP_FP32
        if a.dtype not in (np.float32, np.float64):
            a, dt = a.astype(np.float64), VP_FP64
        req = vp_request(int(rid), make_grid(grid), int(basis), make_pusher(pusher), int(precision),
                         int(projection), int(steps), 1 if keep_f else 0, a.ctypes.data, dt)
        self._err(lib().vp_server_submit(self.h, C.byref(req)))

    def run(self, rounds=1):
        q, a = C.c_int32(), C.c_int32()
        self._err(lib().vp_server_run(self.h, int(rounds), C.byref(q), C.byref(a)))
        return q.value, a.value

    def poll(self, max_results=4096):
        buf = (vp_result * max_results)()
        n = C.c_int32()
        self._err(lib().vp_server_poll(self.h, buf, max_results, C.byref(n)))
        out = []
        for k in range(n.value):
            r = buf[k]
            out.append(dict(id=r.id, status=r.status, batched=r.batched, t_submit=r.t_submit,
                            t_admit=r.t_admit, t_finish=r.t_finish, moments=r.moments.as_dict()))
        return out

    def cancel(self, rid):
        """Cancel a queued or running request; its result comes back with VP_ERR_CANCELLED."""
        self._err(lib().vp_server_cancel(self.h, int(rid)))

    def take_f(self, rid, shape, dtype=np.float64):
        out = np.empty(shape, dtype=dtype)
        dt = VP_FP64 if out.dtype == np.float64 else VP_FP32
        self._err(lib().vp_server_take_f(self.h, int(rid), out.ctypes.data_as(C.c_void_p), dt, out.size))
        return out

    @staticmethod
    def clock():
        return lib().vp_server_clock()

    def close(self):
        if getattr(self, "h", None):
            lib().vp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_configs(workloads):
    """vp_tune_config array for objects with .grid, .basis and .pusher."""
    arr = (vp_tune_config * len(workloads))()
    for k, w in enumerate(workloads):
        arr[k].grid = make_grid(w.grid)
        arr[k].basis = int(w.basis)
        arr[k].pusher = make_pusher(w.pusher)
    return arr


def autotune(workloads, precision=VP_FP32, projection=VP_PROJ_GALERKIN, kernel=VP_KERNEL_AUTO,
             batched=False, min_steps=0, min_ms=0.0, use_cache=True, stream=None, device="cuda"):
    """Tile shapes chosen by the library's autotuner (vp_autotune); one dict per workload.

    The tuning workspace is a temporary torch allocation, released on return."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    cfgs = tune_configs(list(workloads))
    n = len(cfgs)
    opts = vp_opts(precision, projection, kernel, 0, 0, 0, C.c_void_p(stream.cuda_stream))
    topts = vp_tune_opts(int(min_steps), 1 if batched else 0, 1 if use_cache else 0, 0, float(min_ms))
    nbytes = C.c_size_t()
    _check(lib().vp_autotune_workspace_size(cfgs, n, C.byref(opts), C.byref(topts), C.byref(nbytes)))
    ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=device)
    aligned = (ws.data_ptr() + 255) // 256 * 256
    out = (vp_tune_result * n)()
    _check(lib().vp_autotune(cfgs, n, C.byref(opts), C.byref(topts), C.c_void_p(aligned),
                             nbytes.value, out))
    del ws
    return [out[k].as_dict() for k in range(n)]


def autotune_clear_cache():
    lib().vp_autotune_clear_cache()
