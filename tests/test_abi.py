"""The C-ABI library builds, loads and exports every symbol include/vlasov.h declares.

No CUDA device is needed: only host-side entry points (workspace sizing and
argument checks) are called.
"""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)
from paper_2007_12227_gb300 import build as B
from paper_2007_12227_gb300 import inputs as I
from paper_2007_12227_gb300 import vlasov as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vlasov.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return V.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vp_[a-z_]+)\s*\(", text)))


def test_every_declared_function_is_exported_and_bound(lib):
    names = declared_functions()
    assert len(names) >= 14
    bound = {n for n, _, _ in V._SIGNATURES}
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
        assert n in bound, f"{n} has no binding"
    out = subprocess.run(["nm", "-D", "--defined-only", V.LIB_PATH], capture_output=True, text=True)
    if out.returncode == 0:
        exported = set(re.findall(r"\bT (vp_[a-z_]+)\b", out.stdout))
        assert set(names) <= exported


def test_struct_layouts_match_the_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "vlasov.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", '
                   'sizeof(vp_grid), sizeof(vp_pusher), sizeof(vp_opts), sizeof(vp_moments_t), '
                   'offsetof(vp_moments_t, step), sizeof(vp_server_opts), sizeof(vp_request), '
                   'sizeof(vp_result), offsetof(vp_request, f0), sizeof(vp_plan_info), '
                   'sizeof(vp_tune_config), sizeof(vp_tune_opts), sizeof(vp_tune_result), '
                   'offsetof(vp_tune_config, pusher)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [C.sizeof(V.vp_grid), C.sizeof(V.vp_pusher), C.sizeof(V.vp_opts),
            C.sizeof(V.vp_moments_t), V.vp_moments_t.step.offset, C.sizeof(V.vp_server_opts),
            C.sizeof(V.vp_request), C.sizeof(V.vp_result), V.vp_request.f0.offset,
            C.sizeof(V.vp_plan_info), C.sizeof(V.vp_tune_config), C.sizeof(V.vp_tune_opts),
            C.sizeof(V.vp_tune_result), V.vp_tune_config.pusher.offset]
    assert got == want


def _cfg(nx=128, np_=96, basis=V.VP_BASIS_CUBIC_BSPLINE, precision=V.VP_FP32, kind=0, pot=1):
    g = V.vp_grid(nx, np_, -3.141592653589793, 3.141592653589793, -3.0, 3.0)
    pu = V.vp_pusher(kind, pot, 1.0, 1.0, 0.05, 0.0, 0.0)
    o = V.vp_opts(precision, 0, 0, 0, 0, 0, None)
    return g, basis, pu, o


def test_workspace_size_scales_with_grid_and_precision(lib):
    g, b, pu, o = _cfg()
    N = 128 * 96
    n32 = V.vp_workspace_size(g, b, pu, o)
    # the one-pass plan: two state buffers (its weights are read out through the idle one) and
    # tables that do not grow with the mesh (the field history alone is 64 KiB here)
    assert n32 >= 2 * N * 4
    o64 = V.vp_opts(V.VP_FP64, 0, 0, 0, 0, 0, None)
    n64 = V.vp_workspace_size(g, b, pu, o64)
    assert n64 > n32
    # a step that needs a third mesh-sized buffer: the separate-filter path (the x solve's
    # output) and the separate-x-pass plan (the deposit between its two launches)
    tiled = V.vp_workspace_size(g, b, pu, V.vp_opts(V.VP_FP32, 0, V.VP_KERNEL_TILED, 0, 0, 0, None))
    xpass = V.vp_workspace_size(g, b, pu, V.vp_opts(V.VP_FP32, 0, V.VP_KERNEL_FUSED_XPASS, 64, 0, 0, None))
    assert tiled >= 3 * N * 4 and xpass - n32 >= N * 4
    tent = V.vp_workspace_size(g, V.VP_BASIS_TENT, pu, o)
    assert tent <= n32


@pytest.mark.parametrize("bad", ["small_grid", "bad_basis", "bad_kind", "bad_precision",
                                 "period", "tiles", "nan_dt", "huge_row"])
def test_invalid_arguments_are_rejected_on_the_host(lib, bad):
    g, b, pu, o = _cfg()
    if bad == "small_grid":
        g.nx = 3
    elif bad == "bad_basis":
        b = 7
    elif bad == "bad_kind":
        pu.kind = 9
    elif bad == "bad_precision":
        o.precision = 5
    elif bad == "period":
        g.x1 = 2.0                         # pendulum needs a 2 pi multiple period
    elif bad == "tiles":                   # the tiled kernel cannot hold a 4096^2 tile
        o.kernel = V.VP_KERNEL_TILED
        o.tile_x = 4096
        o.tile_p = 4096
        g.nx, g.np = 8192, 8192
    elif bad == "nan_dt":
        pu.dt = float("nan")
    elif bad == "huge_row":
        g.nx, g.np = 65536, 64             # cyclic row solve keeps a row in shared memory
    n = C.c_size_t()
    st = lib.vp_workspace_size(C.byref(g), b, C.byref(pu), C.byref(o), C.byref(n))
    assert st in (V.VP_ERR_ARG, V.VP_ERR_UNSUPPORTED)


def test_create_rejects_missing_workspace(lib):
    g, b, pu, o = _cfg()
    h = C.c_void_p()
    st = lib.vp_create(C.byref(g), b, C.byref(pu), C.byref(o), None, 0, C.byref(h))
    assert st == V.VP_ERR_WORKSPACE and not h.value


def test_planner_picks_the_fused_kernel_for_large_meshes(lib):
    g, b, pu, o = _cfg(nx=4096, np_=2048)
    o.kernel = V.VP_KERNEL_FUSED
    assert V.vp_workspace_size(g, b, pu, o) > 0
    g2, b2, pu2, o2 = _cfg(nx=520, np_=64)       # window (480 + halo + guard) wider than the mesh
    o2.kernel = V.VP_KERNEL_FUSED
    o2.tile_x = 480
    n = C.c_size_t()
    st = lib.vp_workspace_size(C.byref(g2), b2, C.byref(pu2), C.byref(o2), C.byref(n))
    assert st == V.VP_ERR_UNSUPPORTED


def test_status_strings(lib):
    for s in range(8):
        assert lib.vp_status_string(s)
    assert lib.vp_last_error(None) == b"NULL simulation"


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(V, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(V, "_lib", None)
    with pytest.raises(RuntimeError):
        V.lib()


def test_server_host_paths_without_a_gpu(lib):
    """Create, queue an invalid request, report its status, destroy: no device work."""
    buf = (C.c_char * 4096)()
    base = (C.addressof(buf) + 255) // 256 * 256
    o = V.vp_server_opts(1024, 0, 0, None)
    h = C.c_void_p()
    assert lib.vp_server_create(C.byref(o), C.c_void_p(base), 1024, C.byref(h)) == V.VP_OK
    f0 = (C.c_float * 24)()
    req = V.vp_request(11, V.vp_grid(3, 8, -3.14, 3.14, -1.0, 1.0), 1,
                       V.vp_pusher(0, 1, 1.0, 1.0, 0.1, 0.0, 0.0), 0, 0, 5, 0,
                       C.cast(f0, C.c_void_p), 0)
    assert lib.vp_server_submit(h, C.byref(req)) == V.VP_OK
    q, a = C.c_int32(), C.c_int32()
    assert lib.vp_server_run(h, 3, C.byref(q), C.byref(a)) == V.VP_OK
    assert q.value == 0 and a.value == 0
    res = (V.vp_result * 4)()
    n = C.c_int32()
    assert lib.vp_server_poll(h, res, 4, C.byref(n)) == V.VP_OK
    assert n.value == 1 and res[0].id == 11 and res[0].status == V.VP_ERR_ARG
    bad = V.vp_request(12, V.vp_grid(8, 8, 0, 1, 0, 1), 1, V.vp_pusher(), 0, 0, -1, 0, None, 0)
    assert lib.vp_server_submit(h, C.byref(bad)) == V.VP_ERR_ARG
    lib.vp_server_destroy(h)


def _tune_cfg(nx, np_):
    g, b, pu, o = _cfg(nx=nx, np_=np_)
    c = V.vp_tune_config()
    c.grid, c.basis, c.pusher = g, b, pu
    return c, o


def test_autotune_host_checks(lib):
    c, o = _tune_cfg(1024, 512)
    cfgs = (V.vp_tune_config * 2)(c, c)
    t = V.vp_tune_opts(0, 0, 0, 0, 0.0)
    n = C.c_size_t()
    assert lib.vp_autotune_workspace_size(cfgs, 1, C.byref(o), C.byref(t), C.byref(n)) == V.VP_OK
    # the tuning workspace holds the largest candidate plan and a density buffer
    assert n.value >= V.vp_workspace_size(c.grid, c.basis, c.pusher, o) + 4 * 1024 * 512
    # several configurations are tuned only together (batched)
    assert lib.vp_autotune_workspace_size(cfgs, 2, C.byref(o), C.byref(t), C.byref(n)) == V.VP_ERR_ARG
    tb = V.vp_tune_opts(0, 1, 0, 0, 0.0)
    assert lib.vp_autotune_workspace_size(cfgs, 2, C.byref(o), C.byref(tb), C.byref(n)) == V.VP_OK
    o64 = V.vp_opts(V.VP_FP64, 0, 0, 0, 0, 0, None)
    assert lib.vp_autotune_workspace_size(cfgs, 2, C.byref(o64), C.byref(tb),
                                          C.byref(n)) == V.VP_ERR_UNSUPPORTED
    out = (V.vp_tune_result * 1)()
    # no workspace: refused before any device work
    assert lib.vp_autotune(cfgs, 1, C.byref(o), C.byref(t), None, 0, out) == V.VP_ERR_WORKSPACE
    assert lib.vp_autotune(cfgs, 0, C.byref(o), C.byref(t), None, 0, out) == V.VP_ERR_ARG
    lib.vp_autotune_clear_cache()
