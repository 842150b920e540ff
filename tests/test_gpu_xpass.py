"""The one-pass tile with a separate x-solve row pass (VP_KERNEL_FUSED_XPASS) against the FP64
oracle: the same update as the in-tile x solve (Sec. III update equation, Lambda = Lambda_x (x)
Lambda_p), with Lambda_x^{-1} applied as an exact cyclic solve over whole rows.

Tolerances as in test_gpu_parity: FP64 <= 1e-12 relative L-infinity, FP32 <= 1e-5 relative L1.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402

FP64_TOL = 1e-12
FP32_TOL = 1e-5
PI = math.pi
XP = V.VP_KERNEL_FUSED_XPASS


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def pend(nx, np_, precision, dt=0.05, pr=(-3.0, 3.0), pc=1.0, s=0.3):
    return I.Workload("t", I.Grid(nx, np_, -PI, PI, *pr),
                      I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, dt), I.BASIS_CUBIC, precision, 0,
                      "gaussian", dict(xc=0.0, pc=pc, sx=s, sp=s))


def run(wl, steps, kernel=XP, tile=(0, 0), f0=None):
    f0 = I.make_f0(wl) if f0 is None else f0
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=wl.precision, kernel=kernel,
                tile_x=tile[0], tile_p=tile[1])
    plan = sim.plan()
    sim.set_f(f0 if wl.precision == I.FP64 else f0.astype(np.float32))
    sim.step(steps)
    got, mom = sim.get_f(), sim.moments()
    sim.close()
    return got, mom, plan


def oracle(wl, steps, f0=None):
    f0 = I.make_f0(wl) if f0 is None else f0
    st = O.State(wl.grid, wl.pusher, wl.basis, I.PROJ_GALERKIN,
                 f0 if wl.precision == I.FP64 else f0.astype(np.float32).astype(np.float64))
    st.run(steps)
    return st


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("shape,tile", [((200, 150), (64, 64)), ((301, 130), (96, 48)),
                                        ((600, 97), (0, 0)), ((1100, 96), (224, 63))])
def test_xpass_fp64_ragged_tiles(shape, tile):
    """Ragged last tiles in both directions; nx = 301 takes the row pass's scalar copies."""
    wl = pend(shape[0], shape[1], I.FP64, dt=0.07, pc=0.8, s=0.5)
    got, _, plan = run(wl, 12, tile=tile)
    assert plan["kernel"] == XP and plan["launches_per_step"] == 2
    st = oracle(wl, 12)
    e = rel_linf(got, st.w)
    assert e <= FP64_TOL, f"rel Linf {e:.3e}"


@pytest.mark.parametrize("tile", [(224, 64), (480, 32), (96, 128), (224, 63), (200, 48), (100, 64)])
def test_xpass_fp32_windowed_tiles(tile):
    """Widths 200 and 100 are not multiples of the row pass's 32-node chunks: chunks that cross a
    tile boundary record their per-tile maxima (the next step's window scale) piece by piece."""
    wl = pend(1100, 700, I.FP32, dt=0.02, pr=(-4.0, 4.0), pc=0.5, s=0.4)
    got, mom, _ = run(wl, 25, tile=tile)
    st = oracle(wl, 25)
    e = rel_l1(got, st.w)
    assert e <= FP32_TOL, f"rel L1 {e:.3e}"
    om = st.moments()
    assert abs(mom["mass"] - om["mass"]) <= 1e-6 * om["mass"]


@pytest.mark.parametrize("nx,precision", [(9000, I.FP32), (20000, I.FP32), (9000, I.FP64)])
def test_xpass_long_rows(nx, precision):
    """Rows longer than 256 chunks of 32 (FP32) or 512 of 16 (FP64): the row pass runs 288 to
    640 threads per row.

    FP64 on a mesh this fine is limited by the oracle itself: it pushes absolute coordinates,
    so each node's position carries up to (nx / 2) eps cells of rounding per step (1e-12 cells
    at nx = 9000), and the deposits move by that much. The bound is steps * nx * eps; the row
    pass itself is checked against the in-tile x solve on the same input (<= 1e-13)."""
    wl = pend(nx, 40, precision, dt=0.05, pr=(-3.0, 3.0), pc=0.3, s=0.6)
    steps = 3
    f0 = I.make_f0(wl)
    got, _, plan = run(wl, steps, f0=f0)
    assert plan["kernel"] == XP
    st = oracle(wl, steps, f0=f0)
    if precision == I.FP64:
        assert rel_linf(got, st.w) <= steps * nx * np.finfo(np.float64).eps
        ref, _, _ = run(wl, steps, kernel=V.VP_KERNEL_FUSED, f0=f0)
        assert rel_linf(got, ref) <= 1e-13
    else:
        assert rel_l1(got, st.w) <= FP32_TOL


def test_xpass_matches_in_tile_solve_fp64():
    """The separate row pass and the in-tile solve (truncated at |z|^28) give the same update."""
    wl = pend(600, 400, I.FP64, dt=0.03, pr=(-4.0, 4.0), pc=0.5, s=0.4)
    f0 = I.make_f0(wl)
    a, _, _ = run(wl, 10, kernel=V.VP_KERNEL_FUSED, f0=f0)
    b, _, _ = run(wl, 10, kernel=XP, f0=f0)
    assert rel_linf(b, a) <= 1e-13


def test_xpass_8192_fp32_full_size():
    """The 8192^2 pendulum, one step with the separate x pass at the benchmark's tile."""
    wl = I.pendulum_8192_fp32_cubic()
    got, _, plan = run(wl, 1, tile=(224, 63))
    assert plan["threads"] == 256
    st = oracle(wl, 1)
    e = rel_l1(got, st.w)
    assert e <= FP32_TOL, f"rel L1 {e:.3e}"


def test_xpass_is_deterministic():
    wl = pend(1100, 300, I.FP32, dt=0.02, pr=(-4.0, 4.0), pc=0.5, s=0.4)
    f0 = I.make_f0(wl)
    a, _, _ = run(wl, 20, f0=f0)
    b, _, _ = run(wl, 20, f0=f0)
    assert np.array_equal(a, b)


def fel(nth, np_, precision, dt=0.05, a0=0.05, sp=0.1, pr=(-1.0, 1.0), sigma2=0.0, kind=None):
    return I.Workload("t", I.Grid(nth, np_, 0.0, 2 * PI, *pr),
                      I.Pusher(kind if kind is not None else I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, dt, a0, 0.0,
                               0.0, sigma2),
                      I.BASIS_CUBIC, precision, 0, "fel_gaussian", dict(sp=sp, eps=1e-4))


def run_fel(wl, steps, kernel=XP, tile=(0, 0)):
    f0 = I.make_f0(wl)
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=wl.precision, kernel=kernel,
                tile_x=tile[0], tile_p=tile[1])
    plan = sim.plan()
    sim.set_f(f0 if wl.precision == I.FP64 else f0.astype(np.float32))
    sim.step(steps)
    got, hist = sim.get_f(), sim.field_history()
    sim.close()
    st = O.State(wl.grid, wl.pusher, wl.basis, I.PROJ_GALERKIN,
                 f0 if wl.precision == I.FP64 else f0.astype(np.float32).astype(np.float64))
    ohist = st.run(steps, history=True)
    return got, hist, st, ohist, plan


# Against the oracle these FP64 FEL meshes (640 and 700 theta points) run 8 steps: the oracle
# pushes absolute phases, whose rounding (up to (nx / 2) eps cells per node and step) reaches the
# 1e-12 bound over longer runs on meshes this fine (as for the one-pass kernel in
# test_gpu_fel_full). The longer run compares the two GPU plans with each other.
@pytest.mark.parametrize("shape,tile", [((640, 96), (0, 0)), ((700, 130), (96, 48))])
def test_xpass_fel_fp64_field_history(shape, tile):
    """FEL with the separate x pass: the tile's bunching sums come from the deposit r, divided by
    the eigenvalue of Lambda_x at exp(-i theta); f and the field history must match the oracle's
    (which sums the weights themselves) to the FP64 bound."""
    wl = fel(shape[0], shape[1], I.FP64)
    got, hist, st, ohist, plan = run_fel(wl, 8, tile=tile)
    assert plan["kernel"] == XP
    assert rel_linf(got, st.w) <= FP64_TOL
    amp = np.max(np.hypot(ohist[:, 0], ohist[:, 1]))
    assert np.max(np.abs(hist - ohist)) <= FP64_TOL * amp


@pytest.mark.parametrize("sigma2", [0.0, 0.3])
def test_xpass_fel_fp64_matches_one_pass_over_30_steps(sigma2):
    """30 steps: the separate-x-pass plan and the one-pass kernel give the same f and field (the
    in-tile solve truncates at |z|^28; the bunching identity holds to rounding). sigma2 != 0: the
    space-charge kick reads the stored state the row pass wrote."""
    wl = fel(640, 96, I.FP64, sigma2=sigma2)
    f0 = I.make_f0(wl)
    out = []
    for kernel in (V.VP_KERNEL_FUSED, XP):
        sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=I.FP64, kernel=kernel)
        sim.set_f(f0)
        sim.step(30)
        out.append((sim.get_f(), sim.field_history()))
        sim.close()
    (fa, ha), (fb, hb) = out
    assert rel_linf(fb, fa) <= 1e-13
    assert np.max(np.abs(hb - ha)) <= 1e-13 * np.max(np.hypot(ha[:, 0], ha[:, 1]))


def test_xpass_fel_fp64_space_charge():
    """sigma^2 != 0 against the oracle."""
    wl = fel(640, 96, I.FP64, sigma2=0.3)
    got, hist, st, ohist, _ = run_fel(wl, 8)
    assert rel_linf(got, st.w) <= FP64_TOL
    amp = np.max(np.hypot(ohist[:, 0], ohist[:, 1]))
    assert np.max(np.abs(hist - ohist)) <= FP64_TOL * amp


def test_xpass_fel_fp32_reduced_grid():
    """The 4096 x 2048 FEL workload's physics (sigma_p 0.05) on 1024 x 512, 60 steps: f within
    the FP32 bound, |A| within the FP32 field bound of the parity tests (5e-4)."""
    wl = fel(1024, 512, I.FP32, dt=0.01, a0=0.05, sp=0.05, pr=(-0.8, 0.8))
    got, hist, st, ohist, _ = run_fel(wl, 60)
    assert rel_l1(got, st.w) <= FP32_TOL
    amp = np.hypot(ohist[:, 0], ohist[:, 1])
    assert np.max(np.abs(np.hypot(hist[:, 0], hist[:, 1]) - amp) / amp) <= 5e-4


def test_xpass_fel_4096x2048_full_size():
    wl = I.fel_4096x2048_fp32_cubic()
    got, hist, st, ohist, plan = run_fel(wl, 3)
    assert plan["kernel"] == XP
    assert rel_l1(got, st.w) <= FP32_TOL
    assert np.max(np.abs(hist - ohist)) <= 1e-6 * np.max(np.hypot(ohist[:, 0], ohist[:, 1]))


def test_xpass_unsupported_plans():
    rk4 = fel(512, 128, I.FP32, kind=I.PUSH_FEL_RK4)
    tent = pend(512, 128, I.FP32)
    for wl, kw in ((rk4, {}), (tent, dict(projection=I.PROJ_LUMPED))):
        with pytest.raises(V.VlasovError) as ei:
            V.Sim(wl.grid, wl.basis, wl.pusher, precision=I.FP32, kernel=XP, **kw)
        assert ei.value.status == V.VP_ERR_UNSUPPORTED
    long_row = pend(32772, 8, I.FP32)
    with pytest.raises(V.VlasovError) as ei:
        V.Sim(long_row.grid, long_row.basis, long_row.pusher, precision=I.FP32, kernel=XP)
    assert ei.value.status == V.VP_ERR_UNSUPPORTED
