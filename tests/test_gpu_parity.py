"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 GPU mode <= 1e-12 relative L-infinity (max|d| / max|f_oracle|);
FP32 mode <= 1e-5 relative L1 (sum|d| / sum|f_oracle|). FEL field histories: FP64
within the FP64 bound on |A|; FP32 within 5e-4 relative on |A| (FP32_FIELD_TOL): the
theta modulation of the initial state is 1e-4 of f, so FP32 rounding of f (about
1e-7 per value) is a perturbation of order 1e-4 relative of the early bunching and
hence of A.
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
# FEL field history in FP32 mode (stated, not given by the target): the initial theta
# modulation of f is 1e-4, so FP32 rounding of f (random, ~1e-7 per value per step)
# is a ~1e-4 relative perturbation of the early bunching and of |A|.
FP32_FIELD_TOL = 5e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def run_pair(wl: I.Workload, steps: int, kernel=V.VP_KERNEL_AUTO, tile=(0, 0), f0=None,
             projection=I.PROJ_GALERKIN):
    f0 = I.make_f0(wl) if f0 is None else f0
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=wl.precision, projection=projection,
                kernel=kernel, tile_x=tile[0], tile_p=tile[1])
    sim.set_f(f0 if wl.precision == I.FP64 else f0.astype(np.float32))
    sim.step(steps)
    got = sim.get_f()
    mom = sim.moments()
    hist = sim.field_history()
    st = O.State(wl.grid, wl.pusher, wl.basis, projection,
                 f0 if wl.precision == I.FP64 else f0.astype(np.float32).astype(np.float64))
    ohist = st.run(steps, history=True)
    sim.close()
    return got, st, mom, hist, ohist


def check(got, want, precision):
    if precision == I.FP64:
        e = rel_linf(got, want)
        assert e <= FP64_TOL, f"rel Linf {e:.3e}"
    else:
        e = rel_l1(got, want)
        assert e <= FP32_TOL, f"rel L1 {e:.3e}"
    return e


PI = math.pi


def pend(nx, np_, basis, precision, dt=0.05, pr=(-3.0, 3.0), pc=1.0, s=0.3, v_sign=1.0):
    return I.Workload("t", I.Grid(nx, np_, -PI, PI, *pr),
                      I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, v_sign, 1.0, dt), basis, precision, 0,
                      "gaussian", dict(xc=0.0, pc=pc, sx=s, sp=s))


def fel(nth, np_, precision, dt=0.01, a0=1e-3, sp=0.05, pr=(-4.0, 4.0), basis=I.BASIS_CUBIC):
    return I.Workload("t", I.Grid(nth, np_, 0.0, 2 * PI, *pr),
                      I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, dt, a0, 0.0), basis, precision, 0,
                      "fel_gaussian", dict(sp=sp, eps=1e-4))


# ------------------------------------------------------------------ the 128 x 128 FP64 workload
@pytest.mark.parametrize("kernel", [V.VP_KERNEL_TILED, V.VP_KERNEL_SCATTER])
def test_pendulum_128_fp64_tent_full_run(kernel):
    wl = I.pendulum_128_fp64_tent()
    got, st, mom, _, _ = run_pair(wl, wl.steps, kernel=kernel)
    check(got, st.w, I.FP64)
    om = st.moments()
    assert abs(mom["mass"] - om["mass"]) <= 1e-12 * om["mass"]
    assert abs(mom["lost_mass"] - st.lost[0] * wl.grid.hx * wl.grid.hp) <= 1e-15 + 1e-10 * om["mass"]


# ------------------------------------------------------------- every basis / pusher, FP64
@pytest.mark.parametrize("basis,proj", [(I.BASIS_TENT, I.PROJ_GALERKIN),
                                        (I.BASIS_CUBIC, I.PROJ_GALERKIN),
                                        (I.BASIS_CUBIC, I.PROJ_LUMPED)])
@pytest.mark.parametrize("shape,tile", [((200, 150), (64, 64)), ((96, 97), (32, 32)),
                                        ((37, 23), (0, 0)), ((300, 130), (96, 48))])
@pytest.mark.parametrize("kernel", [V.VP_KERNEL_TILED, V.VP_KERNEL_FUSED])
def test_pendulum_fp64_ragged_tiles(basis, proj, shape, tile, kernel):
    wl = pend(shape[0], shape[1], basis, I.FP64, dt=0.07, pc=0.8, s=0.5)
    got, st, _, _, _ = run_pair(wl, 15, kernel=kernel, tile=tile, projection=proj)
    check(got, st.w, I.FP64)


@pytest.mark.parametrize("pusher", ["rotation", "harmonic_kdk", "free", "paper_pendulum"])
@pytest.mark.parametrize("basis", [I.BASIS_TENT, I.BASIS_CUBIC])
def test_other_pushers_fp64(pusher, basis):
    if pusher == "rotation":
        pu = I.Pusher(I.PUSH_ROTATION, I.POT_HARMONIC, 1.0, 1.3, PI / 10 / 1.3)
        g = I.Grid(96, 80, -6.0, 6.0, -6.0, 6.0)
        args = dict(xc=0.8, pc=-0.3, sx=0.7, sp=0.9)
    elif pusher == "harmonic_kdk":
        pu = I.Pusher(I.PUSH_KDK, I.POT_HARMONIC, 1.0, 0.9, 0.2)
        g = I.Grid(96, 80, -6.0, 6.0, -6.0, 6.0)
        args = dict(xc=-0.5, pc=0.4, sx=0.7, sp=0.9)
    elif pusher == "free":
        pu = I.Pusher(I.PUSH_KDK, I.POT_FREE, 1.0, 1.0, 0.13)
        g = I.Grid(80, 64, -PI, PI, -3.0, 3.0)
        args = dict(xc=0.0, pc=0.0, sx=0.5, sp=0.8)
    else:   # the paper's pendulum sign and step (Sec. IV.A)
        pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, -1.0, 1.0, 2 * PI / 20)
        g = I.Grid(64, 64, -PI, PI, -3.0, 3.0)
        args = dict(xc=PI, pc=0.0, sx=1.2, sp=1.0)
    wl = I.Workload("t", g, pu, basis, I.FP64, 0, "gaussian", args)
    got, st, _, _, _ = run_pair(wl, 12)
    check(got, st.w, I.FP64)


def test_large_displacement_wraps_many_periods():
    """Rows move by more than a whole period per step (tiny grid, fast stream)."""
    g = I.Grid(16, 12, -PI, PI, -20.0, 20.0)
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.9)
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "gaussian", dict(xc=0.0, pc=0.0, sx=1.0, sp=9.0))
    for kernel in (V.VP_KERNEL_TILED, V.VP_KERNEL_SCATTER, V.VP_KERNEL_FUSED):
        got, st, _, _, _ = run_pair(wl, 4, kernel=kernel)
        check(got, st.w, I.FP64)


# ----------------------------------------------------------------------------- FEL, FP64
@pytest.mark.parametrize("basis,proj", [(I.BASIS_CUBIC, I.PROJ_GALERKIN), (I.BASIS_TENT, I.PROJ_GALERKIN),
                                        (I.BASIS_CUBIC, I.PROJ_LUMPED)])
@pytest.mark.parametrize("kernel", [V.VP_KERNEL_TILED, V.VP_KERNEL_SCATTER, V.VP_KERNEL_FUSED])
def test_fel_fp64_field_history(basis, proj, kernel):
    wl = fel(64, 96, I.FP64, dt=0.05, a0=0.05, sp=0.1, pr=(-1.0, 1.0), basis=basis)
    got, st, mom, hist, ohist = run_pair(wl, 40, kernel=kernel, projection=proj)
    check(got, st.w, I.FP64)
    amp = np.max(np.hypot(ohist[:, 0], ohist[:, 1]))
    assert np.max(np.abs(hist - ohist)) <= FP64_TOL * amp
    assert abs(mom["a_re"] - st.fel[0]) <= FP64_TOL * amp
    assert mom["step"] == 40 and abs(mom["tau"] - 40 * 0.05) < 1e-12


# ------------------------------------------------------------------------------- FP32
def test_pendulum_fp32_cubic_reduced_grid():
    """The 8192^2 workload's physics (two Gaussians, dt 0.02, p in [-4, 4]) on 512 x 512."""
    big = I.pendulum_8192_fp32_cubic(512, 512)
    got, st, _, _, _ = run_pair(big, 60)
    check(got, st.w, I.FP32)


def test_fel_fp32_cubic_reduced_grid():
    """The 4096 x 2048 FEL workload's physics (sigma_p 0.05 resolved by ~8 cells) on 256 x 256,
    150 steps. (FP32 rounding noise grows like sqrt(steps) under the Galerkin update; the
    long-run drift is measured separately, not gated here.)"""
    wl = fel(256, 256, I.FP32, pr=(-0.8, 0.8))
    got, st, _, hist, ohist = run_pair(wl, 150)
    check(got, st.w, I.FP32)
    amp = np.hypot(ohist[:, 0], ohist[:, 1])
    rel = np.max(np.abs(np.hypot(hist[:, 0], hist[:, 1]) - amp) / amp)
    assert rel <= FP32_FIELD_TOL, f"|A| rel err {rel:.2e}"


@pytest.mark.parametrize("kernel", [V.VP_KERNEL_TILED, V.VP_KERNEL_SCATTER, V.VP_KERNEL_FUSED])
def test_fp32_tent_and_lumped(kernel):
    for basis, proj in ((I.BASIS_TENT, I.PROJ_GALERKIN), (I.BASIS_CUBIC, I.PROJ_LUMPED)):
        wl = pend(300, 260, basis, I.FP32, dt=0.03, pr=(-4.0, 4.0), pc=0.5, s=0.5)
        got, st, _, _, _ = run_pair(wl, 30, kernel=kernel, projection=proj)
        check(got, st.w, I.FP32)


@pytest.mark.parametrize("tile", [(224, 64), (480, 32), (96, 128)])
def test_fused_fp32_galerkin_windowed_tiles(tile):
    """Fused one-pass kernel, windowed (not whole-row) tiles, ragged last tiles."""
    wl = pend(1100, 700, I.BASIS_CUBIC, I.FP32, dt=0.02, pr=(-4.0, 4.0), pc=0.5, s=0.4)
    got, st, mom, _, _ = run_pair(wl, 25, kernel=V.VP_KERNEL_FUSED, tile=tile)
    check(got, st.w, I.FP32)
    om = st.moments()
    assert abs(mom["mass"] - om["mass"]) <= 1e-6 * om["mass"]


def test_fused_fp32_fel_windowed():
    wl = fel(1024, 512, I.FP32, pr=(-0.8, 0.8), a0=0.05)
    got, st, _, hist, ohist = run_pair(wl, 60, kernel=V.VP_KERNEL_FUSED)
    check(got, st.w, I.FP32)
    amp = np.hypot(ohist[:, 0], ohist[:, 1])
    assert np.max(np.abs(np.hypot(hist[:, 0], hist[:, 1]) - amp) / amp) <= FP32_FIELD_TOL


def test_fused_matches_tiled_on_gpu():
    """Both GPU step kernels compute the same update (FP64, several steps)."""
    wl = pend(600, 400, I.BASIS_CUBIC, I.FP64, dt=0.03, pr=(-4.0, 4.0), pc=0.5, s=0.4)
    f0 = I.make_f0(wl)
    outs = []
    for kernel in (V.VP_KERNEL_TILED, V.VP_KERNEL_FUSED):
        sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=I.FP64, kernel=kernel)
        sim.set_f(f0)
        sim.step(10)
        outs.append(sim.get_f())
        sim.close()
    assert rel_linf(outs[1], outs[0]) <= 1e-13


# ------------------------------------------------------------------------------ edge cases
def test_zero_density_stays_zero():
    wl = pend(64, 64, I.BASIS_CUBIC, I.FP32)
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=I.FP32)
    sim.set_f(np.zeros((64, 64), dtype=np.float32))
    sim.step(3)
    assert not np.any(sim.get_f())
    sim.close()


def test_flattop_with_exact_zeros_and_negative_weights_fp64():
    g = I.Grid(64, 128, 0.0, 2 * PI, -0.5, 0.5)
    pu = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, 0.05, 1e-2, 0.0)
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "fel_flattop", dict(half_width=0.1, eps=1e-2))
    got, st, mom, _, _ = run_pair(wl, 10)
    check(got, st.w, I.FP64)
    om = st.moments()
    assert mom["neg_mass"] < 0 and abs(mom["neg_mass"] - om["neg_mass"]) <= 1e-12 * abs(om["neg_mass"]) + 1e-15


def test_minimum_grid_4x4():
    g = I.Grid(4, 4, -PI, PI, -1.0, 1.0)
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.3)
    f0 = np.random.default_rng(4).random((4, 4))
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "gaussian", {})
    got, st, _, _, _ = run_pair(wl, 3, f0=f0)
    check(got, st.w, I.FP64)


def test_moments_match_oracle_fp64():
    wl = pend(160, 120, I.BASIS_CUBIC, I.FP64, dt=0.05)
    got, st, mom, _, _ = run_pair(wl, 25)
    om = st.moments()
    for k in ("sum_w", "mass", "mean_x", "mean_p", "var_x", "var_p", "cov_xp", "energy",
              "trapped", "entropy", "neg_mass", "b_re", "b_im", "max_abs_w"):
        scale = max(abs(om[k]), 1e-3 * abs(om["sum_w"]) if k in ("neg_mass", "b_re", "b_im") else 1e-300)
        assert abs(mom[k] - om[k]) <= 1e-11 * scale, k


def test_nonfinite_input_is_reported_not_faulted():
    wl = pend(64, 64, I.BASIS_CUBIC, I.FP32)
    f0 = I.make_f0(wl).astype(np.float32)
    f0[10, 10] = np.nan
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=I.FP32)
    sim.set_f(f0)
    sim.step(1)
    with pytest.raises(V.VlasovError) as ei:
        sim.sync()
    assert ei.value.status == V.VP_ERR_NONFINITE
    sim.close()


def test_step_before_set_f_is_a_state_error():
    wl = pend(64, 64, I.BASIS_CUBIC, I.FP32)
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=I.FP32)
    with pytest.raises(V.VlasovError) as ei:
        sim.step(1)
    assert ei.value.status == V.VP_ERR_STATE
    sim.close()


@pytest.mark.parametrize("basis", [I.BASIS_TENT, I.BASIS_CUBIC])
def test_device_set_and_get_roundtrip(basis):
    """Tent: the state is w, the round trip is exact. Cubic Galerkin (one-pass kernel):
    the state is Lambda_p w, and w comes back through Lambda_p^{-1} within FP32 rounding."""
    wl = pend(640, 96, basis, I.FP32)
    f0 = torch.rand(96, 640, dtype=torch.float64, device="cuda")
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=I.FP32)
    sim.set_f(f0)
    out = torch.empty(96, 640, dtype=torch.float32, device="cuda")
    sim.get_f_device(out)
    torch.cuda.synchronize()
    if basis == I.BASIS_TENT:
        assert torch.equal(out, f0.float())
    else:
        assert torch.max(torch.abs(out.double() - f0)).item() <= 1e-6
    sim.close()


# ---------------------------------------------------------------- full-size workloads (bench config)
def test_pendulum_8192_fp32_cubic_one_step_full_size():
    """The benchmark's configuration (8192^2, tiles from the planner) for one step."""
    wl = I.pendulum_8192_fp32_cubic()
    got, st, _, _, _ = run_pair(wl, 1)
    check(got, st.w, I.FP32)


def test_fel_4096x2048_fp32_cubic_few_steps_full_size():
    wl = I.fel_4096x2048_fp32_cubic()
    got, st, _, hist, ohist = run_pair(wl, 3)
    check(got, st.w, I.FP32)
    assert np.max(np.abs(hist - ohist)) <= 1e-6 * np.max(np.hypot(ohist[:, 0], ohist[:, 1]))


@pytest.mark.parametrize("tile,steps", [((224, 63), 2), ((224, 60), 1)])
def test_pendulum_8192_fp32_cubic_at_bench_tiles(tile, steps):
    """The 8192^2 pendulum at the tile shapes the benchmark times: the autotuner's heights
    63 and 60 are not multiples of the 16-row p-solve chunk, so the last chunk of every
    tile column is ragged."""
    wl = I.pendulum_8192_fp32_cubic()
    got, st, _, _, _ = run_pair(wl, steps, kernel=V.VP_KERNEL_FUSED, tile=tile)
    check(got, st.w, I.FP32)


def test_pendulum_8192_fp32_cubic_at_the_autotuned_tile():
    """Exactly the plan the benchmark's headline line uses: the kernel and shape the autotuner
    picks on this device for the 8192^2 pendulum, two steps against the oracle."""
    wl = I.pendulum_8192_fp32_cubic()
    tuned = V.autotune([wl])[0]
    got, st, _, _, _ = run_pair(wl, 2, kernel=tuned["kernel"], tile=(tuned["tile_x"], tuned["tile_p"]))
    check(got, st.w, I.FP32)


def test_pendulum_8192_fp32_cubic_lumped_at_the_autotuned_tile():
    """The benchmark's lumped line: the 8192^2 pendulum with Lambda replaced by its row sum (the
    deposit alone), on the plan the autotuner picks for it, one step against the oracle."""
    wl = I.pendulum_8192_fp32_cubic()
    tuned = V.autotune([wl], projection=I.PROJ_LUMPED)[0]
    got, st, _, _, _ = run_pair(wl, 1, kernel=tuned["kernel"], tile=(tuned["tile_x"], tuned["tile_p"]),
                                projection=I.PROJ_LUMPED)
    check(got, st.w, I.FP32)
