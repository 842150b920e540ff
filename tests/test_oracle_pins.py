"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the dense
integral definitions of Sec. III (brute force), closed forms (free streaming,
rigid rotation, B-spline moment identities, the Lambda^{-1} decay law, the FEL
dispersion relation), invariants (mass, symplecticity, reversibility) and an
independent ODE integrator. No GPU is used.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp

from oracle import brute as B
from oracle import oracle as O
from paper_2007_12227_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CLOSED = json.load(open(os.path.join(GOLD, "closed_forms.json")))
PAPER = json.load(open(os.path.join(GOLD, "paper_parameters.json")))


def _pushed_cells(g, pu, a=(0.0, 0.0)):
    X, P = np.meshgrid(g.x_nodes(), g.p_nodes())
    xo, po = O.push(pu, X, P, a)
    return ((xo - g.x0) / g.hx).reshape(g.np, g.nx), ((po - g.p0) / g.hp).reshape(g.np, g.nx)


# --------------------------------------------------------------------------- brute force
@pytest.mark.parametrize("shape", [(8, 8), (9, 7)])
@pytest.mark.parametrize("pusher", ["pendulum", "rotation", "fel"])
@pytest.mark.parametrize("basis,proj", [(O.TENT, O.GALERKIN), (O.CUBIC, O.GALERKIN),
                                        (O.CUBIC, O.LUMPED), (O.SEPTIC, O.GALERKIN),
                                        (O.SEPTIC, O.LUMPED)])
def test_step_equals_dense_integral_definition(shape, pusher, basis, proj):
    """Sec. III: w_fin = Lambda^{-1} Delta^T w_in with Lambda, Delta as integrals."""
    nx, np_ = shape
    rng = np.random.default_rng(nx * 100 + np_ + 7 * basis + proj)
    if pusher == "pendulum":
        g = I.Grid(nx, np_, -math.pi, math.pi, -3.0, 3.0)
        pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.37)
        fel = None
        a = (0.0, 0.0)
    elif pusher == "rotation":
        g = I.Grid(nx, np_, -4.0, 4.0, -4.0, 4.0)
        pu = I.Pusher(I.PUSH_ROTATION, I.POT_HARMONIC, 1.0, 1.3, 0.41)
        fel = None
        a = (0.0, 0.0)
    else:
        g = I.Grid(nx, np_, 0.0, 2 * math.pi, -2.0, 2.0)
        pu = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, 0.3, 0.4, -0.2)
        fel = np.array([0.4, -0.2, 0.1, 0.05])
        h = pu.dt
        a = (fel[0] + 0.5 * h * fel[2], fel[1] + 0.5 * h * fel[3])
    w = rng.random((np_, nx)) - 0.2
    u, v = _pushed_cells(g, pu, a)
    kind = {O.TENT: "box", O.CUBIC: "tent", O.SEPTIC: "cubic"}[basis]
    want = B.dense_step(nx, np_, g.hx, g.hp, kind, u, v, w, lumped=(proj == O.LUMPED))
    got, _, _ = O.step(g, basis, proj, pu, w, fel)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_dense_brute_force_catches_a_planted_error():
    """The brute force is sensitive: a one-cell index slip in the deposit fails it."""
    g = I.Grid(8, 8, -math.pi, math.pi, -3.0, 3.0)
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.37)
    w = np.random.default_rng(3).random((8, 8))
    u, v = _pushed_cells(g, pu)
    good = B.dense_step(8, 8, g.hx, g.hp, "tent", u, v, w)
    bad = B.dense_step(8, 8, g.hx, g.hp, "tent", u + 1.0, v, w)
    got, _, _ = O.step(g, O.CUBIC, O.GALERKIN, pu, w)
    assert np.max(np.abs(got - good)) < 1e-12
    assert np.max(np.abs(got - bad)) > 1e-3


# --------------------------------------------------------------- deposit moment identities
def _single_node_step(basis, proj, dt, p_node_shift=0.0):
    """Push one interior node with free streaming and return its footprint."""
    nx, np_ = 96, 96
    g = I.Grid(nx, np_, -3.0, 3.0, -3.0, 3.0)
    pu = I.Pusher(I.PUSH_KDK, I.POT_FREE, 1.0, 1.0, dt)
    w = np.zeros((np_, nx))
    i0, j0 = 40, 55
    w[j0, i0] = 1.0
    out, _, lost = O.step(g, basis, proj, pu, w)
    x0, p0 = g.x_nodes()[i0], g.p_nodes()[j0]
    u = (x0 + dt * p0 - g.x0) / g.hx
    v = float(j0)
    c = np.arange(nx)
    c = c + nx * np.round((u - c) / nx)        # unwrap columns around u
    r = np.arange(np_)
    return out, u, v, c, r, lost


@pytest.mark.parametrize("dt", [0.0137, 0.29, -0.61])
def test_tent_deposit_moments(dt):
    """box basis: sum tent(u-c) = 1, sum c tent = u, sum c^2 tent = u^2 + t(1-t)."""
    out, u, v, c, r, lost = _single_node_step(O.TENT, O.GALERKIN, dt)
    col = out.sum(axis=0)
    t = u - math.floor(u)
    assert abs(col.sum() - 1.0) < 1e-14
    assert abs((col * c).sum() - u) < 1e-12
    assert abs((col * c * c).sum() - (u * u + t * (1 - t))) < 1e-10
    assert lost == 0.0


@pytest.mark.parametrize("dt", [0.0137, 0.29, -0.61])
def test_bspline_deposit_moments_lumped(dt):
    """tent basis, lumped: sum B3 = 1, first moment u, second u^2 + 1/3."""
    out, u, v, c, r, lost = _single_node_step(O.CUBIC, O.LUMPED, dt)
    col = out.sum(axis=0)
    ex = CLOSED["bspline_moments"]["second_moment_excess"]
    assert abs(col.sum() - 1.0) < 1e-14
    assert abs((col * c).sum() - u) < 1e-12
    assert abs((col * c * c).sum() - (u * u + ex)) < 1e-10


@pytest.mark.parametrize("dt", [0.0137, 0.29, -0.61])
def test_bspline_galerkin_transports_moments_exactly(dt):
    """tent basis, Galerkin: mass, first and second moments of the pushed node exactly."""
    out, u, v, c, r, lost = _single_node_step(O.CUBIC, O.GALERKIN, dt)
    col = out.sum(axis=0)
    row = out.sum(axis=1)
    assert abs(col.sum() - 1.0) < 1e-12
    assert abs((col * c).sum() - u) < 1e-10
    assert abs((col * c * c).sum() - u * u) < 1e-8
    assert abs((row * r).sum() - v) < 1e-10
    assert abs((row * r * r).sum() - v * v) < 1e-8


# ---------------------------------------------------------------- closed-form transports
@pytest.mark.parametrize("basis,proj", [(O.TENT, O.GALERKIN), (O.CUBIC, O.GALERKIN)])
def test_zero_step_is_identity(basis, proj):
    g = I.Grid(32, 24, -math.pi, math.pi, -3.0, 3.0)
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.0)
    w = np.random.default_rng(1).random((24, 32))
    out, _, lost = O.step(g, basis, proj, pu, w)
    assert np.max(np.abs(out - w)) < 1e-14 * np.max(np.abs(w)) * 10
    if basis == O.TENT:
        assert lost == 0.0
    else:   # the B3 footprint of an edge node reaches past the grid; Galerkin still returns w
        assert lost > 0.0


@pytest.mark.parametrize("basis", [O.TENT, O.CUBIC])
@pytest.mark.parametrize("m", [1, 3])
def test_free_streaming_integer_shift_is_exact(basis, m):
    """V = 0 and dt = m hx / hp: row j moves by m (j - jc) cells exactly."""
    nx, np_ = 64, 41
    hp = 0.1
    g = I.Grid(nx, np_, -math.pi, math.pi, -2.0, -2.0 + hp * (np_ - 1))
    jc = 20                                   # p_jc = 0
    dt = m * g.hx / g.hp
    pu = I.Pusher(I.PUSH_KDK, I.POT_FREE, 1.0, 1.0, dt)
    w = np.random.default_rng(m).random((np_, nx))
    out, _, _ = O.step(g, basis, O.GALERKIN, pu, w)
    want = np.empty_like(w)
    for j in range(np_):
        want[j] = np.roll(w[j], m * (j - jc))
    assert np.max(np.abs(out - want)) < 1e-12


def test_free_streaming_converges_to_characteristics():
    """V = 0: f(x, p, t) = f0(x - p t, p); Galerkin-B3 error falls faster than 2nd order."""
    errs = []
    for n in (32, 64):
        g = I.Grid(n, n, -math.pi, math.pi, -3.0, 3.0)
        pu = I.Pusher(I.PUSH_KDK, I.POT_FREE, 1.0, 1.0, 0.1)
        x, p = g.x_nodes(), g.p_nodes()
        f0 = lambda X, P: np.exp(-0.5 * ((X + math.pi) % (2 * math.pi) - math.pi) ** 2 / 0.5 ** 2) * \
            np.exp(-0.5 * P ** 2 / 0.7 ** 2)
        X, P = np.meshgrid(x, p)
        st = O.State(g, pu, O.CUBIC, O.GALERKIN, f0(X, P))
        st.run(10)
        err = np.max(np.abs(st.w - f0(X - P * 1.0, P)))
        errs.append(err)
    assert errs[1] < errs[0] / 3.0


# --------------------------------------------------------------------------- pushers
def test_exact_rotation_one_revolution_and_ode():
    """Sec. IV.A: phase advance pi/10 per step; 20 steps are one revolution."""
    adv = PAPER["oscillator_phase_advance_per_step"]["float"]
    nrev = PAPER["oscillator_steps_per_revolution"]["value"]
    omega = 1.7
    pu = I.Pusher(I.PUSH_ROTATION, I.POT_HARMONIC, 1.0, omega, adv / omega)
    rng = np.random.default_rng(5)
    x0, p0 = rng.normal(size=50), rng.normal(size=50)
    x, p = x0.copy(), p0.copy()
    for _ in range(nrev):
        x, p = O.push(pu, x, p)
    assert np.max(np.abs(x - x0)) < 1e-13 and np.max(np.abs(p - p0)) < 1e-13
    # one step against an independent ODE integration of x'' = -omega^2 x
    x1, p1 = O.push(pu, x0[:5], p0[:5])
    for k in range(5):
        sol = solve_ivp(lambda t, y: [y[1], -omega ** 2 * y[0]], (0, pu.dt), [x0[k], p0[k]],
                        method="DOP853", rtol=1e-13, atol=1e-14)
        assert abs(sol.y[0, -1] - x1[k]) < 1e-10 and abs(sol.y[1, -1] - p1[k]) < 1e-10


def test_kdk_pendulum_symplectic_reversible_second_order():
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.1)
    rng = np.random.default_rng(9)
    x, p = rng.uniform(-3, 3, 20), rng.uniform(-2, 2, 20)
    # area preservation: det of the finite-difference Jacobian = 1
    e = 1e-6
    xa, pa = O.push(pu, x + e, p)
    xb, pb = O.push(pu, x - e, p)
    xc, pc = O.push(pu, x, p + e)
    xd, pd = O.push(pu, x, p - e)
    det = ((xa - xb) * (pc - pd) - (xc - xd) * (pa - pb)) / (4 * e * e)
    assert np.max(np.abs(det - 1.0)) < 1e-7
    # time reversibility: KDK(-h) o KDK(h) = id
    x1, p1 = O.push(pu, x, p)
    back = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, -0.1)
    x2, p2 = O.push(back, x1, p1)
    assert np.max(np.abs(x2 - x)) < 1e-14 and np.max(np.abs(p2 - p)) < 1e-14
    # local error O(h^3) against an independent integrator of x'' = -sin x
    def err(h):
        q = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, h)
        xo, po = O.push(q, x[:4], p[:4])
        m = 0.0
        for k in range(4):
            s = solve_ivp(lambda t, y: [y[1], -math.sin(y[0])], (0, h), [x[k], p[k]],
                          method="DOP853", rtol=1e-13, atol=1e-14)
            m = max(m, abs(s.y[0, -1] - xo[k]) + abs(s.y[1, -1] - po[k]))
        return m
    r = err(0.2) / err(0.1)
    assert 6.0 < r < 10.0


def test_pendulum_sign_reading():
    """v_sign = -1 is the paper's H = p^2/2 + cos x: its stable centre sits at x = pi."""
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, PAPER["pendulum_hamiltonian"]["v_sign"], 1.0, 0.1)
    x, p = O.push(pu, np.array([math.pi - 0.1]), np.array([0.0]))
    assert p[0] > 0          # pulled back toward x = pi
    x, p = O.push(pu, np.array([0.1]), np.array([0.0]))
    assert p[0] > 0          # pushed away from the X-point at x = 0


# ---------------------------------------------------------------- mass-matrix inverse
def test_cyclic_and_open_inverse_decay_law():
    """Lambda^{-1} of a unit impulse decays as sqrt(3) z1^|d| per axis (interior)."""
    z1 = CLOSED["tent_basis_mass_matrix_inverse"]["z1"]
    c0 = CLOSED["tent_basis_mass_matrix_inverse"]["c0"]
    g = I.Grid(64, 80, -math.pi, math.pi, -4.0, 4.0)
    r = np.zeros((80, 64))
    r[40, 10] = 1.0
    w = O.mass_solve(g, r)
    di = np.arange(64) - 10
    di = (di + 32) % 64 - 32
    dj = np.arange(80) - 40
    want = np.outer(c0 * z1 ** np.abs(dj), c0 * z1 ** np.abs(di)) / (g.hx * g.hp)
    assert np.max(np.abs(w - want)) < 1e-12 * np.max(np.abs(want))
    # the open-edge rows differ from the lattice law, and match the dense inverse
    r = np.zeros((80, 64))
    r[0, 10] = 1.0
    w = O.mass_solve(g, r)
    T = (np.diag(np.full(80, 2 / 3)) + np.diag(np.full(79, 1 / 6), 1) + np.diag(np.full(79, 1 / 6), -1))
    col = w[:, 10] * g.hp * g.hx / c0          # x factor at zero offset is c0 / hx
    want_col = np.linalg.inv(T)[:, 0]
    assert np.max(np.abs(col - want_col)) < 1e-12


# --------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("basis,proj", [(O.TENT, O.GALERKIN), (O.CUBIC, O.GALERKIN),
                                        (O.CUBIC, O.LUMPED)])
def test_mass_conserved_when_nothing_reaches_the_momentum_edge(basis, proj):
    """Sec. III global volume conservation; Sec. IV loss only through the open momentum edge."""
    g = I.Grid(64, 64, -math.pi, math.pi, -3.0, 3.0)
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.05)
    wl = I.Workload("t", g, pu, basis, I.FP64, 40, "gaussian", dict(xc=0.0, pc=0.3, sx=0.3, sp=0.3))
    st = O.State(g, pu, basis, proj, I.make_f0(wl))
    m0 = st.moments()["mass"]
    st.run(40)
    m1 = st.moments()["mass"]
    lost_mass = st.lost[0] * g.hx * g.hp
    assert lost_mass < 1e-10           # only far tails of the numerical spreading reach the edge
    if proj == O.LUMPED or basis == O.TENT:
        assert abs(m1 + lost_mass - m0) < 1e-14     # exact accounting: deposit sums to one
    else:
        assert abs(m1 - m0) < 1e-11


def test_lost_weight_accounts_for_mass_change_tent():
    """TENT: mass lost = weight deposited beyond the open momentum edge."""
    g = I.Grid(32, 32, -math.pi, math.pi, -1.0, 1.0)
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.2)
    wl = I.Workload("t", g, pu, I.BASIS_TENT, I.FP64, 10, "gaussian",
                    dict(xc=0.0, pc=0.5, sx=0.5, sp=0.4))
    st = O.State(g, pu, O.TENT, O.GALERKIN, I.make_f0(wl))
    s0 = st.w.sum()
    st.run(10)
    assert st.lost[0] > 1e-3 * s0
    assert abs(st.w.sum() + st.lost[0] - s0) < 1e-12 * s0


def test_tent_mode_positive_and_l1_contractive():
    g = I.Grid(48, 48, -math.pi, math.pi, -3.0, 3.0)
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, -1.0, 1.0, 2 * math.pi / 20)
    w = np.random.default_rng(2).random((48, 48))
    st = O.State(g, pu, O.TENT, O.GALERKIN, w)
    l1 = np.abs(st.w).sum()
    st.run(15)
    assert st.w.min() >= 0.0
    assert np.abs(st.w).sum() <= l1 * (1 + 1e-14)


def test_galerkin_rotation_rotates_covariance_exactly():
    """Affine push + Galerkin tent basis: mean and covariance rotate exactly."""
    omega = 1.0
    g = I.Grid(128, 128, -9.0, 9.0, -9.0, 9.0)
    pu = I.Pusher(I.PUSH_ROTATION, I.POT_HARMONIC, 1.0, omega, math.pi / 10)
    X, P = np.meshgrid(g.x_nodes(), g.p_nodes())
    f0 = np.exp(-0.5 * ((X - 0.8) / 0.5) ** 2 - 0.5 * ((P + 0.3) / 0.9) ** 2 - 0.4 * (X - 0.8) * (P + 0.3))
    st = O.State(g, pu, O.CUBIC, O.GALERKIN, f0)
    m0 = st.moments()
    nst = 3
    st.run(nst)
    m1 = st.moments()
    th = omega * pu.dt * nst
    R = np.array([[math.cos(th), math.sin(th) / omega], [-omega * math.sin(th), math.cos(th)]])
    mu0 = np.array([m0["mean_x"], m0["mean_p"]])
    S0 = np.array([[m0["var_x"], m0["cov_xp"]], [m0["cov_xp"], m0["var_p"]]])
    mu1 = np.array([m1["mean_x"], m1["mean_p"]])
    S1 = np.array([[m1["var_x"], m1["cov_xp"]], [m1["cov_xp"], m1["var_p"]]])
    assert np.max(np.abs(mu1 - R @ mu0)) < 1e-12
    assert np.max(np.abs(S1 - R @ S0 @ R.T)) < 1e-12


def test_lumped_bspline_adds_one_third_cell_squared_per_step():
    g = I.Grid(128, 128, -9.0, 9.0, -9.0, 9.0)
    pu = I.Pusher(I.PUSH_ROTATION, I.POT_HARMONIC, 1.0, 1.0, 0.0)   # no motion
    X, P = np.meshgrid(g.x_nodes(), g.p_nodes())
    st = O.State(g, pu, O.CUBIC, O.LUMPED, np.exp(-0.5 * (X ** 2 + P ** 2)))
    v0 = st.moments()
    st.run(2)
    v1 = st.moments()
    ex = CLOSED["bspline_moments"]["second_moment_excess"]
    assert abs(v1["var_x"] - v0["var_x"] - 2 * ex * g.hx ** 2) < 1e-13
    assert abs(v1["var_p"] - v0["var_p"] - 2 * ex * g.hp ** 2) < 1e-13


# ------------------------------------------------------------------------------ moments
def test_moments_of_a_resolved_gaussian():
    g = I.Grid(128, 129, -math.pi, math.pi, -4.0, 4.0)
    sx, sp, pc = 0.4, 0.5, 0.25
    wl = I.Workload("t", g, I.Pusher(), I.BASIS_CUBIC, I.FP64, 0, "gaussian",
                    dict(xc=0.0, pc=pc, sx=sx, sp=sp))
    w = I.make_f0(wl)
    m = O.moments(g, I.Pusher(I.PUSH_KDK, I.POT_HARMONIC, 1.0, 2.0, 0.1), w)
    assert abs(m["mass"] - 1.0) < 1e-13
    assert abs(m["mean_p"] - pc) < 1e-10 and abs(m["mean_x"]) < 1e-12
    assert abs(m["var_x"] - sx ** 2) < 1e-10 and abs(m["var_p"] - sp ** 2) < 1e-10
    assert abs(m["energy"] - (0.5 * (sp ** 2 + pc ** 2) + 0.5 * 4.0 * sx ** 2)) < 1e-9
    assert abs(m["entropy"] - math.log(2 * math.pi * math.e * sx * sp)) < 1e-8
    assert m["neg_mass"] == 0.0


def test_pendulum_trapped_mass_converges_with_grid():
    """The region H < 1 is invariant under the flow: trapped mass drift shrinks with h."""
    drifts = []
    for n in (64, 128):
        g = I.Grid(n, n, -math.pi, math.pi, -3.0, 3.0)
        pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.05)
        wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "gaussian",
                        dict(xc=0.0, pc=1.0, sx=0.3, sp=0.3))
        st = O.State(g, pu, O.CUBIC, O.GALERKIN, I.make_f0(wl))
        t0 = st.moments()["trapped"]
        st.run(40)
        drifts.append(abs(st.moments()["trapped"] - t0) / t0)
    assert drifts[1] < 0.7 * drifts[0]
    assert drifts[1] < 0.05


# ---------------------------------------------------------------------------------- FEL
def _fel_root(sp, delta=0.0, sigma2=0.0, lam=None):
    """Growing root of the linearised FEL equations of Sec. IV.B for a Gaussian f0 of spread sp.

    With f = f0(p) + f1(p) e^{i theta + lambda z}, A ~ e^{lambda z} and b = <e^{-i theta}>,
    d theta/dz = delta + p and the kick amplitude A + i sigma2 b give
    b = (A + i sigma2 b) J(lambda), J = int f0'(p) / (lambda + i (delta + p)) dp, and
    dA/dz = b gives lambda A = b:  lambda (1 - i sigma2 J) = J.
    """
    def J(l):
        f = lambda p: -p / sp ** 2 * math.exp(-0.5 * (p / sp) ** 2) / (math.sqrt(2 * math.pi) * sp)
        re = quad(lambda p: (f(p) / (l + 1j * (delta + p))).real, -12 * sp, 12 * sp, limit=400)[0]
        im = quad(lambda p: (f(p) / (l + 1j * (delta + p))).imag, -12 * sp, 12 * sp, limit=400)[0]
        return re + 1j * im

    def disp(l):
        j = J(l)
        return l * (1 - 1j * sigma2 * j) - j
    if lam is None:
        lam = complex(CLOSED["fel_cold_beam_growth"]["lambda_re"], CLOSED["fel_cold_beam_growth"]["lambda_im"])
    for _ in range(50):
        d = disp(lam)
        e = 1e-7
        der = (disp(lam + e) - d) / e
        step = d / der
        lam -= step
        if abs(step) < 1e-13:
            break
    return lam


def test_fel_dispersion_root_cold_limit():
    lam = _fel_root(1e-3)
    assert abs(lam.real - math.sqrt(3) / 2) < 2e-3
    assert abs(lam.imag - 0.5) < 2e-3


def test_fel_linear_growth_rate_matches_warm_beam_theory():
    """ln|A| grows at Re(lambda) of the warm-beam dispersion relation (Sec. IV.B model)."""
    sp = 0.05
    g = I.Grid(32, 256, 0.0, 2 * math.pi, -0.4, 0.4)
    pu = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, 0.01, 1e-6, 0.0)
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "fel_gaussian", dict(sp=sp, eps=1e-6))
    st = O.State(g, pu, O.CUBIC, O.GALERKIN, I.make_f0(wl))
    nst = 1000
    hist = st.run(nst, history=True)
    tau = (np.arange(nst) + 1) * pu.dt
    amp = np.log(np.hypot(hist[:, 0], hist[:, 1]))
    sel = (tau >= 5.0) & (tau <= 10.0)       # growing mode dominant, still linear (|A| < 0.01)
    slope = np.polyfit(tau[sel], amp[sel], 1)[0]
    lam = _fel_root(sp)
    assert abs(slope - lam.real) < 5e-3 * lam.real
    assert lam.real < math.sqrt(3) / 2          # a warm beam grows slower than a cold one
    assert amp[-1] < math.log(0.01)


def _cold_root(delta, sigma2):
    """Cold beam (f0 = a delta function): J = i / (lambda + i delta)^2, so
    lambda (lambda + i delta)^2 + sigma2 lambda - i = 0; the root of largest growth."""
    r = np.roots([1.0, 2j * delta, sigma2 - delta ** 2, -1j])
    return r[np.argmax(r.real)]


@pytest.mark.parametrize("delta,sigma2", [(0.3, 0.2), (-0.4, 0.1), (0.0, 0.3)])
def test_fel_dispersion_with_detuning_and_space_charge_cold_limit(delta, sigma2):
    """The warm-beam relation reduces to the cold-beam cubic as the energy spread vanishes."""
    c = _cold_root(delta, sigma2)
    lam = _fel_root(1e-3, delta, sigma2, lam=c)
    assert abs(lam - c) < 2e-3
    # space charge slows the growth, and so does detuning from resonance
    assert c.real < math.sqrt(3) / 2


@pytest.mark.parametrize("delta,sigma2", [(0.3, 0.2), (-0.4, 0.1), (0.0, 0.3)])
def test_fel_growth_with_detuning_and_space_charge_matches_theory(delta, sigma2):
    """Full FEL model of Sec. IV.B: ln|A| grows at Re(lambda) and the phase of A turns at
    Im(lambda) of the warm-beam relation with detuning delta and space charge sigma2."""
    sp = 0.05
    g = I.Grid(32, 256, 0.0, 2 * math.pi, -0.5, 0.5)
    pu = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, 0.01, 1e-6, 0.0, delta, sigma2)
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "fel_gaussian", dict(sp=sp, eps=1e-6))
    st = O.State(g, pu, O.CUBIC, O.GALERKIN, I.make_f0(wl))
    nst = 1000
    hist = st.run(nst, history=True)
    tau = (np.arange(nst) + 1) * pu.dt
    a = hist[:, 0] + 1j * hist[:, 1]
    sel = (tau >= 5.0) & (tau <= 10.0)
    growth = np.polyfit(tau[sel], np.log(np.abs(a[sel])), 1)[0]
    turn = np.polyfit(tau[sel], np.unwrap(np.angle(a[sel])), 1)[0]
    lam = _fel_root(sp, delta, sigma2, lam=_cold_root(delta, sigma2))
    assert abs(growth - lam.real) < 5e-3 * lam.real
    assert abs(turn - lam.imag) < 5e-3 * max(1.0, abs(lam.imag))


def _energy_drifts(kind, dts, sigma2=0.0):
    """|change of <p> + |A|^2| over tau = 1 (no weight leaves the momentum range)."""
    out = []
    for dt in dts:
        g = I.Grid(64, 256, 0.0, 2 * math.pi, -2.5, 2.5)
        pu = I.Pusher(kind, I.POT_FREE, 1.0, 1.0, dt, 0.3, 0.0, 0.0, sigma2)
        wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "fel_gaussian", dict(sp=0.1, eps=1e-2))
        st = O.State(g, pu, O.CUBIC, O.GALERKIN, I.make_f0(wl))
        e0 = st.moments()["energy"]
        st.run(int(round(1.0 / dt)))
        assert st.lost[0] < 1e-30
        out.append(abs(st.moments()["energy"] - e0))
    return out


@pytest.mark.parametrize("sigma2", [0.0, 0.3])
def test_fel_rk4_is_fourth_order_and_dkd_second(sigma2):
    """<p> + |A|^2 is invariant under the FEL equations (also with space charge: the i sigma2 |b|^2
    term is imaginary). The Galerkin update carries the mean of p exactly, so its drift is the
    integrator's: halving dt cuts it ~16x for RK4 (Sec. IV.B's integrator) and ~4x for DKD."""
    rk = _energy_drifts(I.PUSH_FEL_RK4, (0.2, 0.1, 0.05), sigma2)
    dkd = _energy_drifts(I.PUSH_FEL, (0.2, 0.1, 0.05), sigma2)
    for a, b in zip(rk, rk[1:]):
        assert 12.0 < a / b < 20.0
    for a, b in zip(dkd, dkd[1:]):
        assert 3.5 < a / b < 4.5
    assert rk[-1] < dkd[-1] / 100


@pytest.mark.parametrize("delta,sigma2", [(0.0, 0.0), (0.3, 0.2)])
def test_fel_rk4_growth_matches_theory(delta, sigma2):
    """The RK4 integrator gives the same linear growth and phase velocity of A."""
    sp = 0.05
    g = I.Grid(32, 256, 0.0, 2 * math.pi, -0.5, 0.5)
    pu = I.Pusher(I.PUSH_FEL_RK4, I.POT_FREE, 1.0, 1.0, 0.02, 1e-6, 0.0, delta, sigma2)
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "fel_gaussian", dict(sp=sp, eps=1e-6))
    st = O.State(g, pu, O.CUBIC, O.GALERKIN, I.make_f0(wl))
    nst = 500
    hist = st.run(nst, history=True)
    tau = (np.arange(nst) + 1) * pu.dt
    a = hist[:, 0] + 1j * hist[:, 1]
    sel = (tau >= 5.0) & (tau <= 10.0)
    growth = np.polyfit(tau[sel], np.log(np.abs(a[sel])), 1)[0]
    turn = np.polyfit(tau[sel], np.unwrap(np.angle(a[sel])), 1)[0]
    lam = _fel_root(sp, delta, sigma2, lam=_cold_root(delta, sigma2))
    assert abs(growth - lam.real) < 5e-3 * lam.real
    assert abs(turn - lam.imag) < 5e-3 * max(1.0, abs(lam.imag))


def test_fel_energy_invariant_drift_is_second_order():
    """<p> + |A|^2 is conserved by the FEL equations; DKD drift falls ~4x when dt halves."""
    drift = []
    for dt in (0.04, 0.02):
        g = I.Grid(32, 128, 0.0, 2 * math.pi, -1.0, 1.0)
        pu = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, dt, 0.3, 0.0)
        wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "fel_gaussian", dict(sp=0.1, eps=1e-2))
        st = O.State(g, pu, O.CUBIC, O.GALERKIN, I.make_f0(wl))
        e0 = st.moments()["energy"]
        st.run(int(round(1.0 / dt)))
        drift.append(abs(st.moments()["energy"] - e0))
    assert drift[1] < drift[0] / 2.5


# ---------------------------------------------------------------- paper's qualitative claims
def test_flattop_fel_grows_negative_weights_gaussian_does_not():
    """Sec. IV.B: a hard edge in energy gives negative weights almost at once; a Gaussian not."""
    hw = PAPER["fel_flattop_half_width"]["value"]
    g = I.Grid(32, 128, 0.0, 2 * math.pi, -0.5, 0.5)
    pu = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, 0.05, 1e-2, 0.0)
    res = {}
    for name, args in (("fel_flattop", dict(half_width=hw, eps=1e-2)),
                       ("fel_gaussian", dict(sp=0.05, eps=1e-2))):
        wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, name, args)
        st = O.State(g, pu, O.CUBIC, O.GALERKIN, I.make_f0(wl))
        st.run(5)
        res[name] = st.moments()["neg_mass"]
    assert res["fel_flattop"] < -1e-4
    assert res["fel_gaussian"] > -1e-8


def test_paper_pendulum_negative_weights_galerkin_only():
    """Sec. IV.A: negative weights near the X-point for the tent basis, never for TENT deposit."""
    g = I.Grid(64, 64, -math.pi, math.pi, -3.0, 3.0)
    h = PAPER["pendulum_step"]["float"]
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, PAPER["pendulum_hamiltonian"]["v_sign"], 1.0, h)
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "gaussian",
                    dict(xc=math.pi, pc=0.0, sx=1.2, sp=1.0))
    f0 = I.make_f0(wl)
    gal = O.State(g, pu, O.CUBIC, O.GALERKIN, f0)
    tent = O.State(g, pu, O.TENT, O.GALERKIN, f0)
    gal.run(30)
    tent.run(30)
    assert gal.moments()["neg_mass"] < -1e-6
    assert tent.moments()["neg_mass"] == 0.0
    assert abs(gal.moments()["mass"] + gal.lost[0] * g.hx * g.hp - 1.0) < 5e-3


# ------------------------------------------------- smoother basis (Sec. V remark), measured
def test_cubic_spline_basis_galerkin_has_more_negative_weight_than_tent_basis():
    """Sec. V suggests smoother basis functions might ameliorate the negative weights. With the
    Galerkin (L2) projection onto cubic B-spline basis functions (B7 deposit, 7-band Lambda) the
    negative mass of the paper's flat-top FEL and pendulum runs is larger than with the tent
    basis, not smaller; the lumped projection (non-negative deposit) keeps every weight >= 0."""
    hw = PAPER["fel_flattop_half_width"]["value"]
    g = I.Grid(64, 128, 0.0, 2 * math.pi, -0.5, 0.5)
    pu = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, 0.05, 1e-2, 0.0)
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "fel_flattop", dict(half_width=hw, eps=1e-2))
    neg = {}
    for basis in (O.CUBIC, O.SEPTIC):
        st = O.State(g, pu, basis, O.GALERKIN, I.make_f0(wl))
        st.run(5)
        neg[basis] = st.moments()["neg_mass"]
    assert neg[O.SEPTIC] < 1.2 * neg[O.CUBIC] < 0.0
    st = O.State(g, pu, O.SEPTIC, O.LUMPED, I.make_f0(wl))
    st.run(5)
    assert st.moments()["neg_mass"] == 0.0


def test_septic_galerkin_transports_mean_and_covariance_under_rotation():
    """The cubic B-spline basis Galerkin step also carries the mean and covariance of a
    Gaussian exactly through a rigid rotation (as the tent basis does)."""
    omega = 1.0
    g = I.Grid(96, 96, -9.0, 9.0, -9.0, 9.0)
    pu = I.Pusher(I.PUSH_ROTATION, I.POT_HARMONIC, 1.0, omega, math.pi / 10)
    X, P = np.meshgrid(g.x_nodes(), g.p_nodes())
    f0 = np.exp(-0.5 * ((X - 0.8) / 0.5) ** 2 - 0.5 * ((P + 0.3) / 0.9) ** 2 - 0.4 * (X - 0.8) * (P + 0.3))
    st = O.State(g, pu, O.SEPTIC, O.GALERKIN, f0)
    m0 = st.moments()
    nst = 3
    st.run(nst)
    m1 = st.moments()
    th = omega * pu.dt * nst
    R = np.array([[math.cos(th), math.sin(th) / omega], [-omega * math.sin(th), math.cos(th)]])
    mu0 = np.array([m0["mean_x"], m0["mean_p"]])
    S0 = np.array([[m0["var_x"], m0["cov_xp"]], [m0["cov_xp"], m0["var_p"]]])
    mu1 = np.array([m1["mean_x"], m1["mean_p"]])
    S1 = np.array([[m1["var_x"], m1["cov_xp"]], [m1["cov_xp"], m1["var_p"]]])
    assert np.max(np.abs(mu1 - R @ mu0)) < 1e-12
    assert np.max(np.abs(S1 - R @ S0 @ R.T)) < 1e-11
