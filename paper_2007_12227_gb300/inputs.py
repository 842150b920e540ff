"""Seeded synthetic inputs for the phase-space Vlasov step.

This module is shared by the CUDA path, the tests and the benchmark. It holds
no arithmetic of the method itself (no push, no deposit, no mass-matrix solve):
only the grids, the initial densities sampled at mesh nodes, a counter-based
random generator and the concrete workload definitions.

Grid convention (the paper fixes periodic coordinates and open momenta, Sec. IV):
  x_i = x0 + i * (x1 - x0) / nx,   i = 0 .. nx-1   (periodic, period x1 - x0)
  p_j = p0 + j * (p1 - p0) / (np - 1), j = 0 .. np-1 (open, both ends included)
Arrays are row-major [np][nx]: x is the fastest index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

# enum values mirror include/vlasov.h
# deposit kernels: tent (top-hat basis), B3 (tent basis), B7 (cubic B-spline basis)
BASIS_TENT, BASIS_CUBIC, BASIS_SEPTIC = 0, 1, 2
PUSH_KDK, PUSH_ROTATION, PUSH_FEL, PUSH_FEL_RK4 = 0, 1, 2, 3
POT_FREE, POT_PENDULUM, POT_HARMONIC = 0, 1, 2
FP32, FP64 = 0, 1
PROJ_GALERKIN, PROJ_LUMPED = 0, 1

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014): counter-based 64-bit generator."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """53-bit uniform in [lo, hi)."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def loguniform(self, lo: float, hi: float) -> float:
        return math.exp(self.uniform(math.log(lo), math.log(hi)))

    def choice(self, items):
        return items[self.next_u64() % len(items)]

    def exponential(self, rate: float) -> float:
        u = self.uniform()
        return -math.log1p(-u) / rate


@dataclass
class Grid:
    nx: int
    np: int
    x0: float
    x1: float
    p0: float
    p1: float

    @property
    def hx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def hp(self) -> float:
        return (self.p1 - self.p0) / (self.np - 1)

    def x_nodes(self) -> np.ndarray:
        return self.x0 + np.arange(self.nx, dtype=np.float64) * self.hx

    def p_nodes(self) -> np.ndarray:
        return self.p0 + np.arange(self.np, dtype=np.float64) * self.hp

    @property
    def nodes(self) -> int:
        return self.nx * self.np


@dataclass
class Pusher:
    kind: int = PUSH_KDK
    potential: int = POT_PENDULUM
    v_sign: float = 1.0        # pendulum: V(x) = -v_sign * cos(x)
    omega: float = 1.0         # harmonic: V(x) = omega^2 x^2 / 2
    dt: float = 0.05
    a0_re: float = 0.0         # FEL field amplitude at tau = 0
    a0_im: float = 0.0
    delta: float = 0.0         # FEL detuning: d theta/dz = delta + p
    sigma2: float = 0.0        # FEL space charge: kick amplitude A + i sigma2 <exp(-i theta)>


@dataclass
class Workload:
    name: str
    grid: Grid
    pusher: Pusher
    basis: int
    precision: int
    steps: int
    f0: str                    # initial-density recipe name
    f0_args: dict = field(default_factory=dict)
    projection: int = PROJ_GALERKIN


def _wrap(d: np.ndarray, period: float) -> np.ndarray:
    """Distance wrapped into [-period/2, period/2)."""
    return (d + 0.5 * period) % period - 0.5 * period


def gaussian2d(grid: Grid, xc: float, pc: float, sx: float, sp: float) -> np.ndarray:
    x = _wrap(grid.x_nodes() - xc, grid.x1 - grid.x0)
    p = grid.p_nodes() - pc
    return np.exp(-0.5 * (p[:, None] / sp) ** 2) * np.exp(-0.5 * (x[None, :] / sx) ** 2)


def normalise(grid: Grid, f: np.ndarray) -> np.ndarray:
    """Scale so that sum(f) * hx * hp == 1."""
    return f / (f.sum() * grid.hx * grid.hp)


def make_f0(wl: Workload) -> np.ndarray:
    """Initial nodal weights w_ij = f0(x_i, p_j), normalised, float64 [np][nx]."""
    g, a = wl.grid, wl.f0_args
    if wl.f0 == "gaussian":
        f = gaussian2d(g, a["xc"], a["pc"], a["sx"], a["sp"])
    elif wl.f0 == "two_gaussians":
        f = a["c1"] * gaussian2d(g, a["xc1"], a["pc1"], a["s1"], a["s1"]) + \
            a["c2"] * gaussian2d(g, a["xc2"], a["pc2"], a["s2"], a["s2"])
    elif wl.f0 == "fel_gaussian":
        th = g.x_nodes()
        p = g.p_nodes()
        f = np.exp(-0.5 * ((p - a.get("pc", 0.0)) / a["sp"]) ** 2)[:, None] * \
            (1.0 + a["eps"] * np.cos(th))[None, :]
    elif wl.f0 == "fel_flattop":
        th = g.x_nodes()
        p = g.p_nodes()
        f = (np.abs(p) < a["half_width"]).astype(np.float64)[:, None] * \
            (1.0 + a["eps"] * np.cos(th))[None, :]
    else:
        raise ValueError(f"unknown f0 recipe {wl.f0!r}")
    return normalise(g, f)


# ----------------------------------------------------------------------------
# Concrete workloads. Seeds: 2007122270 (pendulum weights), 2007122271 (batch),
# 2007122272 (serving trace).
# ----------------------------------------------------------------------------
PI = math.pi


def pendulum_128_fp64_tent() -> Workload:
    """Pendulum H = p^2/2 - cos x, 128 x 128, FP64, tent deposition, 200 steps."""
    return Workload(
        name="pendulum_128x128_fp64_tent",
        grid=Grid(128, 128, -PI, PI, -3.0, 3.0),
        pusher=Pusher(PUSH_KDK, POT_PENDULUM, 1.0, 1.0, 0.05),
        basis=BASIS_TENT, precision=FP64, steps=200,
        f0="gaussian", f0_args=dict(xc=0.0, pc=1.0, sx=0.3, sp=0.3))


def pendulum_8192_fp32_cubic(nx: int = 8192, np_: int = 8192, steps: int = 2000) -> Workload:
    """Pendulum, FP32 state, cubic B-spline deposition, trapped + streaming Gaussians."""
    rng = SplitMix64(2007122270)
    c1 = rng.uniform(0.5, 1.5)
    c2 = rng.uniform(0.5, 1.5)
    return Workload(
        name=f"pendulum_{nx}x{np_}_fp32_cubic",
        grid=Grid(nx, np_, -PI, PI, -4.0, 4.0),
        pusher=Pusher(PUSH_KDK, POT_PENDULUM, 1.0, 1.0, 0.02),
        basis=BASIS_CUBIC, precision=FP32, steps=steps,
        f0="two_gaussians",
        f0_args=dict(c1=c1, xc1=0.0, pc1=0.5, s1=0.4, c2=c2, xc2=0.0, pc2=2.5, s2=0.2))


def fel_4096x2048_fp32_cubic(nth: int = 4096, np_: int = 2048, steps: int = 2000,
                             sp: float = 0.05, a0: float = 1e-3) -> Workload:
    """1-D FEL in universal scaling, theta x p = 4096 x 2048, tau = 20."""
    return Workload(
        name=f"fel_{nth}x{np_}_fp32_cubic",
        grid=Grid(nth, np_, 0.0, 2 * PI, -4.0, 4.0),
        pusher=Pusher(PUSH_FEL, POT_FREE, 1.0, 1.0, 0.01, a0, 0.0),
        basis=BASIS_CUBIC, precision=FP32, steps=steps,
        f0="fel_gaussian", f0_args=dict(sp=sp, eps=1e-4))


@dataclass
class BatchInstance:
    workload: Workload


def batch_256(seed: int = 2007122271, count: int = 256, steps: int = 500,
              sizes=(64, 128, 256, 512, 1024, 2048)) -> List[Workload]:
    """Ragged batch: half pendulum, half FEL, square grids drawn per instance."""
    rng = SplitMix64(seed)
    out = []
    for k in range(count):
        n = rng.choice(list(sizes))
        sp = rng.uniform(0.02, 0.2)
        if k % 2 == 0:
            out.append(Workload(
                name=f"batch{k}_pendulum_{n}",
                grid=Grid(n, n, -PI, PI, -4.0, 4.0),
                pusher=Pusher(PUSH_KDK, POT_PENDULUM, 1.0, 1.0, 0.02),
                basis=BASIS_CUBIC, precision=FP32, steps=steps,
                f0="gaussian", f0_args=dict(xc=0.0, pc=1.0, sx=0.3, sp=sp)))
        else:
            a0 = rng.loguniform(1e-4, 1e-2)
            out.append(Workload(
                name=f"batch{k}_fel_{n}",
                grid=Grid(n, n, 0.0, 2 * PI, -4.0, 4.0),
                pusher=Pusher(PUSH_FEL, POT_FREE, 1.0, 1.0, 0.01, a0, 0.0),
                basis=BASIS_CUBIC, precision=FP32, steps=steps,
                f0="fel_gaussian", f0_args=dict(sp=sp, eps=1e-4)))
    return out


@dataclass
class Request:
    rid: int
    arrival: float
    workload: Workload


def serving_trace(seed: int = 2007122272, count: int = 2000, rate: float = 500.0,
                  nmin: int = 128, nmax: int = 4096, smin: int = 100,
                  smax: int = 5000) -> List[Request]:
    """Poisson arrivals of mixed pendulum / FEL solves (log-uniform sizes and lengths)."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(rate)
        n = int(round(rng.loguniform(nmin, nmax)))
        steps = int(round(rng.loguniform(smin, smax)))
        fel = rng.uniform() < 0.5
        sp = rng.uniform(0.02, 0.2)
        if fel:
            a0 = rng.loguniform(1e-4, 1e-2)
            wl = Workload(f"req{k}_fel_{n}", Grid(n, n, 0.0, 2 * PI, -4.0, 4.0),
                          Pusher(PUSH_FEL, POT_FREE, 1.0, 1.0, 0.01, a0, 0.0),
                          BASIS_CUBIC, FP32, steps, "fel_gaussian", dict(sp=sp, eps=1e-4))
        else:
            wl = Workload(f"req{k}_pendulum_{n}", Grid(n, n, -PI, PI, -4.0, 4.0),
                          Pusher(PUSH_KDK, POT_PENDULUM, 1.0, 1.0, 0.02),
                          BASIS_CUBIC, FP32, steps, "gaussian",
                          dict(xc=0.0, pc=1.0, sx=0.3, sp=sp))
        out.append(Request(k, t, wl))
    return out


def with_steps(wl: Workload, steps: int) -> Workload:
    return replace(wl, steps=steps)
