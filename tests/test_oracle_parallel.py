"""The band-parallel oracle step gives bitwise the serial oracle's step.

The parallel mode exists only to time the oracle on all host cores: it splits the
target rows into bands and keeps the serial order of every addition, so its
weights, field state and lost weight must equal the serial step's exactly, for
any thread count, on every deposit, projection and pusher it supports.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2007_12227_gb300 import inputs as I

PI = math.pi


def cases():
    pend = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.07)
    rot = I.Pusher(I.PUSH_ROTATION, I.POT_HARMONIC, 1.0, 1.3, PI / 10 / 1.3)
    fel = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, 0.05, 0.3, 0.1)
    g1 = I.Grid(67, 53, -PI, PI, -2.0, 2.0)          # the pendulum reaches both momentum edges
    g2 = I.Grid(48, 40, -6.0, 6.0, -6.0, 6.0)
    g3 = I.Grid(64, 57, 0.0, 2 * PI, -1.0, 1.0)
    out = []
    for basis, proj in ((I.BASIS_TENT, I.PROJ_GALERKIN), (I.BASIS_CUBIC, I.PROJ_GALERKIN),
                        (I.BASIS_CUBIC, I.PROJ_LUMPED)):
        out.append(("pendulum", g1, pend, basis, proj, dict(xc=0.3, pc=1.2, sx=0.6, sp=0.7)))
        out.append(("rotation", g2, rot, basis, proj, dict(xc=0.8, pc=-0.3, sx=0.7, sp=0.9)))
        out.append(("fel", g3, fel, basis, proj, dict(xc=1.0, pc=0.2, sx=1.5, sp=0.3)))
    return out


@pytest.mark.parametrize("name,g,pu,basis,proj,args", cases(),
                         ids=[f"{c[0]}-b{c[3]}-p{c[4]}" for c in cases()])
@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_parallel_step_is_bitwise_the_serial_step(name, g, pu, basis, proj, args, threads):
    wl = I.Workload("t", g, pu, basis, I.FP64, 0, "gaussian", args)
    w = I.make_f0(wl)
    fel = None
    if pu.kind == I.PUSH_FEL:
        br, bi = O.bunching(g, w)
        fel = [pu.a0_re, pu.a0_im, br, bi]
    for _ in range(3):
        ws, fs, ls = O.step(g, basis, proj, pu, w, fel)
        wp, fp, lp = O.step_par(g, basis, proj, pu, w, fel, threads=threads)
        assert np.array_equal(ws, wp)
        assert np.array_equal(fs, fp)
        assert ls == lp
        w, fel = ws, fs
    assert ls > 0.0 or name != "pendulum"    # the case exercises the lost-weight order
