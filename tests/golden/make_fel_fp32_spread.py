"""Writes fel_fp32_spread.json: how far an FP32 state drifts from the FP64 state on the FEL run.

The FEL of Sec. IV.B is an instability: the bunching <exp(-i theta)> and the field A
grow exponentially from the 1e-4 theta modulation of the initial state until
saturation, and every perturbation of that modulation grows with them. This script
runs the FP64 oracle twice on the FEL workload's physics (universal scaling,
dt = 0.01 to tau = 20, cubic B-spline Galerkin) on a 128 x 1024 mesh:

  * as it is (FP64 state), and
  * with its state rounded to FP32 after every step (the field A stays FP64),

and records the relative L1 distance of the two weight arrays at a few step counts
and the largest relative distance of |A|. The second run is the FP64 scheme with
only FP32 storage of the state added, so its distance from the first is a floor for
any FP32 implementation of the scheme: an FP32 GPU run cannot be expected to come
closer to the FP64 oracle than that.

Only the oracle is called. Run: python tests/golden/make_fel_fp32_spread.py
"""
from __future__ import annotations

import json
import os
import sys
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2007_12227_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "fel_fp32_spread.json")
MESH = (128, 1024)
CHECKPOINTS = (200, 500, 1000, 2000)


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def runs(mesh=MESH, checkpoints=CHECKPOINTS):
    """(FP64 snapshots, FP32-rounded snapshots, FP64 |A| history, FP32-rounded |A| history)."""
    wl = I.fel_4096x2048_fp32_cubic(*mesh)
    f0 = I.make_f0(wl).astype(np.float32).astype(np.float64)
    out = {}

    def go(rounded):
        st = O.State(wl.grid, wl.pusher, wl.basis, I.PROJ_GALERKIN, f0)
        snaps, hist, done = {}, [], 0
        for upto in checkpoints:
            if rounded:
                for _ in range(upto - done):
                    hist.append(st.run(1, history=True))
                    st.w[:] = st.w.astype(np.float32).astype(np.float64)
            else:
                hist.append(st.run(upto - done, history=True))
            done = upto
            snaps[upto] = st.w.copy()
        out[rounded] = (snaps, np.hypot(*np.concatenate(hist).reshape(-1, 2).T))

    O.lib()
    th = [threading.Thread(target=go, args=(r,)) for r in (False, True)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return out[False][0], out[True][0], out[False][1], out[True][1]


def spread(mesh=MESH, checkpoints=CHECKPOINTS):
    s64, s32, a64, a32 = runs(mesh, checkpoints)
    return {"mesh": list(mesh), "steps": list(checkpoints),
            "rel_l1_f": [rel_l1(s32[k], s64[k]) for k in checkpoints],
            "max_rel_abs_a": float(np.max(np.abs(a32 - a64) / a64)),
            "max_abs_a": float(a64.max())}


def main():
    res = spread()
    res["_about"] = ("Relative L1 distance between the FP64 oracle and the same oracle with its "
                     "state rounded to FP32 after every step, FEL of Sec. IV.B (universal scaling, "
                     "dt = 0.01 to tau = 20, theta modulation 1e-4, cubic B-spline Galerkin) on a "
                     "128 x 1024 mesh; written by make_fel_fp32_spread.py from the oracle alone")
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
