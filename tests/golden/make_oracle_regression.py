"""Writes tests/golden/oracle_regression_small.txt: FP64 oracle outputs on
fixed small workloads, read back by tests/test_oracle_golden.py.

The paper prints no worked numerical example (its Sec. 5 reports scaling runs
only), so these are regression values, not independent pins: they hold the
oracle to what it computes now, so that a change of its arithmetic shows up
and has to name the passage that justifies it.  The independent pins (closed
forms of Sec. 2.3, the group laws of Sec. 2.4, brute-force integration) are
in tests/test_oracle_pins.py and tests/test_oracle_shell_pins.py.

Run from the repository root: python tests/golden/make_oracle_regression.py
It calls only oracle/ and the seeded input generators.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1809_01334_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression_small.txt")
PIXELS = [(0, 0), (5, 17), (31, 31), (32, 32), (40, 9), (63, 63), (12, 50), (50, 12)]


def cases():
    """(name, forest, tf, camera, integrator, rows) of the fixed workloads."""
    f, tf, cam, integ = I.preset_c1()  # Sec. 2.3 RK4 (Eq. 2.31), 4 steps per segment
    yield "c1_rk4", f, tf, cam, integ
    yield "c1_dopri5", f, tf, cam, {"method": "dopri5", "tol": 1e-6, "c_rk": 0.5, "max_depth": 16}
    f, tf, cam = I.preset_shell_small()  # cubed-sphere shell, levels 1..3
    yield "shell_small_dopri5", f, tf, cam, {"method": "dopri5", "tol": 1e-5, "c_rk": 0.5,
                                             "max_depth": 16}


def compute():
    rows = []
    for name, f, tf, cam, integ in cases():
        px = [(i % cam.w, j % cam.h) for i, j in PIXELS]
        need = sorted({j for _, j in px})
        r = O.render(f, tf, cam, integ, rows=np.array(need, np.int32))
        at = {j: k for k, j in enumerate(need)}
        for i, j in px:
            v = r["rgba"][at[j], i]
            rows.append((name, i, j, int(r["counts"][at[j], i]), *map(float, v)))
    return rows


def main():
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle regression values (see make_oracle_regression.py); index\n")
        fh.write("# decisions (visibility, rays, segment end points) in FP32, values in FP64.\n")
        fh.write("# case i j segments r g b alpha\n")
        for name, i, j, n, r, g, b, a in compute():
            fh.write(f"{name} {i} {j} {n} {r:.17g} {g:.17g} {b:.17g} {a:.17g}\n")
    print(OUT)


if __name__ == "__main__":
    main()
