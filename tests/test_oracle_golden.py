"""The FP64 oracle against its stored regression values
(tests/golden/oracle_regression_small.txt, written by
tests/golden/make_oracle_regression.py from the oracle alone): segment counts
exactly, RGBA within 1e-12 (host math libraries may differ in the last bits).
These hold the oracle to its current arithmetic; the independent pins are in
test_oracle_pins.py and test_oracle_shell_pins.py."""
import os

import numpy as np

from tests.golden.make_oracle_regression import OUT, compute


def test_oracle_matches_stored_regression_values():
    stored = {}
    with open(OUT) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            f = line.split()
            stored[(f[0], int(f[1]), int(f[2]))] = (int(f[3]), np.array([float(x) for x in f[4:8]]))
    assert len(stored) == 24
    for name, i, j, n, *v in compute():
        sn, sv = stored[(name, i, j)]
        assert n == sn, (name, i, j)
        assert np.abs(np.array(v) - sv).max() <= 1e-12, (name, i, j)
