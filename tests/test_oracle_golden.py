"""The oracle reproduces its committed regression snapshot (no GPU)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_snapshot(oracle_mod):
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden
    want = {}
    for line in open(os.path.join(HERE, "golden", "hopper_fp64_seed0.txt")):
        if line.startswith("#"):
            continue
        name, k, *vals = line.split()
        want[(name, int(k))] = np.array([float(v) for v in vals])
    got = make_golden.snapshot()
    assert len(got) == len(want)
    for name, k, v in got:
        ref = want[(name, k)]
        assert np.allclose(v, ref, rtol=1e-13, atol=1e-15), (name, k)
