"""Writes the oracle regression snapshot ``hopper_fp64_seed0.txt``.

It calls only ``oracle/`` (and the shared seeded generator).  The paper prints
no worked numeric example for the discretization (Sec. VI reports settings and
solve times only), so nothing here is a value from the paper: the snapshot only
guards the pinned oracle against unintended changes.  A deliberate change to
the oracle's arithmetic regenerates it, and the commit names the passage that
justifies the change.

Usage: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2604_09993_gb300 import synth  # noqa: E402


def snapshot():
    p = synth.hopper_fp64(seed=0)
    o = oracle.discretize(p.robot.as_dict(), p.X, p.U, p.s, p.n_sub, threads=1)
    rows = []
    for k in (0, 4, 9):
        rows.append(("defect", k, o["defect"][k]))
        rows.append(("penalty", k, o["penalty"][k]))
        rows.append(("S", k, o["S"][k]))
        rows.append(("A_theta_rows", k, o["A"][k][[2, 5, 8], :].reshape(-1)))
        rows.append(("Bm_omega_rows", k, o["Bm"][k][[11, 14, 17], :].reshape(-1)))
        rows.append(("Bp_y_row", k, o["Bp"][k][18, :]))
    return rows


if __name__ == "__main__":
    with open(os.path.join(HERE, "hopper_fp64_seed0.txt"), "w") as f:
        f.write("# oracle snapshot: hopper, N=10, n_sub=4, seed 0 (tests/golden/make_golden.py)\n")
        for name, k, v in snapshot():
            f.write(f"{name} {k} " + " ".join(repr(float(x)) for x in v) + "\n")
