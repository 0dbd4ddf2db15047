"""Writes the oracle regression fixtures in this folder.

Calls only the seeded input generator and the CPU oracle.  The paper prints no
worked example with reproducible numbers (its error tables depend on meshes,
time-step control and tolerances it does not give), so these fixtures record
the oracle's own results on the 2D disc translation workload (periodic in x and
y, the first test case); a change to the oracle's arithmetic shows up here and
must cite the passage that justifies it.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1305_3417_gb300 import inputs as I  # noqa: E402


def disc2d_history():
    w = I.make_workload("disc2d")
    om = O.OracleMesh(w.mesh)
    _, vc, _, _ = om.geometry()
    a = w.alpha0.copy()
    rows = []
    for k in range(w.n_steps):
        F, U, dt = w.step_inputs(k)
        a, st, s = om.advect(a, U, F, dt)
        rows.append((k + 1, (a * vc).sum(), st[O.S["boundary_out"]], st[O.S["min_pre"]], st[O.S["max_pre"]],
                     int(st[O.S["n_interface"]]), int(st[O.S["n_band"]])))
    ex = w.exact(w.n_steps * w.dt)
    l1 = (np.abs(a - ex) * vc).sum()
    return rows, l1, a


def main():
    rows, l1, a = disc2d_history()
    with open(os.path.join(HERE, "disc2d_oracle.txt"), "w") as f:
        f.write("# oracle regression: 2D disc R=0.15 at (0.5,0.75), 32x32x1 periodic in x and y, U=(1,1,0), Co 0.5\n")
        f.write("# written by tests/golden/make_golden.py (oracle + input generator only)\n")
        f.write(f"# L1 = sum V|alpha - exact| after 20 steps: {l1:.17e}\n")
        f.write("# step mass boundary_out min_pre max_pre n_interface n_band\n")
        for r in rows:
            f.write(f"{r[0]} {r[1]:.17e} {r[2]:.17e} {r[3]:.17e} {r[4]:.17e} {r[5]} {r[6]}\n")
    np.savetxt(os.path.join(HERE, "disc2d_oracle_alpha20.txt"), a, fmt="%.17e",
               header="oracle alpha after 20 steps of the periodic 2D disc translation (cell order)")


if __name__ == "__main__":
    main()
