"""Study of the unpinned 2D filter readings against Table 2's filtered columns (oracle only, CPU).

For each reading (the one in use, and the alternatives selectable through orc_problem.filter_study)
the oracle runs Example 3.4(a) (isentropic vortex, P^k, 80^2 on [0,10] x [-5,5], periodic, T = 10,
filter on) and prints the domain-normalised L2 error of density at the k+1 Gauss points per
direction next to the printed "with filter" value of Table 2.

Usage: python -m oracle.study_table2_filter [threads]. About an hour on 8 cores.
"""
import json
import os
import sys
import time

import oracle as O

PRINTED = {1: 6.26e-03, 2: 1.23e-03, 3: 1.65e-03}      # Table 2, 80^2, L2 with filter
STUDIES = {0: "readings in use (beta and Hbar at the average, max of the combined x + y sum)",
           1: "beta^x, beta^y: largest over the cell's Gauss points",
           2: "Hbar: cell average of H",
           4: "max over components per direction, the two added"}
VORTEX = [5.0, 0.0, 5.0, 0.0]


def run(k, study, n=80):
    p = O.Problem(dim=2, nx=n, ny=n, x0=0.0, x1=10.0, y0=-5.0, y1=5.0, k=k, eq=O.EQ_EULER, basis=O.BASIS_P,
                  bc=(O.BC_PERIODIC,) * 4, filter=1, filter_study=study)
    u0 = O.project(p, O.IC_VORTEX2D, VORTEX)
    u, t, steps = O.advance(p, u0, 0.0, 10.0)
    _, l2, _ = O.errors(p, u, O.EX_VORTEX2D, VORTEX[:3], t, var=0, nq_err=k + 1)
    return l2 / 10.0, steps


if __name__ == "__main__":
    O.set_threads(int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1))
    for study, what in STUDIES.items():
        for k in (1, 2, 3):
            t0 = time.time()
            l2, steps = run(k, study)
            print(json.dumps({"study": study, "reading": what, "k": k, "l2": l2, "printed": PRINTED[k],
                              "ratio_to_printed": l2 / PRINTED[k], "steps": steps,
                              "seconds": round(time.time() - t0, 1)}), flush=True)
