"""Screen seeded 1D Riemann problems and write riemann1d_seeds.txt.

A seed is accepted when the exact solution has no vacuum (2 (cL + cR)/(gamma - 1) > uR - uL), its
minimum pressure is at least 0.05, and the FP64 oracle (P3, LLF, SSP-RK3, jump filter, CFL 0.1,
outflow) on 256 cells of [0,1] reaches T = 0.2 with every cell average physical. Calls only oracle/
and the seeded input generator. Run: python tests/golden/make_riemann1d_seeds.py [first last]
"""
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def screen(seed):
    import numpy as np
    import oracle as O
    from paper_2407_19169_gb300 import inputs as I
    O.set_threads(1)
    prm = I.riemann1d_params(seed)
    try:
        W = np.array([O.riemann_exact(1.4, prm[0:3], prm[3:6], xi) for xi in np.linspace(-20, 20, 4001)])
    except ValueError:
        return seed, False, 0
    if W[:, 2].min() < 0.05:
        return seed, False, 0
    p = O.Problem(dim=1, nx=256, k=3, eq=O.EQ_EULER, bc=(O.BC_OUTFLOW,) * 4)
    u = O.project(p, O.IC_RIEMANN1D, prm)
    try:
        _, t, n = O.advance(p, u, 0.0, 0.2)
        return seed, True, n
    except FloatingPointError:
        return seed, False, 0


if __name__ == "__main__":
    a, b = (int(sys.argv[1]), int(sys.argv[2])) if len(sys.argv) > 2 else (1, 32)
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(screen, range(a, b + 1))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "riemann1d_seeds.txt")
    with open(out, "w") as f:
        f.write("# seed accepted steps_to_T (256-cell P3 oracle, T=0.2); written by make_riemann1d_seeds.py\n")
        for s, ok, n in res:
            f.write("%d %d %d\n" % (s, int(ok), n))
    print(open(out).read())
