"""Screen seeded four-quadrant Riemann problems and write quadrant_seeds.txt.

A seed is accepted when the FP64 oracle (Q2, LLF, SSP-RK3, jump filter, CFL 0.1, outflow) on a 64x64
mesh of [0,1]^2 reaches T = 0.25 with every cell average physical (the scheme has no positivity
limiter, so seeds that create near-vacuum states are rejected up front). Calls only oracle/ and the
seeded input generator.
Run: python tests/golden/make_quadrant_seeds.py [first last]
"""
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def screen(seed):
    import oracle as O
    from paper_2407_19169_gb300 import inputs as I
    O.set_threads(1)
    p = O.Problem(dim=2, nx=64, ny=64, x0=0, x1=1, y0=0, y1=1, k=2, eq=O.EQ_EULER, bc=(O.BC_OUTFLOW,) * 4)
    u = O.project(p, O.IC_QUADRANT2D, I.quadrant_params(seed))
    try:
        _, t, n = O.advance(p, u, 0.0, 0.25)
        return seed, True, n
    except FloatingPointError:
        return seed, False, 0


if __name__ == "__main__":
    a, b = (int(sys.argv[1]), int(sys.argv[2])) if len(sys.argv) > 2 else (1, 24)
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(screen, range(a, b + 1))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "quadrant_seeds.txt")
    with open(out, "w") as f:
        f.write("# seed accepted steps_to_T (64x64 Q2 oracle, T=0.25); written by make_quadrant_seeds.py\n")
        for s, ok, n in res:
            f.write("%d %d %d\n" % (s, int(ok), n))
    print(open(out).read())
