"""Batched stepping (dg_batch_run): uneven 1D/2D Euler instances of degrees 1-3 advanced together in
one graph-captured work-list launch per stage. Each result must equal the same solve stepped alone.
"""
import numpy as np
import pytest

from paper_2407_19169_gb300 import _native as N
from paper_2407_19169_gb300 import inputs as I

pytestmark = pytest.mark.gpu
F32 = N.PREC_FP32_MIXED


def make(spec):
    kind, n, k = spec["kind"], spec["n"], spec["k"]
    pos = spec.get("pos", 0)
    if kind == "riemann1d":
        s = N.Solver(dim=1, nx=n, k=k, eq=N.EQ_EULER, bc=(N.BC_OUTFLOW,) * 4, precision=F32,
                     positivity=pos)
        s.set_initial(N.IC_RIEMANN1D, I.riemann1d_params(spec["seed"]))
    elif kind == "entropy1d":
        s = N.Solver(dim=1, nx=n, k=k, eq=N.EQ_EULER, bc=(N.BC_PERIODIC,) * 4, precision=F32)
        s.set_initial(N.IC_ENTROPY1D, [1.0, 0.2, 2 * np.pi, 1.0, 1.0])
    elif kind == "quadrant2d":
        s = N.Solver(dim=2, nx=n, ny=n, k=k, eq=N.EQ_EULER, bc=(N.BC_OUTFLOW,) * 4, precision=F32,
                     positivity=pos)
        s.set_initial(N.IC_QUADRANT2D, I.quadrant_params(spec["seed"]))
    else:
        s = N.Solver(dim=2, nx=n, ny=n, x0=0, x1=10, y0=-5, y1=5, k=k, eq=N.EQ_EULER,
                     bc=(N.BC_PERIODIC,) * 4, precision=F32)
        s.set_initial(N.IC_VORTEX2D, [5.0, 0.0, 5.0, 0.0])
    return s


SPECS = [
    dict(kind="riemann1d", n=1000, k=1, seed=1), dict(kind="riemann1d", n=3000, k=3, seed=2),
    dict(kind="entropy1d", n=517, k=2), dict(kind="riemann1d", n=20000, k=2, seed=4),
    dict(kind="quadrant2d", n=64, k=2, seed=1), dict(kind="vortex2d", n=70, k=1),
    dict(kind="quadrant2d", n=96, k=3, seed=4), dict(kind="vortex2d", n=130, k=2),
    dict(kind="quadrant2d", n=34, k=1, seed=7),   # even: the split x = 0.5 lies on a face
]


def rel(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def test_batch_equals_alone():
    steps = 25
    mix = [make(sp) for sp in SPECS]
    assert N.batch_run(mix, steps) == 0
    for sp, sb in zip(SPECS, mix):
        alone = make(sp)
        alone.advance_steps(steps)
        st, t_alone, n_alone = alone.sync()
        assert st == 0 and n_alone == steps
        ua, _ = alone.read_state()
        ub, tb = sb.read_state()
        assert tb == t_alone, sp
        assert rel(ub, ua) <= 1e-12, (sp, rel(ub, ua))


def test_batch_against_the_oracle():
    """A batched mix (1D and 2D, degrees 1-3, one dg_batch_run) against the FP64 oracle: smooth
    instances within the FP32 form's 1e-5 relative L1; the 1D Riemann instance's L1 density error
    against the exact solution within 2% of the oracle's own error at the same step count."""
    import math

    import oracle as O
    from _helpers import rel_l1
    steps = 30
    specs = [dict(kind="entropy1d", n=160, k=2), dict(kind="vortex2d", n=40, k=1),
             dict(kind="vortex2d", n=28, k=3), dict(kind="riemann1d", n=400, k=3, seed=1),
             dict(kind="entropy1d", n=90, k=3)]
    mix = [make(sp) for sp in specs]
    u0s = [s.read_state()[0] for s in mix]
    assert N.batch_run(mix, steps) == 0
    for sp, s, u0 in zip(specs, mix, u0s):
        ub, tb = s.read_state()
        if sp["kind"] == "entropy1d":
            p = O.Problem(dim=1, nx=sp["n"], k=sp["k"], eq=O.EQ_EULER, bc=(O.BC_PERIODIC,) * 4)
        elif sp["kind"] == "vortex2d":
            p = O.Problem(dim=2, nx=sp["n"], ny=sp["n"], x0=0, x1=10, y0=-5, y1=5, k=sp["k"],
                          eq=O.EQ_EULER, bc=(O.BC_PERIODIC,) * 4)
        else:
            p = O.Problem(dim=1, nx=sp["n"], k=sp["k"], eq=O.EQ_EULER, bc=(O.BC_OUTFLOW,) * 4)
        uo, to, no = O.advance(p, u0, 0.0, math.inf, steps)
        assert no == steps
        if sp["kind"] == "riemann1d":
            prm = I.riemann1d_params(sp["seed"])
            eb = O.errors(p, ub, O.EX_RIEMANN1D, prm, tb, var=0)[0]
            eo = O.errors(p, uo, O.EX_RIEMANN1D, prm, to, var=0)[0]
            assert abs(eb - eo) <= 0.02 * eo, (sp, eb, eo)
        else:
            assert abs(tb - to) <= 1e-6 * to
            assert rel_l1(p, ub, uo) <= 1e-5, (sp, rel_l1(p, ub, uo))


def test_batch_per_instance_end_times():
    mix = [make(sp) for sp in SPECS[:6]]
    ends = [0.002, 0.004, 0.003, 0.0005, 0.01, 0.02]
    for s, T in zip(mix, ends):
        s.set_target(T)
    # more steps than any instance needs: finished instances idle
    assert N.batch_run(mix, 400) == 0
    for sp, s, T in zip(SPECS[:6], mix, ends):
        ub, tb = s.read_state()
        assert tb == T
        alone = make(sp)
        alone.advance_to(T)
        ua, ta = alone.read_state()
        assert ta == T and rel(ub, ua) <= 1e-12


def test_batch_failure_is_isolated():
    good = make(SPECS[4])
    bad = N.Solver(dim=2, nx=40, ny=40, k=1, eq=N.EQ_EULER, bc=(N.BC_PERIODIC,) * 4, precision=F32)
    u = I.random_modal_state(bad.shape, 3, I.EULER2D_AVG, high_scale=0.02)
    u[3, 0, 777] = -5.0                               # negative energy in one cell
    bad.write_state(u)
    assert N.batch_run([good, bad], 10) == -4
    st_bad = bad.sync()[0]
    st_good, t_good, n_good = good.sync()
    assert st_bad == -4 and st_good == 0 and n_good == 10
    alone = make(SPECS[4])
    alone.advance_steps(10)
    assert alone.sync()[0] == 0
    assert rel(good.read_state()[0], alone.read_state()[0]) <= 1e-12


def test_batch_rejects_unsupported():
    s64 = N.Solver(dim=1, nx=50, k=1, eq=N.EQ_EULER, precision=N.PREC_FP64)
    assert N.batch_run([s64], 1) == -8
