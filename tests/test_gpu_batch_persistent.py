"""Persistent batched stepping (dg_batch_run_persistent): one cooperative launch per class runs every
step, with per-instance stage barriers on device counters. Each result must equal the graph-replayed
batched run (dg_batch_run) and the same solve stepped alone, bit for bit up to 1e-12."""
import numpy as np
import pytest

from paper_2407_19169_gb300 import _native as N
from paper_2407_19169_gb300 import inputs as I
from test_gpu_batch import SPECS, make, rel

pytestmark = pytest.mark.gpu

# the batch test mix plus instances with the positivity limiter (their own 2D and 1D classes)
MIX = SPECS + [dict(kind="quadrant2d", n=48, k=2, seed=3, pos=1), dict(kind="quadrant2d", n=30, k=3, seed=5, pos=1),
               dict(kind="riemann1d", n=700, k=2, seed=6, pos=1)]


def test_persistent_equals_graph_and_alone():
    steps = 25
    a = [make(sp) for sp in MIX]
    b = [make(sp) for sp in MIX]
    l0 = a[0].kernel_launches()
    assert N.batch_run(a, steps, persistent=True) == 0
    classes = len({(sp["kind"].endswith("2d"), sp["k"], sp.get("pos", 0) if sp["kind"].endswith("2d") else 0)
                   for sp in MIX})
    assert a[0].kernel_launches() - l0 == 1 + classes        # the begin kernel and one launch per class
    assert N.batch_run(b, steps) == 0
    for sp, sa, sb in zip(MIX, a, b):
        ua, ta = sa.read_state()
        ub, tb = sb.read_state()
        st, _, n = sa.sync()
        assert st == 0 and n == steps, sp
        assert ta == tb, sp
        assert rel(ua, ub) <= 1e-12, (sp, rel(ua, ub))
        alone = make(sp)
        alone.advance_steps(steps)
        uo, to = alone.read_state()
        assert to == ta and rel(ua, uo) <= 1e-12, (sp, rel(ua, uo))


def test_persistent_per_instance_end_times():
    """Instances stop at their own T inside one launch; finished instances' items are skipped."""
    mix = [make(sp) for sp in SPECS[:6]]
    ends = [0.002, 0.004, 0.003, 0.0005, 0.01, 0.02]
    for s, T in zip(mix, ends):
        s.set_target(T)
    assert N.batch_run(mix, 400, persistent=True) == 0
    for sp, s, T in zip(SPECS[:6], mix, ends):
        ub, tb = s.read_state()
        assert tb == T
        alone = make(sp)
        alone.advance_to(T)
        ua, ta = alone.read_state()
        assert ta == T and rel(ub, ua) <= 1e-12


def test_persistent_failure_is_isolated():
    good = make(SPECS[4])
    bad = N.Solver(dim=2, nx=40, ny=40, k=1, eq=N.EQ_EULER, bc=(N.BC_PERIODIC,) * 4, precision=N.PREC_FP32_MIXED)
    u = I.random_modal_state(bad.shape, 3, I.EULER2D_AVG, high_scale=0.02)
    u[3, 0, 777] = -5.0                               # negative energy in one cell
    bad.write_state(u)
    assert N.batch_run([good, bad], 10, persistent=True) == -4
    st_bad = bad.sync()[0]
    st_good, t_good, n_good = good.sync()
    assert st_bad == -4 and st_good == 0 and n_good == 10
    alone = make(SPECS[4])
    alone.advance_steps(10)
    assert alone.sync()[0] == 0
    assert rel(good.read_state()[0], alone.read_state()[0]) <= 1e-12


def test_persistent_rejects_unsupported():
    s64 = N.Solver(dim=1, nx=50, k=1, eq=N.EQ_EULER, precision=N.PREC_FP64)
    assert N.batch_run([s64], 1, persistent=True) == -8


def test_bounded_wait_gives_up():
    """The persistent kernels' wait on a counter that nothing releases ends after its poll limit with
    the timeout status, and the context stays usable."""
    import ctypes as C
    L = N.load()
    status, ms = C.c_uint(0), C.c_double(0.0)
    assert L.dg_probe_wait_timeout(20000, C.byref(status), C.byref(ms)) == 0
    assert status.value == 1
    assert 0.0 < ms.value < 1000.0
    s = make(SPECS[0])
    assert N.batch_run([s], 3, persistent=True) == 0
    assert s.sync()[:1] == (0,) and s.sync()[2] == 3
