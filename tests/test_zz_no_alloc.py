"""dg_step_noalloc, the entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc where they want a step (stream capture, a
framework-owned memory arena, latency-critical loops); its stage states live in a static device
array. Checked here through the C ABI against the allocating path (dg_create / dg_step /
dg_read_state) on the same input, for two calls in a row: with the positivity limiter off and on
(the limiter moves the CFL rate to its points, so dt depends on the per-mode geometry and the Gauss
rules that the entry point sets up for itself), once in a fresh process whose first library call is
dg_step_noalloc, and for its size limit.
"""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def _case(N, I, case):
    """(solver keywords, state shape, initial state, positivity) of a named case."""
    if case == "euler2d_q2":
        kw = dict(dim=2, nx=64, ny=40, x0=0.0, x1=1.0, y0=0.0, y1=0.625, bc=(N.BC_OUTFLOW,) * 4, k=2,
                  eq=N.EQ_EULER)
        shape = (4, 9, 64 * 40)
        return kw, shape, I.random_modal_state(shape, 91, I.EULER2D_AVG, high_scale=0.02), 0
    if case == "burgers1d_p3":
        kw = dict(dim=1, nx=300, ny=1, x0=0.0, x1=2.0, y0=0.0, y1=1.0, bc=(N.BC_PERIODIC,) * 4, k=3,
                  eq=N.EQ_BURGERS)
        shape = (1, 4, 300)
        return kw, shape, I.random_modal_state(shape, 92, [(-0.5, 1.5)]), 0
    if case == "euler2d_q2_quadrant_limiter":
        # seeded four-quadrant data after 30 steps of the allocating path: near-vacuum cells where
        # the positivity limiter acts and its points set the CFL rate
        kw = dict(dim=2, nx=40, ny=40, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=(N.BC_OUTFLOW,) * 4, k=2,
                  eq=N.EQ_EULER)
        s = N.Solver(positivity=1, **kw)
        s.set_initial(N.IC_QUADRANT2D, I.quadrant_params(3))
        s.advance_steps(30)
        assert s.sync()[0] == 0
        u0, _ = s.read_state()
        s.close()
        return kw, u0.shape, u0, 1
    if case == "euler1d_p3_limiter":
        kw = dict(dim=1, nx=70, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=(N.BC_PERIODIC,) * 4, k=3,
                  eq=N.EQ_EULER)
        shape = (3, 4, 70)
        # rough cells near vacuum made admissible by the oracle's limiter (as the limiter's parity
        # test does); the limiter then acts in the steps and its points set the CFL rate
        import oracle as O
        p = O.Problem(dim=1, nx=70, k=3, eq=O.EQ_EULER, bc=(O.BC_PERIODIC,) * 4, positivity=1)
        u0 = I.random_modal_state(shape, 74, [(0.5, 1.0), (-0.2, 0.2), (1.0, 2.0)], high_scale=0.4, decay=0.6)
        return kw, shape, O.positivity(p, u0), 1
    raise KeyError(case)


def _check_two_calls(case):
    """The allocation-free step twice in a row against dg_step twice: dt to 1e-15, state to 1e-11."""
    import torch

    from paper_2407_19169_gb300 import _native as N
    from paper_2407_19169_gb300 import inputs as I

    L = N.load()
    kw, shape, u0, pos = _case(N, I, case)

    # the allocation-free path first: in a fresh process it is then the first library call
    mesh = N.Mesh(kw["dim"], kw["nx"], kw["ny"], kw["x0"], kw["x1"], kw["y0"], kw["y1"], (C.c_int * 4)(*kw["bc"]))
    prm = N.Params()
    assert L.dg_params_default(C.byref(prm)) == 0
    prm.positivity = pos
    a = torch.tensor(np.ascontiguousarray(u0).ravel(), dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    stream = torch.cuda.current_stream().cuda_stream
    dt = C.c_double()
    got, dts = [], []
    for src, dst in ((a, b), (b, c)):
        st = L.dg_step_noalloc(C.byref(mesh), kw["k"], kw["eq"], C.byref(prm), C.c_void_p(src.data_ptr()),
                               C.c_void_p(dst.data_ptr()), C.byref(dt), C.c_void_p(stream))
        assert st == 0, N.STATUS.get(st, st)
        got.append(dst.cpu().numpy().reshape(shape))
        dts.append(dt.value)

    # the allocating path on the same input
    s = N.Solver(positivity=pos, **kw)
    s.write_state(np.ascontiguousarray(u0), 0.0)
    for i in range(2):
        dt_ref = s.step()
        ref, _ = s.read_state()
        assert dts[i] == pytest.approx(dt_ref, rel=1e-15)
        assert _rel_l1(got[i], ref) <= 1e-11
    s.close()


@pytest.mark.parametrize("case", ["euler2d_q2", "burgers1d_p3", "euler2d_q2_quadrant_limiter",
                                  "euler1d_p3_limiter"])
def test_noalloc_matches_allocating_path_two_calls(case):
    _check_two_calls(case)


def test_noalloc_first_call_in_a_fresh_process():
    # no dg_create before it: the entry point's own per-device set-up must load the Gauss rules
    # that the CFL rate at the limiter's points reads
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
            "import test_zz_no_alloc as T\n"
            "T._check_two_calls('euler1d_p3_limiter')\n"
            "print('fresh ok')\n") % (ROOT, os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_noalloc_rejects_meshes_beyond_its_array():
    from paper_2407_19169_gb300 import _native as N

    L = N.load()
    mesh = N.Mesh(2, 2048, 2048, 0.0, 1.0, 0.0, 1.0, (C.c_int * 4)(1, 1, 1, 1))
    prm = N.Params()
    assert L.dg_params_default(C.byref(prm)) == 0
    # two FP64 stage states of a 2048^2 Q2 Euler mesh need 2.4 GB: refused before any launch
    st = L.dg_step_noalloc(C.byref(mesh), 2, N.EQ_EULER, C.byref(prm), C.c_void_p(16), C.c_void_p(32),
                           None, None)
    assert st == -3
    prm.precision = N.PREC_FP32_MIXED
    small = N.Mesh(1, 64, 1, 0.0, 1.0, 0.0, 1.0, (C.c_int * 4)(0, 0, 0, 0))
    st = L.dg_step_noalloc(C.byref(small), 2, N.EQ_BURGERS, C.byref(prm), C.c_void_p(16), C.c_void_p(32),
                           None, None)
    assert st == -8
