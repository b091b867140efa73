"""dg_step_noalloc, the entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc where they want a step (stream capture, a
framework-owned memory arena, latency-critical loops); its stage states live in a static device
array. Checked here through the C ABI against the allocating path (dg_create / dg_step /
dg_read_state) on the same input, for two calls in a row, and for its size limit.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("case", ["euler2d_q2", "burgers1d_p3"])
def test_noalloc_matches_allocating_path_two_calls(case):
    import torch

    from paper_2407_19169_gb300 import _native as N
    from paper_2407_19169_gb300 import inputs as I

    L = N.load()
    if case == "euler2d_q2":
        kw = dict(dim=2, nx=64, ny=40, x0=0.0, x1=1.0, y0=0.0, y1=0.625, bc=(N.BC_OUTFLOW,) * 4, k=2,
                  eq=N.EQ_EULER)
        shape = (4, 9, 64 * 40)
        u0 = I.random_modal_state(shape, 91, I.EULER2D_AVG, high_scale=0.02)
    else:
        kw = dict(dim=1, nx=300, ny=1, x0=0.0, x1=2.0, y0=0.0, y1=1.0, bc=(N.BC_PERIODIC,) * 4, k=3,
                  eq=N.EQ_BURGERS)
        shape = (1, 4, 300)
        u0 = I.random_modal_state(shape, 92, [(-0.5, 1.5)])

    # the allocating path
    s = N.Solver(**kw)
    s.write_state(u0, 0.0)
    dts = [s.step()]
    ref1, _ = s.read_state()
    dts.append(s.step())
    ref2, _ = s.read_state()
    s.close()

    # the allocation-free path on the caller's device buffers
    mesh = N.Mesh(kw["dim"], kw["nx"], kw["ny"], kw["x0"], kw["x1"], kw["y0"], kw["y1"], (C.c_int * 4)(*kw["bc"]))
    prm = N.Params()
    assert L.dg_params_default(C.byref(prm)) == 0
    a = torch.tensor(u0.ravel(), dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    stream = torch.cuda.current_stream().cuda_stream
    dt = C.c_double()
    for src, dst, ref, dt_ref in ((a, b, ref1, dts[0]), (b, c, ref2, dts[1])):
        st = L.dg_step_noalloc(C.byref(mesh), kw["k"], kw["eq"], C.byref(prm), C.c_void_p(src.data_ptr()),
                               C.c_void_p(dst.data_ptr()), C.byref(dt), C.c_void_p(stream))
        assert st == 0, N.STATUS.get(st, st)
        got = dst.cpu().numpy().reshape(shape)
        assert dt.value == pytest.approx(dt_ref, rel=1e-15)
        assert _rel_l1(got, ref) <= 1e-11


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
